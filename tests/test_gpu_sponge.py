"""GPU sponge term (ps_set_sponge) against the oracle step with the same
sponge (Sec. 4.1, Eq. penalized Navier--Stokes, the vorticity damping term;
damping reading, see ``oracle.step``)."""
import math

import numpy as np
import pytest
import torch

from oracle import mask as OM
from oracle import step as S
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def sponge_mask(n, L):
    """1 in slabs at the x faces of the box, a smooth ramp inside them."""
    x = np.arange(n) * (L / n)
    d = np.minimum(x, L - x) / L
    prof = np.clip((0.2 - d) / 0.1, 0.0, 1.0)
    return np.broadcast_to(prof[:, None, None], (n, n, n)).copy()


@pytest.mark.parametrize("n,prec,tol", [(32, "fp64", 1e-12), (48, "fp64", 1e-12), (32, "fp32", 2e-5),
                                        (48, "fp32", 2e-5)])
def test_sponge_step_matches_oracle(n, prec, tol):
    L, nu, eta, dt, c_sp = 4.0, 1.527e-4, 1e-2, 5e-4, 0.05
    dx = L / n
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xw0, tri = inputs.elliptic_wing_mesh(300)
    xw, vw, fr = inputs.revolving_wing(0.2, xw0, inputs.flapping_amplitudes(xw0))
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
    u = inputs.random_field(n, L, seed=n + 5, rms=0.3)
    csp = sponge_mask(n, L)
    o = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0)))
    o.set_velocity(u)
    o.set_mask(chi, us)
    o.set_sponge(csp, c_sp)
    g = Solver(n, L, nu, eta, dt, precision=prec, x0=(2.0, 2.0, 2.0))
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi, dtype), dev(us, dtype))
    csp_d = dev(csp, dtype)
    g.set_sponge(csp_d, c_sp)
    o.step(3)
    g.step(3)
    got = g.velocity().double().cpu().numpy()
    v = o.velocity()
    err = np.linalg.norm(got - v) / np.linalg.norm(v)
    F, M = g.forces()
    ef = np.linalg.norm(np.array(F) - o.F) / np.linalg.norm(o.F)
    print("%s n=%d sponge step: rel L2 %.2e, force %.2e" % (prec, n, err, ef))
    assert err < tol
    assert ef < (1e-10 if prec == "fp64" else 1e-4)
    # the sponge changes the answer (it is on) ...
    o2 = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0)))
    o2.set_velocity(u)
    o2.set_mask(chi, us)
    o2.step(3)
    assert np.linalg.norm(o2.velocity() - v) > 100 * tol * np.linalg.norm(v)
    # ... and turning it off gives the plain step again
    g.set_sponge(None)
    g.set_velocity(dev(u, dtype))
    g.step(3)
    err2 = np.linalg.norm(g.velocity().double().cpu().numpy() - o2.velocity()) / np.linalg.norm(o2.velocity())
    assert err2 < tol


def test_uniform_sponge_taylor_green_recurrence():
    """chi_sp = 1: the sponge term is -u/C_sp and the 2-D Taylor-Green
    amplitude follows the scalar IF-AB2 recurrence (FP64, 48^3 = 3 x 16)."""
    n, L, nu, dt, c_sp, K = 48, 2 * math.pi, 0.02, 1e-2, 0.5, 10
    g = Solver(n, L, nu, 1.0, dt, precision="fp64")
    u0 = inputs.taylor_green_2d(n, L)
    g.set_velocity(dev(u0, torch.float64))
    ones = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
    g.set_sponge(ones, c_sp)
    g.step(K)
    E = math.exp(-nu * 2.0 * dt)
    a_prev, a = None, 1.0
    for k in range(K):
        N = -a / c_sp
        new = E * (a + dt * N) if k == 0 else E * a + 0.5 * dt * (3 * E * N - E * E * (-a_prev / c_sp))
        a_prev, a = a, new
    assert np.max(np.abs(g.velocity().cpu().numpy() - a * u0)) < 1e-12
