"""GPU pressure and pressure loads (ps_pressure, ps_pressure_loads) against
the oracle (Sec. 4.1: total pressure of the rotational form, delta
interpolation to the mass points, per-triangle p A/3 normal loads)."""
import math

import numpy as np
import pytest
import torch

from oracle import mask as OM
from oracle import pressure as OP
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


def _case(n, nodes=300):
    L, nu, eta, dt = 4.0, 1.527e-4, 1e-2, 5e-4
    dx = L / n
    xw0, tri = inputs.elliptic_wing_mesh(nodes)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0))
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
    u = inputs.random_field(n, L, seed=n + 11, rms=0.3)
    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0))
    return p, u, chi, us, xw, tri, fr


@pytest.mark.parametrize("n,prec,tol", [(32, "fp64", 1e-11), (32, "fp32", 2e-5), (48, "fp64", 1e-11),
                                        (48, "fp32", 2e-5), (12, "fp64", 1e-11), (24, "fp32", 2e-5)])
def test_pressure_matches_oracle(n, prec, tol):
    p, u, chi, us, xw, tri, fr = _case(n)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    o = S.Solver(p)
    o.set_velocity(u)
    o.set_mask(chi, us)
    o.step(2)
    g = Solver(n, p.L, p.nu, p.eta, p.dt, precision=prec, x0=p.x0)
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi, dtype), dev(us, dtype))
    g.step(2)
    F0, M0 = g.forces()
    v0 = g.velocity().clone()
    got = g.pressure().double().cpu().numpy()
    want = OP.static_pressure(p, o.uh, chi, us)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    print("%s n=%d pressure max rel err %.2e" % (prec, n, err))
    assert err < tol
    # the state and the last step's forces are left as they were
    F1, M1 = g.forces()
    assert F1 == F0 and M1 == M0
    assert torch.equal(g.velocity(), v0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pressure_loads_match_oracle(prec):
    n = 32
    p, u, chi, us, xw, tri, fr = _case(n)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    g = Solver(n, p.L, p.nu, p.eta, p.dt, precision=prec, x0=p.x0)
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi, dtype), dev(us, dtype))
    pf = g.pressure()
    pn, fn = g.pressure_loads(pf, dev(xw, torch.float64), dev(tri, torch.int32), fr)
    pfh = pf.double().cpu().numpy()
    xg = OM.global_nodes(xw, fr)
    pn_o = OP.interpolate(pfh, p.L, xg)
    fn_o = OP.node_loads(pn_o, xg, tri)
    assert np.max(np.abs(pn.cpu().numpy() - pn_o)) < 1e-12 * np.max(np.abs(pn_o))
    assert np.max(np.abs(fn.cpu().numpy() - fn_o)) < 1e-12 * np.max(np.abs(fn_o))
    # the total load equals -sum_v p_v sum_T (A/3) n over the wing
    assert np.allclose(fn.cpu().numpy().sum(axis=0), fn_o.sum(axis=0), rtol=1e-12, atol=1e-15)


def test_pressure_taylor_green_768_fp32_closed_form():
    """3-D Taylor-Green at 768^3 (L = 2 pi, no mask): p = (cos 2x + cos 2y)
    (cos 2z + 2)/16 - 1/8 at sampled grid points."""
    n, L = 768, 2 * math.pi
    g = Solver(n, L, 0.01, 1.0, 1e-3, precision="fp32")
    x = torch.arange(n, device="cuda", dtype=torch.float64) * (L / n)
    s, c = torch.sin(x), torch.cos(x)
    u = torch.zeros((3, n, n, n), dtype=torch.float32, device="cuda")
    u[0] = (s[:, None, None] * c[None, :, None] * c[None, None, :]).float()
    u[1] = (-c[:, None, None] * s[None, :, None] * c[None, None, :]).float()
    g.set_velocity(u)
    del u
    pf = g.pressure()
    rng = np.random.default_rng(16)
    ijk = rng.integers(0, n, (8192, 3))
    idx = torch.from_numpy(ijk).cuda()
    got = pf[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    X = ijk * (L / n)
    want = (np.cos(2 * X[:, 0]) + np.cos(2 * X[:, 1])) * (np.cos(2 * X[:, 2]) + 2.0) / 16.0 - 0.125
    err = np.max(np.abs(got - want))
    print("768^3 TG-3D pressure: max sampled error %.2e" % err)
    assert err < 1e-5
    g.close()


@pytest.mark.parametrize("n,prec", [(32, "fp64"), (48, "fp32"), (128, "fp32")])
def test_keep_uw_resume_is_bitwise_identical(n, prec):
    """keep_uw: the step after ps_pressure starts at its z pass with the u
    and omega the pressure left in B. The coupling order (step, pressure,
    new mask, step, pressure twice, step) gives the same bits as a context
    that runs every pass."""
    L, nu, eta, dt = 4.0, 1.527e-4, 1e-2, 5e-4
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xw0, tri = inputs.elliptic_wing_mesh(300)
    amp = inputs.flapping_amplitudes(xw0)
    u = inputs.random_field(n, L, seed=n + 13, rms=0.3)
    res = []
    for keep in (False, True):
        g = Solver(n, L, nu, eta, dt, precision=prec, x0=(2.0, 2.0, 2.0), keep_uw=keep)
        g.set_velocity(dev(u, dtype))
        for k, t in enumerate((0.3, 0.35)):
            xw, vw, fr = inputs.revolving_wing(t, xw0, amp)
            g.set_mask_from_nodes(dev(xw, torch.float64), dev(vw, torch.float64), dev(tri, torch.int32), fr)
            if k == 0:
                g.step(2)
                p1 = g.pressure().clone()
        g.step(1)
        F1 = g.forces()
        p2 = g.pressure().clone()
        p3 = g.pressure().clone()
        g.step(1)
        res.append((p1, p2, p3, F1, g.forces(), g.velocity().clone()))
        g.close()
    a, b = res
    for k in (0, 1, 2, 5):
        assert torch.equal(a[k], b[k]), k
    assert a[3] == b[3] and a[4] == b[4]
    assert torch.equal(b[1], b[2])
