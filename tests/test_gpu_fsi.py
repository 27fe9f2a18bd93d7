"""GPU staggered fluid-structure coupling (Sec. 4.1, coupling paragraph):
the product loop (GPU step, pressure, loads, rasteriser; host mass-spring
network through ps_ms_*) against the oracle loop composed of the oracle's
step, pressure, load, mask and mass-spring routines."""
import numpy as np
import pytest
import torch

from oracle import fsi as OF
from oracle import massspring as OMS
from oracle import step as S
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.fsi import FSI
from paper_2002_08642_gb300.massspring import MassSpring
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _setup(n, ns=6, nc=2):
    L, nu, eta, dt = 4.0, 1.527e-4, 1e-2, 2e-3
    w = inputs.fsi_wing(ns=ns, nc=nc, veins=(0, nc), kb=0.05, ke=20.0, mass=0.05)

    def frames(t):
        return inputs.revolving_frames(t, tau=0.05)

    u0 = inputs.random_field(n, L, seed=77, rms=0.3)
    return L, nu, eta, dt, w, frames, u0


@pytest.mark.parametrize("prec,tol,keep", [("fp64", 1e-6, False), ("fp32", 2e-3, False), ("fp64", 1e-6, True),
                                           ("fp32", 2e-3, True)])
def test_fsi_loop_matches_oracle(prec, tol, keep):
    n, K = 32, 3
    L, nu, eta, dt, w, frames, u0 = _setup(n)
    dx = L / n
    net = OMS.Network(w["x0"], w["mass"], w["fixed"], w["ext"], w["ke"], w["bend"], w["kb"])
    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0))
    o = OF.Coupled(p, net, w["tri"], frames, u0, 2 * dx, 1.5 * dx, tol=1e-12)
    o.step(K)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    g = Solver(n, L, nu, eta, dt, precision=prec, x0=(2.0, 2.0, 2.0), keep_uw=keep)
    g.set_velocity(torch.from_numpy(u0).to("cuda", dtype))
    ms = MassSpring(w["x0"], w["mass"], w["ext"], w["ke"], w["bend"], w["kb"], fixed=w["fixed"])
    c = FSI(g, ms, w["tri"], frames, tol=1e-12)
    c.step(K)
    x, v = c.state()
    disp = np.max(np.abs(o.x - w["x0"]))
    ex = np.max(np.abs(x - o.x)) / disp
    ev = np.max(np.abs(v - o.v)) / np.max(np.abs(o.v))
    eu = np.linalg.norm(g.velocity().double().cpu().numpy() - o.fluid.velocity()) / np.linalg.norm(o.fluid.velocity())
    print("%s FSI %d steps: displacement %.3e, node error %.2e (rel), velocity %.2e, fluid %.2e"
          % (prec, K, disp, ex, ev, eu))
    assert disp > 1e-6
    assert ex < tol and ev < tol
    assert eu < (1e-9 if prec == "fp64" else 1e-5)
    assert all(1 <= it <= 20 for it in c.newton_iters)
    # the mask follows the nodes: chi^{K} of the product equals the oracle's
    chi, _ = g.mask()
    assert np.max(np.abs(chi.double().cpu().numpy() - o.fluid.chi)) < (1e-8 if prec == "fp64" else 1e-4)
