"""Per-slab GPU passes of the sharded step (the paper's MPI slabs, Sec. 4.1)
on one GPU: P slab contexts each running their share of every pass
(ps_slab_phase), the two exchanges as device-to-device block copies of the
x-pass array, the force as the host sum of the slabs' shares
(paper_2002_08642_gb300/slab.py SlabContexts). Against one context running
the whole step: the spectral state bit for bit (the same arithmetic per
element), the force and moment to rounding (another summation order);
against the oracle's global step; the rasteriser restricted to a slab's
x-planes against the full rasterisation."""
import numpy as np
import pytest
import torch

from oracle import step as S
from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.slab import SlabContexts, balanced
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _case(n):
    rng = np.random.default_rng(n)
    chi = np.zeros((n, n, n))
    a, b = n // 4, n // 2 + 3
    chi[a:b, a + 1:b, a + 2:b - 1] = rng.uniform(0.3, 1.0, (b - a, b - a - 1, b - a - 3))
    us = rng.standard_normal((3, n, n, n)) * 0.1
    u = inputs.random_field(n, 4.0, seed=n + 1, rms=0.5)
    return u, chi, us


@pytest.mark.parametrize("P", [2, 3])
@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp32", 48)])
def test_slab_contexts_match_one_context_and_oracle(P, prec, n):
    L, nu, eta, dt, x0 = 4.0, 0.02, 0.05, 2e-3, (1.9, 2.1, 2.05)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    u, chi, us = _case(n)
    K = 3
    g = Solver(n, L, nu, eta, dt, precision=prec, x0=x0)
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi, dtype), dev(us, dtype))
    g.step(K)
    F, M = g.forces()
    ref = g.state_buffer()
    g.save_state(ref)

    slabs = [Solver(n, L, nu, eta, dt, precision=prec, x0=x0) for _ in range(P)]
    for s in slabs:
        s.set_velocity(dev(u, dtype))
        s.set_mask(dev(chi, dtype), dev(us, dtype))
    Kk = B.ps_grid_info(slabs[0].ctx)[0]
    sc = SlabContexts(slabs, balanced(n, P), balanced(Kk, P))
    sc.step(K)
    F2, M2 = sc.forces()
    st = sc.state()
    assert torch.equal(st[256:], ref[256:])   # U and H, bit for bit
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.allclose(F2, F, rtol=tol, atol=tol * np.abs(F).max())
    assert np.allclose(M2, M, rtol=tol, atol=tol * np.abs(M).max())
    if prec == "fp64":
        o = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=x0))
        o.set_velocity(u)
        o.set_mask(chi, us)
        o.step(K)
        g.restore_state(st)
        v = g.velocity().cpu().numpy()
        assert np.linalg.norm(v - o.velocity()) / np.linalg.norm(o.velocity()) < 1e-12
        assert np.allclose(F2, o.F, rtol=1e-11, atol=1e-12 * np.abs(o.F).max())


def test_slab_rasteriser_covers_its_x_planes_only():
    n, L = 48, 4.0
    xw0, tri = inputs.elliptic_wing_mesh(300)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0))
    d = lambda a, t: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", t)
    g = Solver(n, L, 1e-3, 1e-3, 5e-4, precision="fp64")
    g.set_mask_from_nodes(d(xw, torch.float64), d(vw, torch.float64), d(tri, torch.int32), fr)
    chi, us = [t.clone() for t in g.mask()]
    xo = balanced(n, 3)
    for r in range(3):
        s = Solver(n, L, 1e-3, 1e-3, 5e-4, precision="fp64")
        B.ps_slab_set(s.ctx, xo[r], xo[r + 1], 0, B.ps_grid_info(s.ctx)[0])
        s.set_mask_from_nodes(d(xw, torch.float64), d(vw, torch.float64), d(tri, torch.int32), fr)
        c, u = s.mask()
        sl = slice(xo[r], xo[r + 1])
        assert torch.equal(c[sl], chi[sl]) and torch.equal(u[:, sl], us[:, sl])
        rest = torch.ones(n, dtype=torch.bool, device="cuda")
        rest[sl] = False
        assert c[rest].abs().max().item() == 0.0
        s.close()


def test_slab_bounds_are_checked():
    g = Solver(32, 4.0, 1e-3, 1e-3, 5e-4, precision="fp64")
    K = B.ps_grid_info(g.ctx)[0]
    for bad in ((0, 33, 0, K), (5, 5, 0, K), (0, 32, 3, 2), (0, 32, 0, K + 1)):
        with pytest.raises(B.PsError) as e:
            B.ps_slab_set(g.ctx, *bad)
        assert e.value.status == B.PS_EINVAL
    with pytest.raises(B.PsError) as e:
        B.ps_slab_phase(g.ctx, 0)   # no slab set
    assert e.value.status == B.PS_ESTATE
