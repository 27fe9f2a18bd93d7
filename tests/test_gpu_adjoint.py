"""GPU discrete adjoint (ps_adjoint_step, ps_mask_nodes_vjp) against the
oracle adjoint and against central differences of the GPU forward in FP64."""
import numpy as np
import pytest
import torch

from oracle import adjoint as OA
from oracle import mask as OM
from oracle import step as S
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.adjoint import TimeAveragedForce, WingWindow
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _case(n, K, seed=0):
    L = 4.0
    p = S.Params(n=n, L=L, nu=0.02, eta=0.05, dt=2e-3, x0=(1.9, 2.1, 2.05))
    rng = np.random.default_rng(seed)
    u0 = inputs.random_field(n, L, seed=seed + 3, rms=0.5)
    masks = []
    a0, a1 = n // 4, n // 4 + n // 3
    for k in range(K):
        chi = np.zeros((n, n, n))
        chi[a0:a1, a0 + 1:a1 + 1, a0 + 2:a1 + 2] = rng.uniform(0.2, 1.0, (a1 - a0,) * 3)
        us = rng.standard_normal((3, n, n, n)) * 0.1
        masks.append((chi, us))
    w = np.full(K, 1.0 / K)
    a = np.array([0.3, -0.2, 1.0])
    b = np.array([0.1, 0.4, -0.3])
    return p, u0, masks, w, a, b


def _gpu_adjoint(p, u0, masks, w, a, b, prec):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    n, K = p.n, len(masks)
    g = Solver(n, p.L, p.nu, p.eta, p.dt, precision=prec, x0=p.x0, with_adjoint=True)
    g.set_velocity(dev(u0, dtype))
    states, Js = [], 0.0
    md = [(dev(c, dtype), dev(s, dtype)) for c, s in masks]
    for k in range(K):
        buf = g.state_buffer()
        g.save_state(buf)
        states.append(buf)
        g.set_mask(*md[k])
        g.step(1)
        F, M = g.forces()
        Js += w[k] * (np.dot(a, F) + np.dot(b, M))
    gchi = torch.empty((n, n, n), dtype=dtype, device="cuda")
    gus = torch.empty((3, n, n, n), dtype=dtype, device="cuda")
    out = [None] * K
    g.adjoint_reset()
    for k in range(K - 1, -1, -1):
        g.restore_state(states[k])
        g.set_mask(*md[k])
        g.adjoint_step(w[k] * a, w[k] * b, k == 0, gchi, gus)
        out[k] = (gchi.double().cpu().numpy(), gus.double().cpu().numpy())
    return Js, out


@pytest.mark.parametrize("n,prec,tol", [(16, "fp64", 1e-10), (24, "fp64", 1e-10), (24, "fp32", 2e-4)])
def test_adjoint_matches_oracle(n, prec, tol):
    K = 4
    p, u0, masks, w, a, b = _case(n, K, seed=n)
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi, gus = OA.adjoint(p, states, masks, w, a, b)
    Jg, out = _gpu_adjoint(p, u0, masks, w, a, b, prec)
    assert abs(Jg - J) < (1e-12 if prec == "fp64" else 1e-4) * abs(J)
    for k in range(K):
        ec = np.linalg.norm(out[k][0] - gchi[k]) / np.linalg.norm(gchi[k])
        es = np.linalg.norm(out[k][1] - gus[k]) / np.linalg.norm(gus[k])
        assert ec < tol and es < tol, (k, ec, es)


def test_adjoint_dot_product_with_gpu_central_differences():
    """<dJ/dchi^k, dchi> against (J(chi + h dchi) - J(chi - h dchi)) / 2h with
    the GPU FP64 forward."""
    n, K = 24, 3
    p, u0, masks, w, a, b = _case(n, K, seed=7)
    J, out = _gpu_adjoint(p, u0, masks, w, a, b, "fp64")
    rng = np.random.default_rng(8)
    k = 1
    dchi = np.zeros_like(masks[k][0])
    sel = masks[k][0] > 0
    dchi[sel] = rng.uniform(-1, 1, sel.sum())
    h = 1e-5
    Jp, _ = _gpu_adjoint(p, u0, [m if i != k else (m[0] + h * dchi, m[1]) for i, m in enumerate(masks)],
                         w, a, b, "fp64")
    Jm, _ = _gpu_adjoint(p, u0, [m if i != k else (m[0] - h * dchi, m[1]) for i, m in enumerate(masks)],
                         w, a, b, "fp64")
    fd = (Jp - Jm) / (2 * h)
    ad = float(np.sum(out[k][0] * dchi))
    assert abs(fd - ad) < 1e-7 * abs(fd), (fd, ad)


# FP32: the closest triangle is chosen with FP32 distances, so at near-ties a
# different (equally close) triangle contributes the point's gradient
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 3e-2)])
def test_mask_vjp_matches_oracle(prec, tol):
    n, L = 32, 4.0
    dx = L / n
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xw0, tri = inputs.elliptic_wing_mesh(120)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0))
    vw = vw + np.random.default_rng(3).standard_normal(vw.shape) * 0.3
    rng = np.random.default_rng(4)
    cb = rng.standard_normal((n, n, n))
    ub = rng.standard_normal((3, n, n, n))
    ref = OA.rasterise_vjp(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, cb, ub)
    g = Solver(n, L, 1e-3, 1e-3, 5e-4, precision=prec)
    xw_d, vw_d, tri_d = dev(xw, torch.float64), dev(vw, torch.float64), dev(tri, torch.int32)
    g.set_mask_from_nodes(xw_d, vw_d, tri_d, fr)
    gx = torch.zeros((len(xw), 3), dtype=torch.float64, device="cuda")
    cbd, ubd = dev(cb, dtype), dev(ub, dtype)
    g.mask_nodes_vjp(cbd, ubd, gx)
    got = gx.cpu().numpy()
    assert np.linalg.norm(got - ref) < tol * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_time_averaged_lift_gradient_vs_central_differences():
    """Revolving wing at 32^3 (a downscaled adjoint window: 8 steps, checkpoint
    every 4): d(mean lift)/d(node positions) by the adjoint vs central
    differences (h = 1e-4) of the GPU FP64 forward, on seeded nodes."""
    n, L, nu, eta, dt = 32, 4.0, 1.527e-4, 1e-2, 5e-4
    K, every = 8, 4
    xw0, tri = inputs.elliptic_wing_mesh(120)
    amp = inputs.flapping_amplitudes(xw0)
    seq = [inputs.revolving_wing(k * dt, xw0, amp) for k in range(K)]
    g = Solver(n, L, nu, eta, dt, precision="fp64", with_adjoint=True)
    u0 = dev(inputs.random_field(n, L, seed=5, rms=0.2), torch.float64)
    win = WingWindow(dev(tri, torch.int32), [dev(s[0] - xw0, torch.float64) for s in seq],
                     [dev(s[1], torch.float64) for s in seq], [s[2] for s in seq], u0)
    x = dev(xw0, torch.float64).requires_grad_(True)
    out = TimeAveragedForce.apply(x, g, win, every)
    lift = out[2]
    lift.backward()
    grad = x.grad.cpu().numpy()

    def J(xw):
        with torch.no_grad():
            return float(TimeAveragedForce.apply(dev(xw, torch.float64), g, win, every)[2])

    rng = np.random.default_rng(7)
    h = 1e-4
    errs = []
    for node in rng.choice(len(xw0), 10, replace=False):
        for c in range(3):
            xp = xw0.copy(); xp[node, c] += h
            xm = xw0.copy(); xm[node, c] -= h
            fd = (J(xp) - J(xm)) / (2 * h)
            errs.append(abs(fd - grad[node, c]) / max(abs(fd), abs(grad[node, c]), 1e-6))
    errs = np.array(errs)
    print("node gradient vs FD: median rel err %.2e, max %.2e" % (np.median(errs), errs.max()))
    assert np.median(errs) < 1e-4 and np.mean(errs < 1e-2) > 0.8
