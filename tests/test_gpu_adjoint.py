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


def _wing_window(n, L, K, nodes, u0, dtype, dt):
    xw0, tri = inputs.elliptic_wing_mesh(nodes)
    amp = inputs.flapping_amplitudes(xw0)
    seq = [inputs.revolving_wing(k * dt, xw0, amp) for k in range(K)]
    win = WingWindow(dev(tri, torch.int32), [dev(s[0] - xw0, torch.float64) for s in seq],
                     [dev(s[1], torch.float64) for s in seq], [s[2] for s in seq], dev(u0, dtype))
    return xw0, tri, seq, win


def test_lift_gradient_matches_oracle_gradient():
    """32^3 revolving wing, 8-step window (checkpoint every 4), FP64: the
    library's d(mean lift)/d(node positions) against the oracle's: oracle
    forward over the rasterised masks, oracle adjoint, oracle rasteriser
    transpose, summed over the window."""
    n, L, nu, eta, dt = 32, 4.0, 1.527e-4, 1e-2, 5e-4
    K, every, dx = 8, 4, 4.0 / 32
    u0 = inputs.random_field(n, L, seed=9, rms=0.2)
    xw0, tri, seq, win = _wing_window(n, L, K, 120, u0, torch.float64, dt)
    g = Solver(n, L, nu, eta, dt, precision="fp64", with_adjoint=True)
    x = dev(xw0, torch.float64).requires_grad_(True)
    out = TimeAveragedForce.apply(x, g, win, every)
    out[2].backward()
    got = x.grad.cpu().numpy()

    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0))
    masks = []
    for xw, vw, fr in seq:
        chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
        masks.append((chi, us))
    w = np.full(K, 1.0 / K)
    a, b = np.array([0.0, 0.0, 1.0]), np.zeros(3)
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi, gus = OA.adjoint(p, states, masks, w, a, b)
    ref = np.zeros_like(xw0)
    for k, (xw, vw, fr) in enumerate(seq):
        ref += OA.rasterise_vjp(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, gchi[k], gus[k])
    assert abs(float(out[2]) - J) < 1e-12 * abs(J)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("32^3 node gradient vs oracle: rel %.2e" % err)
    assert err < 1e-9


def test_adjoint_config_128_fp32_vs_central_differences():
    """128^3 revolving wing (600 nodes), 64-step window with a checkpoint
    every 8 steps: d(mean lift)/d(node positions) by the FP32 forward and
    adjoint, against the FP64 adjoint (precision) and against central
    differences (h = 1e-4) of the FP64 forward.

    The objective is only piecewise smooth in the node positions: a band
    point's closest feature (face, edge or vertex region of a triangle)
    switches at kinks, and a difference quotient that straddles one differs
    from the derivative. At this resolution most node coordinates have such
    a switch within h somewhere in the window (over all 60 sampled ones the
    FP64 adjoint differs from the differences by ~1 % in norm). The
    comparison therefore uses the coordinates whose differences at h and
    h/2 agree to 1e-5 (no kink in reach; 5 of 60 here), where the FP64
    adjoint must match to 2e-4 (measured 6.9e-5) and the FP32 adjoint to
    1e-2 (measured 4.8e-3); exactness of the adjoint itself is pinned by the
    32^3 comparison with the oracle gradient."""
    n, L, nu, eta, dt = 128, 4.0, 1.0 / 1800, 1e-3, 5e-4
    K, every, h = 64, 8, 1e-4
    u0 = inputs.random_field(n, L, seed=128)
    grads = {}
    for prec, dtype in (("fp32", torch.float32), ("fp64", torch.float64)):
        xw0, tri, seq, win = _wing_window(n, L, K, 600, u0, dtype, dt)
        g = Solver(n, L, nu, eta, dt, precision=prec, with_adjoint=True)
        x = dev(xw0, torch.float64).requires_grad_(True)
        out = TimeAveragedForce.apply(x, g, win, every)
        out[2].backward()
        grads[prec] = x.grad.cpu().numpy()
        g.close()
    e_prec = np.linalg.norm(grads["fp32"] - grads["fp64"]) / np.linalg.norm(grads["fp64"])

    g64 = Solver(n, L, nu, eta, dt, precision="fp64")

    def J(xw):
        with torch.no_grad():
            return float(TimeAveragedForce.apply(dev(xw, torch.float64), g64, win, every)[2])

    def fd(node, c, hh):
        xp = xw0.copy(); xp[node, c] += hh
        xm = xw0.copy(); xm[node, c] -= hh
        return (J(xp) - J(xm)) / (2 * hh)

    rng = np.random.default_rng(7)
    rows = []
    for node in rng.choice(len(xw0), 20, replace=False):
        for c in range(3):
            f1, f2 = fd(node, c, h), fd(node, c, h / 2)
            rows.append((f1, f2, grads["fp64"][node, c], grads["fp32"][node, c]))
    rows = np.array(rows)
    f1, f2, a64, a32 = rows.T
    smooth = np.abs(f1 - f2) <= 1e-5 * np.abs(f1) + 1e-10
    e_all = np.linalg.norm(a64 - f1) / np.linalg.norm(f1)
    e64 = np.abs(a64 - f2)[smooth] / np.abs(f2)[smooth]
    e32 = np.abs(a32 - f2)[smooth] / np.abs(f2)[smooth]
    print("128^3 node gradient: fp32 vs fp64 adjoint %.2e; fp64 adjoint vs FD over all %d coords %.2e; "
          "%d kink-free coords: fp64 max %.2e, fp32 max %.2e" %
          (e_prec, len(f1), e_all, smooth.sum(), e64.max() if smooth.any() else -1, e32.max() if smooth.any() else -1))
    assert e_prec < 5e-3
    assert smooth.sum() >= 3
    assert e64.max() < 2e-4
    assert e32.max() < 1e-2


def test_adjoint_config_128_fp64_vs_small_step_differences():
    """The 128^3 configuration (600 nodes, 64 steps, checkpoint every 8) on 10
    seeded nodes (seed 7) x 3 coordinates: the FP64 adjoint against central
    differences of the FP64 forward with h = 1e-6. The objective is only
    piecewise smooth: every band point's closest feature (face, edge or
    vertex region) switches somewhere, and over 64 steps such switches lie
    densely in node space (measured: the quotients at h = 1e-4 and 5e-5
    disagree by up to 14 %, at 1e-6 and 5e-7 still by up to 2e-4 on a few
    coordinates). So the check is statistical: most coordinates and the
    median agree to 1e-5 (measured: mostly 1e-7 to 8e-6). Exactness of the
    adjoint is pinned at 32^3 against the oracle's gradient (1e-9)."""
    n, L, nu, eta, dt = 128, 4.0, 1.0 / 1800, 1e-3, 5e-4
    K, every, h = 64, 8, 1e-6
    u0 = inputs.random_field(n, L, seed=128)
    xw0, tri, seq, win = _wing_window(n, L, K, 600, u0, torch.float64, dt)
    g = Solver(n, L, nu, eta, dt, precision="fp64", with_adjoint=True)
    x = dev(xw0, torch.float64).requires_grad_(True)
    out = TimeAveragedForce.apply(x, g, win, every)
    out[2].backward()
    grad = x.grad.cpu().numpy()

    def J(xw):
        with torch.no_grad():
            return float(TimeAveragedForce.apply(dev(xw, torch.float64), g, win, every)[2])

    rng = np.random.default_rng(7)
    coords = [(node, c) for node in rng.choice(len(xw0), 10, replace=False) for c in range(3)]
    fd, a = [], []
    for node, c in coords:
        xp = xw0.copy(); xp[node, c] += h
        xm = xw0.copy(); xm[node, c] -= h
        fd.append((J(xp) - J(xm)) / (2 * h))
        a.append(grad[node, c])
    fd, a = np.array(fd), np.array(a)
    err = np.abs(a - fd) / np.abs(fd)
    print("128^3 FP64 adjoint vs h=1e-6 central differences over %d coordinates: median %.2e, "
          "%d within 1e-5, max %.2e" % (len(fd), np.median(err), (err < 1e-5).sum(), err.max()))
    g.close()
    assert np.median(err) < 1e-5
    assert (err < 1e-5).mean() >= 0.6
