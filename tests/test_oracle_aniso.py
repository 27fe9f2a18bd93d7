"""Pins of the oracle on the paper's anisotropic box (Sec. 4.2: the
revolving-wing domain 4 x 4 x 2 with N x N x N/2 points, the same spacing on
every axis): closed forms that fix the z wavenumbers 2 pi m / Lz, the z
extent of every array and the volume factors."""
import math

import numpy as np
import pytest

from oracle import fft as offt
from oracle import mask as OM
from oracle import pressure as OP
from oracle import step as S


def box(n=16, nu=0.03, dt=0.01, **kw):
    """[0, 2 pi)^2 x [0, pi) with n x n x n/2 points."""
    return S.Params(n=n, L=2 * math.pi, nu=nu, eta=1.0, dt=dt, nz=n // 2, **kw)


def test_params_fill_and_check_the_z_axis():
    p = box(16)
    assert p.nz == 8 and math.isclose(p.Lz, math.pi)
    q = S.Params(n=12, L=4.0, nu=0.0, eta=1.0, dt=1.0)
    assert q.nz == 12 and q.Lz == 4.0
    with pytest.raises(ValueError):
        S.Params(n=16, L=4.0, nu=0.0, eta=1.0, dt=1.0, nz=8, Lz=4.0)


def test_half_spectrum_transforms_match_numpy():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(12, 12, 6))
    U = offt.rfft3(u)
    assert np.allclose(U, np.fft.rfftn(u), atol=1e-12)
    assert np.allclose(offt.irfft3(U, 6), u, atol=1e-13)


def grid(p):
    X, Y, Z = S.grid_coords(p)
    shape = (p.n, p.n, p.nz)
    return [np.broadcast_to(c, shape) for c in (X, Y, Z)]


def test_curl_closed_form():
    """u = (sin 2z, sin x, sin y) on Lz = pi: omega = (cos y, 2 cos 2z, cos x)
    (the z mode m_z = 1 has k_z = 2)."""
    p = box(16)
    X, Y, Z = grid(p)
    u = np.stack([np.sin(2 * Z), np.sin(X), np.sin(Y)])
    w = S.to_physical(S.curl_hat(p, S.to_spectral(u)), p.nz)
    assert np.max(np.abs(w - np.stack([np.cos(Y), 2 * np.cos(2 * Z), np.cos(X)]))) < 1e-12


def test_shear_mode_decays_exactly():
    """u = (sin 2z, 0, 0): u x omega = (0, 0, sin 4z) is a gradient, so the
    projected nonlinear term vanishes and the amplitude is exp(-4 nu t) at
    any dt (the integrating factor is exact); the energy is L^2 Lz / 4
    times the amplitude squared."""
    p = box(16, nu=0.03, dt=0.05)
    X, Y, Z = grid(p)
    u0 = np.stack([np.sin(2 * Z), 0 * Z, 0 * Z])
    s = S.Solver(p)
    s.set_velocity(u0)
    assert math.isclose(s.energy(), (2 * math.pi) ** 2 * math.pi / 4, rel_tol=1e-12)
    s.step(6)
    a = math.exp(-4 * p.nu * 6 * p.dt)
    assert np.max(np.abs(s.velocity() - a * u0)) < 1e-13
    assert s.max_divergence() < 1e-14


def test_taylor_green_2d_decays_exactly():
    p = box(12, nu=0.02, dt=0.1)
    X, Y, Z = grid(p)
    u0 = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y), 0 * Z])
    s = S.Solver(p)
    s.set_velocity(u0)
    s.step(5)
    assert np.max(np.abs(s.velocity() - math.exp(-2 * p.nu * 0.5) * u0)) < 1e-13


def test_z_dependent_taylor_green_first_step():
    """u = (sin x cos y cos 2z, -cos x sin y cos 2z, 0), divergence free on
    Lz = pi. Its vorticity in closed form is
    (-2 cos x sin y sin 2z, -2 sin x cos y sin 2z, 2 sin x sin y cos 2z), and
    the first (integrating-factor Euler) step is E (u_hat + dt P N_hat) with
    N = u x omega from that closed form."""
    p = box(16, nu=0.01, dt=0.02)
    X, Y, Z = grid(p)
    cz, sz = np.cos(2 * Z), np.sin(2 * Z)
    u0 = np.stack([np.sin(X) * np.cos(Y) * cz, -np.cos(X) * np.sin(Y) * cz, 0 * Z])
    w = np.stack([-2 * np.cos(X) * np.sin(Y) * sz, -2 * np.sin(X) * np.cos(Y) * sz, 2 * np.sin(X) * np.sin(Y) * cz])
    assert np.max(np.abs(S.to_physical(S.curl_hat(p, S.to_spectral(u0)), p.nz) - w)) < 1e-12
    s = S.Solver(p)
    s.set_velocity(u0)
    s.step(1)
    nl = np.stack([u0[1] * w[2] - u0[2] * w[1], u0[2] * w[0] - u0[0] * w[2], u0[0] * w[1] - u0[1] * w[0]])
    Nh = S.project(p, S.to_spectral(nl) * S.dealias_mask(p.n, p.nz))
    want = S.to_physical(S.integrating_factor(p) * (S.to_spectral(u0) + p.dt * Nh), p.nz)
    assert np.max(np.abs(s.velocity() - want)) < 1e-13
    # the nonlinear term is not a pure gradient here: the step differs from
    # the viscous decay exp(-nu (1 + 1 + 4) dt) of the initial mode
    assert np.max(np.abs(s.velocity() - math.exp(-6 * p.nu * p.dt) * u0)) > 1e-6


def test_block_force_and_pressure():
    """A uniform flow U through a block mask: F = U dx^3 sum chi / eta; the
    2-D Taylor-Green pressure on the anisotropic grid is
    p = (cos 2x + cos 2y)/4 up to a constant."""
    p = box(12)
    dx = p.L / p.n
    chi = np.zeros((p.n, p.n, p.nz))
    chi[3:7, 2:5, 1:4] = 1.0
    U = np.array([0.3, -0.2, 0.7])
    u = np.broadcast_to(U[:, None, None, None], (3, p.n, p.n, p.nz)).copy()
    F, M = S.penalization_force(p, u, chi, np.zeros_like(u))
    assert np.allclose(F, U * dx ** 3 * chi.sum() / p.eta, rtol=1e-13)
    X, Y, Z = grid(p)
    u0 = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y), 0 * Z])
    s = S.Solver(p)
    s.set_velocity(u0)
    pf = OP.static_pressure(p, s.uh, np.zeros((p.n, p.n, p.nz)), np.zeros((3, p.n, p.n, p.nz)))
    want = (np.cos(2 * X) + np.cos(2 * Y)) / 4
    got = pf - pf.mean()
    assert np.max(np.abs(got - (want - want.mean()))) < 1e-12


def test_mask_and_interpolation_on_the_anisotropic_grid():
    """A horizontal plate at z = Lz/2 covering the middle of the box: chi
    depends on |z - Lz/2| only above its interior; delta interpolation is
    periodic in z with the box's z length and a partition of unity."""
    n, L = 16, 4.0
    nz, dx = 8, L / 16
    xw = np.array([[1.0, 1.0, 0.0], [3.0, 1.0, 0.0], [3.0, 3.0, 0.0], [1.0, 3.0, 0.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]])
    frame = {"R": np.eye(3).reshape(9), "X_O": np.array([0.0, 0.0, 1.0]), "V_O": np.zeros(3),
             "Omega": np.zeros(3)}
    chi, us, arg, best = OM.rasterise(n, L, xw, np.zeros_like(xw), tri, frame, 2 * dx, 1.5 * dx, nz=nz)
    assert chi.shape == (n, n, nz) and us.shape == (3, n, n, nz)
    k = np.arange(nz)
    want = OM.chi_cos(np.abs(k * dx - 1.0), 2 * dx, 1.5 * dx)
    assert np.allclose(chi[8, 8, :], want, atol=1e-14)
    assert np.all(chi[0, 0, :] == 0.0)
    # interpolation wraps z with period Lz = nz dx (and x, y with L)
    rng = np.random.default_rng(4)
    pf = rng.normal(size=(n, n, nz))
    pts = np.array([[1.3, 2.2, 0.07], [0.1, 3.9, 1.91]])
    a = OP.interpolate(pf, L, pts)
    b = OP.interpolate(pf, L, pts + np.array([L, 0.0, nz * dx]))
    assert np.allclose(a, b, atol=1e-13)
    assert np.allclose(OP.interpolate(np.ones((n, n, nz)), L, pts), 1.0, atol=1e-14)


def test_adjoint_on_the_anisotropic_box_matches_central_differences():
    """The oracle adjoint on the N x N x N/2 grid (rfft3* = N irfft3 with
    N = n^2 nz points): dJ/dchi and dJ/du_s against central differences of
    the oracle forward over three masked steps."""
    from oracle import adjoint as OA

    n, nz, K = 16, 8, 3
    p = S.Params(n=n, L=4.0, nu=0.02, eta=0.05, dt=2e-3, x0=(1.9, 2.1, 1.05), nz=nz)
    rng = np.random.default_rng(2)
    X, Y, Z = grid(p)
    u0 = np.stack([np.sin(np.pi * Y / 2) * np.cos(np.pi * Z), np.sin(np.pi * Z) * np.cos(np.pi * X / 2),
                   0.3 * np.cos(np.pi * (X + Y) / 2)])
    masks = []
    for _ in range(K):
        chi = np.zeros((n, n, nz))
        chi[4:10, 5:11, 2:6] = rng.uniform(0.2, 1.0, (6, 6, 4))
        masks.append((chi, rng.standard_normal((3, n, n, nz)) * 0.1))
    w = np.full(K, 1.0 / K)
    a, b = np.array([0.3, -0.2, 1.0]), np.array([0.1, 0.4, -0.3])
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi, gus = OA.adjoint(p, states, masks, w, a, b)
    h = 1e-5
    for k in (0, 2):
        dchi = np.zeros((n, n, nz))
        dchi[4:10, 5:11, 2:6] = rng.uniform(-1, 1, (6, 6, 4))
        dus = rng.standard_normal((3, n, n, nz))
        for which, d, g in ((0, dchi, gchi[k]), (1, dus, gus[k])):
            def shifted(s):
                return [m if i != k else ((m[0] + s * d, m[1]) if which == 0 else (m[0], m[1] + s * d))
                        for i, m in enumerate(masks)]
            fd = (OA.forward(p, u0, shifted(h), w, a, b)[0] - OA.forward(p, u0, shifted(-h), w, a, b)[0]) / (2 * h)
            ad = float(np.sum(g * d))
            assert abs(fd - ad) < 1e-7 * max(abs(fd), 1e-12), (k, which, fd, ad)


def test_rasterise_vjp_on_the_anisotropic_grid():
    """The rasteriser's transpose on a 32 x 32 x 16 grid of a 4 x 4 x 2 box
    (the wing revolving about the centre (2, 2, 1)) against central
    differences of J = sum chi_bar chi + sum us_bar u_s."""
    from oracle import adjoint as OA
    from paper_2002_08642_gb300 import inputs

    n, nz, L = 32, 16, 4.0
    dx = L / n
    xw0, tri = inputs.elliptic_wing_mesh(60)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0), centre=(2.0, 2.0, 1.0))
    rng = np.random.default_rng(7)
    cb = rng.standard_normal((n, n, nz))
    ub = rng.standard_normal((3, n, n, nz))

    def J(x):
        chi, us, _, _ = OM.rasterise(n, L, x, vw, tri, fr, 2 * dx, 1.5 * dx, nz=nz)
        return float(np.sum(cb * chi) + np.sum(ub * us))

    g = OA.rasterise_vjp(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, cb, ub, nz=nz)
    h = 1e-6
    errs = []
    for node in rng.choice(len(xw), 6, replace=False):
        for c in range(3):
            xp = xw.copy()
            xp[node, c] += h
            xm = xw.copy()
            xm[node, c] -= h
            fd = (J(xp) - J(xm)) / (2 * h)
            errs.append(abs(fd - g[node, c]) / max(abs(fd), abs(g[node, c]), 1e-3))
    errs = np.array(errs)
    assert np.median(errs) < 1e-5 and np.mean(errs < 1e-4) > 0.85, errs


def test_coupled_oracle_loop_runs_on_the_anisotropic_box():
    """The oracle's staggered loop on a 16 x 16 x 8 grid of the 4 x 4 x 2 box
    (wing revolving about (2, 2, 1)): the loads move the network, the state
    stays finite and divergence free."""
    from oracle import fsi as OF
    from oracle import massspring as OMS
    from paper_2002_08642_gb300 import inputs

    n, nz, L = 16, 8, 4.0
    dx = L / n
    p = S.Params(n=n, L=L, nu=1.527e-4, eta=1e-2, dt=2e-3, x0=(2.0, 2.0, 1.0), nz=nz)
    w = inputs.fsi_wing(ns=4, nc=2, veins=(0, 2), kb=0.05, ke=20.0, mass=0.05)
    net = OMS.Network(w["x0"], w["mass"], w["fixed"], w["ext"], w["ke"], w["bend"], w["kb"])

    def frames(t):
        return inputs.revolving_frames(t, centre=(2.0, 2.0, 1.0), tau=0.05)

    X, Y, Z = grid(p)
    u0 = 0.3 * np.stack([np.sin(np.pi * Y / 2) * np.cos(np.pi * Z), 0 * X, np.cos(np.pi * X / 2) + 0 * Z])
    o = OF.Coupled(p, net, w["tri"], frames, u0, 2 * dx, 1.5 * dx, tol=1e-12)
    assert o.fluid.chi.shape == (n, n, nz) and o.fluid.chi.max() > 0
    o.step(2)
    assert np.all(np.isfinite(o.x)) and np.max(np.abs(o.x - w["x0"])) > 1e-8
    assert o.fluid.max_divergence() < 1e-12
