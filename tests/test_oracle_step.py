"""Pins of the oracle step against closed forms and exact discrete identities."""
import math

import numpy as np
import pytest

from oracle import step as S
from paper_2002_08642_gb300 import inputs


def _grid(n, L):
    return inputs.grid(n, L)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_curl_closed_form():
    n, L = 16, 2 * math.pi
    p = S.Params(n=n, L=L, nu=0.0, eta=1.0, dt=0.0)
    X, Y, Z = _grid(n, L)
    u = np.stack([np.sin(Y), np.sin(Z), np.sin(X)])
    w = S.to_physical(S.curl_hat(p, S.to_spectral(u)), n)
    ref = np.stack([-np.cos(Z), -np.cos(X), -np.cos(Y)])
    assert np.max(np.abs(w - ref)) < 1e-13


def test_first_step_closed_form():
    """u0 = (sin y, sin z, sin x): P[u x omega] = (-sin z cos y, -sin x cos z,
    -sin y cos x) exactly (the sin 2x-type part is a gradient), so one IF-Euler
    step gives u1 = e^{-nu dt} u0 + dt e^{-2 nu dt} P[u x omega]."""
    n, L, nu, dt = 16, 2 * math.pi, 0.05, 0.01
    p = S.Params(n=n, L=L, nu=nu, eta=1.0, dt=dt)
    X, Y, Z = _grid(n, L)
    u0 = np.stack([np.sin(Y), np.sin(Z), np.sin(X)])
    s = S.Solver(p)
    s.set_velocity(u0)
    s.step(1)
    pn = np.stack([-np.sin(Z) * np.cos(Y), -np.sin(X) * np.cos(Z), -np.sin(Y) * np.cos(X)])
    ref = math.exp(-nu * dt) * u0 + dt * math.exp(-2 * nu * dt) * pn
    assert np.max(np.abs(s.velocity() - ref)) < 1e-14


@pytest.mark.parametrize("dt", [1e-3, 0.05])
def test_taylor_green_2d_exact_decay(dt):
    """2D TG: u x omega is a pure gradient, so the step is exact decay e^{-2 nu t}."""
    n, L, nu = 16, 2 * math.pi, 0.02
    p = S.Params(n=n, L=L, nu=nu, eta=1.0, dt=dt)
    s = S.Solver(p)
    u0 = inputs.taylor_green_2d(n, L)
    s.set_velocity(u0)
    s.step(10)
    assert np.max(np.abs(s.velocity() - math.exp(-2 * nu * 10 * dt) * u0)) < 1e-14


def test_penalized_ab2_recurrence():
    """chi = c constant, u_s = 0 on a 2D TG field: N = -(c/eta) u exactly, so each
    mode follows the scalar IF-AB2 recurrence written out here."""
    n, L, nu, dt, eta, c = 16, 2 * math.pi, 0.03, 0.02, 0.1, 0.4
    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt)
    s = S.Solver(p)
    u0 = inputs.taylor_green_2d(n, L)
    s.set_velocity(u0)
    s.set_mask(np.full((n, n, n), c), np.zeros((3, n, n, n)))
    E = math.exp(-nu * 2.0 * dt)
    lam = -c / eta
    a = [1.0, E * (1.0 + dt * lam)]
    for _ in range(6):
        a.append(E * a[-1] + 0.5 * dt * (3 * E * lam * a[-1] - E * E * lam * a[-2]))
    s.step(7)
    assert np.max(np.abs(s.velocity() - a[7] * u0)) < 1e-14


def test_taylor_green_3d_decay():
    """Config: 32^3, L = 2 pi, nu = 0.01, dt = 1e-3, 20 steps. The (1,1,1) amplitude
    follows exp(-3 nu t) up to an O(t^2) nonlinear correction."""
    n, L, nu, dt = 32, 2 * math.pi, 0.01, 1e-3
    p = S.Params(n=n, L=L, nu=nu, eta=1.0, dt=dt)
    s = S.Solver(p)
    u0 = inputs.taylor_green_3d(n, L)
    s.set_velocity(u0)
    s.step(20)
    u = s.velocity()
    amp = np.sum(u * u0) / np.sum(u0 * u0)
    exact = math.exp(-3 * nu * 20 * dt)
    assert abs(amp - exact) < 1e-4
    assert abs(amp - exact) > 1e-9   # the nonlinear correction is really there


def test_divergence_roundoff_and_energy_identity():
    n, L = 24, 4.0
    p = S.Params(n=n, L=L, nu=0.0, eta=1e-3, dt=5e-4, x0=(2.0, 2.0, 2.0))
    s = S.Solver(p)
    s.set_velocity(inputs.random_field(n, L, seed=5))
    # inviscid, no mask: <u_hat, P N_hat> = 0 exactly
    Nh = s.rhs_hat()
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    dot = np.sum(np.real(np.conj(s.uh) * Nh) * w)
    scale = np.sqrt(np.sum(np.abs(s.uh) ** 2 * w) * np.sum(np.abs(Nh) ** 2 * w))
    assert abs(dot) < 1e-13 * scale
    # with a mask, the state stays solenoidal to round-off
    rng = np.random.default_rng(3)
    s.set_mask(rng.uniform(0, 1, (n, n, n)), rng.standard_normal((3, n, n, n)) * 0.05)
    s.step(3)
    kx, ky, kz = S.wavevectors(p)
    kmax = np.max(np.sqrt(kx ** 2 + ky ** 2 + kz ** 2))
    umax = np.max(np.abs(s.uh)) / n ** 3
    assert s.max_divergence() < 1e-14 * kmax * umax


def test_inviscid_energy_drift_second_order():
    """nu = 0, chi = 0: the semi-discrete energy is conserved, so the drift over a
    fixed time is the scheme's O(dt^2) global error: halving dt quarters it."""
    n, L = 16, 2 * math.pi
    drift = []
    for dt, k in ((0.02, 20), (0.01, 40)):
        p = S.Params(n=n, L=L, nu=0.0, eta=1.0, dt=dt)
        s = S.Solver(p)
        s.set_velocity(inputs.random_field(n, L, seed=11, rms=0.2))
        e0 = s.energy()
        s.step(k)
        drift.append(abs(s.energy() - e0))
    ratio = drift[0] / drift[1]
    assert 3.8 < ratio < 4.3, ratio


def test_energy_parseval():
    n, L = 12, 3.0
    p = S.Params(n=n, L=L, nu=0.0, eta=1.0, dt=0.0)
    s = S.Solver(p)
    u = inputs.random_field(n, L, seed=2)
    s.set_velocity(u)
    v = s.velocity()
    direct = 0.5 * np.sum(v * v) * (L / n) ** 3
    assert abs(s.energy() - direct) < 1e-13 * direct


def test_force_uniform_flow_block():
    """u = U constant, u_s = 0, chi = 1 on a block of cells: F = U dx^3 count/eta and
    M = (dx^3/eta) count (centroid - x0) x U."""
    n, L, eta = 16, 4.0, 1e-2
    x0 = (2.0, 1.5, 2.5)
    p = S.Params(n=n, L=L, nu=0.0, eta=eta, dt=1e-3, x0=x0)
    U = np.array([0.3, -0.2, 0.7])
    chi = np.zeros((n, n, n))
    chi[2:7, 4:9, 10:13] = 1.0
    u = np.broadcast_to(U[:, None, None, None], (3, n, n, n)).copy()
    F, M = S.penalization_force(p, u, chi, np.zeros((3, n, n, n)))
    dx = L / n
    count = 5 * 5 * 3
    centroid = dx * np.array([(2 + 6) / 2, (4 + 8) / 2, (10 + 12) / 2])
    assert np.allclose(F, U * dx ** 3 * count / eta, rtol=1e-14, atol=0)
    Mref = dx ** 3 / eta * count * np.cross(centroid - np.array(x0), U)
    assert np.allclose(M, Mref, rtol=1e-13, atol=1e-15)
    # rigid motion with u = u_s: no force
    F0, M0 = S.penalization_force(p, u, chi, u)
    assert np.all(F0 == 0) and np.all(M0 == 0)


def test_force_is_from_current_velocity():
    n, L = 8, 4.0
    p = S.Params(n=n, L=L, nu=0.0, eta=0.5, dt=0.1, x0=(2, 2, 2))
    s = S.Solver(p)
    u = np.zeros((3, n, n, n))
    u[0] += 0.25
    s.set_velocity(u)
    s.set_mask(np.ones((n, n, n)), np.zeros((3, n, n, n)))
    s.step(1)
    assert abs(s.F[0] - 0.25 * L ** 3 / 0.5) < 1e-12


def test_mean_modes():
    n, L, eta, dt = 8, 4.0, 0.5, 0.1
    u = np.zeros((3, n, n, n))
    u[1] += 1.0
    for mode, expect in ((S.MEAN_FIXED, 1.0), (S.MEAN_FREE, None)):
        p = S.Params(n=n, L=L, nu=0.0, eta=eta, dt=dt, mean_mode=mode)
        s = S.Solver(p)
        s.set_velocity(u)
        s.set_mask(np.ones((n, n, n)), np.zeros((3, n, n, n)))
        s.step(2)
        m = s.velocity()[1].mean()
        if expect is not None:
            assert abs(m - expect) < 1e-15
        else:
            lam = -1.0 / eta
            a1 = 1.0 + dt * lam
            a2 = a1 + 0.5 * dt * (3 * lam * a1 - lam * 1.0)
            assert abs(m - a2) < 1e-14


def test_set_velocity_removes_gradient():
    n, L = 12, 2 * math.pi
    p = S.Params(n=n, L=L, nu=0.0, eta=1.0, dt=0.0)
    X, Y, Z = _grid(n, L)
    # u = grad(sin x cos 2y) + 0.5 (constant mean in z)
    u = np.stack([np.cos(X) * np.cos(2 * Y), -2 * np.sin(X) * np.sin(2 * Y), np.full_like(X, 0.5)])
    s = S.Solver(p)
    s.set_velocity(u)
    v = s.velocity()
    assert np.max(np.abs(v[:2])) < 1e-14 and np.max(np.abs(v[2] - 0.5)) < 1e-14


def test_sponge_uniform_is_linear_damping_recurrence():
    """chi_sp = 1 everywhere on the 2-D Taylor-Green vortex: u x omega is a
    gradient (projected out) and the sponge term is exactly -u/C_sp, so the
    amplitude follows the scalar IF-AB2 recurrence with N = -a/C_sp."""
    n, L, nu, dt, c_sp, K = 16, 2 * math.pi, 0.02, 1e-2, 0.5, 12
    p = S.Params(n=n, L=L, nu=nu, eta=1.0, dt=dt)
    X, Y, Z = np.meshgrid(*(np.arange(n) * (L / n),) * 3, indexing="ij")
    u0 = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y), np.zeros_like(X)])
    o = S.Solver(p)
    o.set_velocity(u0)
    o.set_sponge(np.ones((n, n, n)), c_sp)
    o.step(K)
    E = math.exp(-nu * 2.0 * dt)
    a_prev, a = None, 1.0
    for k in range(K):
        N = -a / c_sp
        new = E * (a + dt * N) if k == 0 else E * a + 0.5 * dt * (3 * E * N - E * E * (-a_prev / c_sp))
        a_prev, a = a, new
    got = o.velocity()
    assert np.max(np.abs(got - a * u0)) < 1e-12
    # off again: the plain decay
    o2 = S.Solver(p)
    o2.set_velocity(u0)
    o2.set_sponge(np.zeros((n, n, n)), c_sp)
    o2.step(3)
    assert np.max(np.abs(o2.velocity() - math.exp(-nu * 2.0 * 3 * dt) * u0)) < 1e-13


def test_sponge_term_is_solenoidal_and_local():
    """A sponge mask on a slab: the sponge term is divergence-free and, for a
    field vanishing on the slab, zero."""
    n, L = 16, 2 * math.pi
    p = S.Params(n=n, L=L, nu=0.0, eta=1.0, dt=1e-3)
    rng = np.random.default_rng(2)
    sh = S.to_spectral(rng.standard_normal((3, n, n, n))) * S.dealias_mask(n)
    Sh = S.sponge_hat(p, sh, 0.3)
    kx, ky, kz = S.wavevectors(p)
    assert np.max(np.abs(kx * Sh[0] + ky * Sh[1] + kz * Sh[2])) < 1e-10 * np.max(np.abs(Sh))
    assert np.max(np.abs(S.sponge_hat(p, np.zeros_like(sh), 0.3))) == 0.0
