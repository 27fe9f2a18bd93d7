"""Pins of the oracle mass-spring network (Sec. 2.1-2.4: extension and
bending springs, the k^b - EI relation, variable-step BDF2) against what the
paper and the mathematics fix: the printed extension force, the
small-deflection cantilever closed form F L^3 / (3 EI), the paper's static
large-deflection table (Sec. 2.4.1, Table 1) and second-order convergence of
BDF2 on a harmonic oscillator."""
import math
import os

import numpy as np
import pytest

from oracle import massspring as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cantilever_large_deflection.txt")


def table():
    return np.loadtxt(GOLDEN)


def test_extension_force_is_the_printed_formula():
    """Sec. 2.2, Eq. (extension_spring): F_i = k^e (|x_ij| - |x_0,ij|) e_ij,
    F_j = -F_i, summed over springs; the oracle takes -grad of the energy."""
    rng = np.random.default_rng(3)
    n = 6
    x0 = rng.normal(size=(n, 3))
    ext = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (0, 3), (2, 5)]
    ke = rng.uniform(0.5, 3.0, len(ext))
    net = M.Network(x0, np.ones(n), np.zeros(n, bool), ext, ke, np.zeros((0, 3), int), [])
    x = x0 + 0.2 * rng.normal(size=(n, 3))
    want = np.zeros((n, 3))
    for s, (i, j) in enumerate(ext):
        d = x[j] - x[i]
        e = d / np.linalg.norm(d)
        f = ke[s] * (np.linalg.norm(d) - np.linalg.norm(x0[j] - x0[i])) * e
        want[i] += f
        want[j] -= f
    assert np.max(np.abs(M.Network.forces(net, x) - want)) < 1e-7 * np.max(np.abs(want))


def test_bending_angle_sign_and_rest_state():
    """Eq. (two_bending_angles): a left turn in the x-y plane is a positive
    theta^y, a bend in x-z a positive theta^z; the rest state has no force."""
    ty, tz = M._angles(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([1.0, 1.0, 0]))
    assert ty == pytest.approx(math.pi / 2) and tz == 0.0
    ty, tz = M._angles(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([2.0, 0, 0.5]))
    assert ty == 0.0 and tz == pytest.approx(math.atan(0.5))
    net = M.cantilever(0.3, 0.24, 8, ke=1e3)
    assert np.max(np.abs(net.forces(net.x0))) < 1e-12


@pytest.mark.parametrize("npts", [4, 7, 12])
def test_small_deflection_matches_beam_closed_form(npts):
    """Sec. 2.3.1, Eq. (EI_k_relation): with k^b from EI the network's tip
    deflection under a small tip load equals the Euler--Bernoulli cantilever
    F L^3 / (3 EI) for any number of points (the relation equates the two
    stored energies, F delta / 2)."""
    L, EI, F = 0.3, 0.24, 1e-4
    net = M.cantilever(L, EI, npts, ke=1e7)
    fe = np.zeros((npts, 3))
    fe[-1, 1] = -F
    x = M.equilibrium(net, fe, steps=1, tol=1e-13)
    want = F * L ** 3 / (3 * EI)
    assert -x[-1, 1] == pytest.approx(want, rel=1e-6)
    assert np.all(x[:2] == net.x0[:2])


def test_large_deflection_table():
    """Sec. 2.4.1, Table 1: tip position of the 22-point network against the
    continuum nonlinear beam. The network converges to the beam as points
    are added (like 1/n: 12 -> 22 points halves the error; at the paper's
    64 points this oracle is within 0.3 % of the paper's own network)."""
    L, EI = 0.3, 0.24
    rows = table()[[1, 2, 4]]
    for F, xr, yr, _, _ in rows:
        err = {}
        for npts in (12, 22):
            net = M.cantilever(L, EI, npts, ke=1e7)
            fe = np.zeros((npts, 3))
            fe[-1, 1] = -F
            x = M.equilibrium(net, fe, steps=8, tol=1e-10)
            err[npts] = (abs(x[-1, 0] * 100 - xr) / abs(xr), abs(x[-1, 1] * 100 - yr) / abs(yr))
        assert err[22][0] < 5e-3 and err[22][1] < 2e-2, (F, err)
        assert err[22][1] < 0.65 * err[12][1], (F, err)


def _oscillator(k=4.0, m=1.0):
    x0 = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    return M.Network(x0, [m, m], [True, False], [(0, 1)], [k], np.zeros((0, 3), int), [])


def _integrate(dts, A=1e-3):
    net = _oscillator()
    x = net.x0.copy()
    x[1, 0] += A
    v = np.zeros_like(x)
    xm1 = vm1 = None
    dt_prev = None
    for dt in dts:
        xn, vn, _ = M.bdf2_step(net, x, v, xm1, vm1, dt, dt_prev, np.zeros_like(x), tol=1e-13)
        xm1, vm1, x, v, dt_prev = x, v, xn, vn, dt
    T = float(np.sum(dts))
    return x[1, 0] - 1.0 - A * math.cos(2.0 * T)


@pytest.mark.parametrize("variable", [False, True])
def test_bdf2_second_order(variable):
    """Eq. (discretized_ODEs) on m x'' = -k x (omega = 2): halving every
    step cuts the error at T = 1 by about 4, with constant steps and with
    steps alternating in ratio 3/2 (xi != 1)."""
    errs = []
    for m in (40, 80, 160):
        if variable:
            base = np.array([1.2, 0.8] * (m // 2)) / m
        else:
            base = np.full(m, 1.0 / m)
        errs.append(abs(_integrate(base)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.7 < r2 < 4.3, errs


def test_first_step_is_backward_euler():
    """With no history (xi = 0) the scheme is backward Euler: one step of
    the oscillator solves x1 = x0 + dt v1, v1 = v0 - dt (k/m) x1 exactly."""
    net = _oscillator()
    A, dt = 1e-3, 0.1
    x = net.x0.copy()
    x[1, 0] += A
    xn, vn, _ = M.bdf2_step(net, x, np.zeros_like(x), None, None, dt, None, np.zeros_like(x), tol=1e-14)
    x1 = A / (1 + 4.0 * dt * dt)
    assert xn[1, 0] - 1.0 == pytest.approx(x1, rel=1e-8)
    assert vn[1, 0] == pytest.approx(-4.0 * dt * x1, rel=1e-8)
    assert np.all(xn[0] == net.x0[0]) and np.all(vn[0] == 0)


def _spin_frame(t, tau=0.5, acc=(0.3, -0.2, 0.1)):
    """Frame turning about z by phi(t) = tau e^{-t/tau} + t - tau (the
    startup of Sec. 4.2) with its origin accelerating uniformly by acc
    (inertial axes). Returns R, X_O and the frame's A_O, Omega, dOmega in
    its own axes."""
    phi = tau * math.exp(-t / tau) + t - tau
    w = 1.0 - math.exp(-t / tau)
    dw = math.exp(-t / tau) / tau
    c, s = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    a = np.asarray(acc)
    return R, 0.5 * a * t * t, dict(A_O=R.T @ a, Omega=(0.0, 0.0, w), dOmega=(0.0, 0.0, dw))


def _free_particles():
    x0 = np.array([[0.4, 0.1, -0.2], [-0.3, 0.5, 0.25]])
    v_in = np.array([[0.2, -0.1, 0.3], [0.0, 0.4, -0.2]])
    net = M.Network(x0, [1.0, 2.5], [False, False], np.zeros((0, 2), int), [], np.zeros((0, 3), int), [])
    return net, x0, v_in


def _moving_frame_error(m, T=1.0):
    net, x0, v_in = _free_particles()
    x, v = x0.copy(), v_in.copy()   # at t = 0 the frames coincide and Omega = 0
    xm1 = vm1 = None
    dt = T / m
    for k in range(m):
        _, _, fr = _spin_frame((k + 1) * dt)
        xn, vn, _ = M.bdf2_step(net, x, v, xm1, vm1, dt, dt, np.zeros_like(x), tol=1e-13, frame=fr)
        xm1, vm1, x, v = x, v, xn, vn
    R, XO, _ = _spin_frame(T)
    want = (x0 + v_in * T - XO[None]) @ R   # rows: R^T (X - X_O)
    return np.max(np.abs(x - want))


def test_moving_frame_free_particle_second_order():
    """Free particles move on straight lines in the inertial frame; solved
    in a frame that spins up and accelerates, the fictitious forces must
    reproduce R^T (X0 + V0 t - X_O(t)) to second order in dt (a wrong sign
    in any of the four terms leaves an O(1) error)."""
    e = [_moving_frame_error(m) for m in (40, 80, 160)]
    assert e[2] < 2e-4, e
    assert 3.5 < e[0] / e[1] < 4.6 and 3.7 < e[1] / e[2] < 4.3, e


def test_cantilever_free_vibration_period():
    """Sec. 2.4.1, dynamic case (beam of length 1, mass per length 0.0571,
    EI = 0.0259): released from a small tip deflection, the 10-point network
    with lumped masses and k^b of Eq. (EI_k_relation) vibrates in its first
    mode with the Euler--Bernoulli period 2 pi / (1.8751^2 sqrt(EI / (mu
    L^4))) to within the 10-point discretisation error (-2.3 %; the host
    solver's test shows the error vanishing with more points)."""
    L, EI, mu, npts, dt = 1.0, 0.0259, 0.0571, 10, 0.02
    seg = L / (npts - 1)
    x0 = np.zeros((npts, 3))
    x0[:, 0] = np.linspace(0.0, L, npts)
    mass = np.full(npts, mu * seg)
    mass[-1] = 0.5 * mu * seg
    fixed = np.zeros(npts, bool)
    fixed[:2] = True
    net = M.Network(x0, mass, fixed, [(i, i + 1) for i in range(npts - 1)], np.full(npts - 1, 1e5),
                    [(i, i + 1, i + 2) for i in range(npts - 2)], np.full(npts - 2, M.kb_from_EI(EI, L, npts - 2)))
    fe = np.zeros((npts, 3))
    fe[-1, 1] = -1e-5
    x = M.equilibrium(net, fe, steps=1, tol=1e-13)
    v = np.zeros_like(x)
    xm1 = vm1 = None
    ys = []
    for _ in range(int(5.5 / dt)):
        xn, vn, _ = M.bdf2_step(net, x, v, xm1, vm1, dt, dt, np.zeros_like(x), tol=1e-12)
        xm1, vm1, x, v = x, v, xn, vn
        ys.append(x[-1, 1])
    ys = np.array(ys)
    ts = dt * np.arange(1, len(ys) + 1)
    up = [ts[i] - ys[i] * dt / (ys[i + 1] - ys[i]) for i in range(len(ys) - 1) if ys[i] < 0 <= ys[i + 1]]
    period = up[1] - up[0]
    want = 2 * math.pi / (1.8751040687 ** 2 * math.sqrt(EI / (mu * L ** 4)))
    assert abs(period / want - 1) < 0.03, (period, want)
