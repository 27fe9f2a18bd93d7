"""Pins of the oracle adjoint: central finite differences of the oracle's own
forward map in FP64 (the definition of the derivative) and a dot-product
check of the step's linear part."""
import math

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import mask as OM
from oracle import step as S
from paper_2002_08642_gb300 import inputs


def _setup(n=16, K=4, seed=0):
    L = 4.0
    p = S.Params(n=n, L=L, nu=0.02, eta=0.05, dt=2e-3, x0=(1.9, 2.1, 2.05))
    rng = np.random.default_rng(seed)
    u0 = inputs.random_field(n, L, seed=seed + 3, rms=0.5)
    masks = []
    for k in range(K):
        chi = np.zeros((n, n, n))
        chi[4:10, 5:11, 6:12] = rng.uniform(0.2, 1.0, (6, 6, 6))
        us = rng.standard_normal((3, n, n, n)) * 0.1
        masks.append((chi, us))
    w = np.full(K, 1.0 / K)
    a = np.array([0.3, -0.2, 1.0])
    b = np.array([0.1, 0.4, -0.3])
    return p, u0, masks, w, a, b


def test_mask_gradient_matches_central_differences():
    p, u0, masks, w, a, b = _setup()
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi, gus = OA.adjoint(p, states, masks, w, a, b)
    rng = np.random.default_rng(5)
    for k in (0, 2, 3):
        dchi = np.zeros_like(masks[k][0])
        dchi[4:10, 5:11, 6:12] = rng.uniform(-1, 1, (6, 6, 6))
        h = 1e-5
        mp = [m if i != k else (m[0] + h * dchi, m[1]) for i, m in enumerate(masks)]
        mm = [m if i != k else (m[0] - h * dchi, m[1]) for i, m in enumerate(masks)]
        fd = (OA.forward(p, u0, mp, w, a, b)[0] - OA.forward(p, u0, mm, w, a, b)[0]) / (2 * h)
        ad = float(np.sum(gchi[k] * dchi))
        assert abs(fd - ad) < 1e-7 * max(abs(fd), 1e-12), (k, fd, ad)


def test_solid_velocity_gradient_matches_central_differences():
    p, u0, masks, w, a, b = _setup(seed=1)
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi, gus = OA.adjoint(p, states, masks, w, a, b)
    rng = np.random.default_rng(6)
    for k in (0, 1, 3):
        dus = rng.standard_normal(masks[k][1].shape)
        h = 1e-5
        mp = [m if i != k else (m[0], m[1] + h * dus) for i, m in enumerate(masks)]
        mm = [m if i != k else (m[0], m[1] - h * dus) for i, m in enumerate(masks)]
        fd = (OA.forward(p, u0, mp, w, a, b)[0] - OA.forward(p, u0, mm, w, a, b)[0]) / (2 * h)
        ad = float(np.sum(gus[k] * dus))
        assert abs(fd - ad) < 1e-7 * max(abs(fd), 1e-12), (k, fd, ad)


def test_force_only_gradient_is_closed_form():
    """One step, zero velocity: J = a . F^0 with F^0 = (dx^3/eta) sum chi (0 - us),
    so dJ/dchi = -(dx^3/eta) a . us and dJ/dus = -(dx^3/eta) chi a exactly."""
    n, L = 8, 4.0
    p = S.Params(n=n, L=L, nu=0.01, eta=0.5, dt=1e-3, x0=(2, 2, 2))
    rng = np.random.default_rng(2)
    chi = rng.uniform(0, 1, (n, n, n))
    us = rng.standard_normal((3, n, n, n))
    a = np.array([1.0, 2.0, -1.0])
    b = np.zeros(3)
    J, states = OA.forward(p, np.zeros((3, n, n, n)), [(chi, us)], [1.0], a, b)
    gchi, gus = OA.adjoint(p, states, [(chi, us)], [1.0], a, b)
    dx3 = (L / n) ** 3
    assert np.allclose(gchi[0], -dx3 / p.eta * np.einsum("c,c...->...", a, us), atol=1e-15)
    assert np.allclose(gus[0], -dx3 / p.eta * chi[None] * a[:, None, None, None], atol=1e-15)


def _wing_J(n, L, xw, vw, tri, fr, cb, ub):
    dx = L / n
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
    return float(np.sum(cb * chi) + np.sum(ub * us))


def test_rasterise_vjp_matches_central_differences():
    n, L = 32, 4.0
    dx = L / n
    xw0, tri = inputs.elliptic_wing_mesh(60)
    amp = inputs.flapping_amplitudes(xw0)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, amp)
    vw = vw + np.random.default_rng(3).standard_normal(vw.shape) * 0.3
    rng = np.random.default_rng(4)
    cb = rng.standard_normal((n, n, n))
    ub = rng.standard_normal((3, n, n, n))
    g = OA.rasterise_vjp(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, cb, ub)
    h = 1e-6
    errs = []
    for node in rng.choice(len(xw), 8, replace=False):
        for c in range(3):
            xp = xw.copy(); xp[node, c] += h
            xm = xw.copy(); xm[node, c] -= h
            fd = (_wing_J(n, L, xp, vw, tri, fr, cb, ub) - _wing_J(n, L, xm, vw, tri, fr, cb, ub)) / (2 * h)
            errs.append(abs(fd - g[node, c]) / max(abs(fd), abs(g[node, c]), 1e-3))
    errs = np.array(errs)
    assert np.median(errs) < 1e-5 and np.mean(errs < 1e-4) > 0.9, errs
