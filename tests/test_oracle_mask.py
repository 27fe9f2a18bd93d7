"""Pins of the oracle mask/solid-velocity rasteriser (Sec. 4.1)."""
import math
import os

import numpy as np
import pytest

from oracle import mask as OM
from paper_2002_08642_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_profile_golden():
    data = np.loadtxt(os.path.join(GOLDEN, "mask_profile.txt"))
    chi = OM.chi_cos(data[:, 0], 2.0, 1.0)
    assert np.max(np.abs(chi - data[:, 1])) < 1e-15


def test_closest_point_vs_dense_sampling():
    rng = np.random.default_rng(0)
    A, B, C = rng.standard_normal(3), rng.standard_normal(3), rng.standard_normal(3)
    P = rng.standard_normal((200, 3)) * 1.5
    d, beta = OM.closest_point_on_triangle(P, A, B, C)
    # the barycentric point is on the triangle and at the stated distance
    assert np.all(beta >= -1e-14) and np.allclose(beta.sum(-1), 1.0)
    q = beta[:, 0:1] * A + beta[:, 1:2] * B + beta[:, 2:3] * C
    assert np.allclose(np.linalg.norm(P - q, axis=-1), d, atol=1e-13)
    # no sampled point of the triangle is closer (up to the sampling pitch)
    m = 160
    s, t = np.meshgrid(np.linspace(0, 1, m + 1), np.linspace(0, 1, m + 1), indexing="ij")
    keep = s + t <= 1 + 1e-12
    S = A + s[keep, None] * (B - A) + t[keep, None] * (C - A)
    dmin = np.min(np.linalg.norm(P[:, None, :] - S[None], axis=-1), axis=1)
    assert np.all(d <= dmin + 1e-12)
    pitch = max(np.linalg.norm(B - A), np.linalg.norm(C - A)) / m
    assert np.all(dmin - d < 2 * pitch)


def test_plate_closed_form_distances():
    """Unpitched 2-triangle plate in z = 2: above the interior delta = |z - 2|;
    beyond the edge x = 2 + c/2 (same y range) delta = hypot(x - edge, z - 2)."""
    xw, vw, tri, fr = inputs.plate(chord=0.3, span=1.0, pitch_deg=0.0)
    xg = OM.global_nodes(xw, fr)
    P = np.array([[2.05, 2.1, 2.03], [1.9, 1.7, 1.96], [2.2, 2.0, 2.04], [2.16, 2.4, 2.0]])
    best = np.full(len(P), np.inf)
    for t in tri:
        d, _ = OM.closest_point_on_triangle(P, *xg[t])
        best = np.minimum(best, d)
    ref = [0.03, 0.04, math.hypot(0.05, 0.04), 0.01]
    assert np.allclose(best, ref, atol=1e-14)


def test_rasterise_matches_bruteforce_and_profile():
    n, L = 32, 4.0
    dx = L / n
    xw0, tri = inputs.elliptic_wing_mesh(120)
    a = inputs.flapping_amplitudes(xw0)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, a)
    tw, h = 2 * dx, 1.5 * dx
    chi, us, arg, best = OM.rasterise(n, L, xw, vw, tri, fr, tw, h)
    xg = OM.global_nodes(xw, fr)
    X = np.stack(inputs.grid(n, L), axis=-1).reshape(-1, 3)
    brute = np.full(X.shape[0], np.inf)
    for t in tri:
        d, _ = OM.closest_point_on_triangle(X, *xg[t])
        brute = np.minimum(brute, d)
    brute = brute.reshape(n, n, n)
    band = brute < tw + h
    assert band.sum() > 100
    assert np.allclose(best[band], brute[band], atol=1e-14)
    assert np.array_equal(chi > 0, band & (brute < tw + h))
    assert np.allclose(chi, OM.chi_cos(np.where(band, brute, 10.0), tw, h), atol=1e-15)


def test_rigid_rotation_velocity():
    """No deformation: u_s = Omega x (x - X_O) wherever chi > 0."""
    n, L = 32, 4.0
    dx = L / n
    xw0, tri = inputs.elliptic_wing_mesh(80)
    xw, vw, fr = inputs.revolving_wing(0.0, xw0, np.zeros(len(xw0)), omega=1.3)
    fr["V_O"] = np.array([0.1, -0.2, 0.05])
    chi, us, arg, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
    X = np.stack(inputs.grid(n, L))
    r = X - np.asarray(fr["X_O"])[:, None, None, None]
    ref = np.stack([-1.3 * r[1], 1.3 * r[0], np.zeros_like(r[0])]) + fr["V_O"][:, None, None, None]
    on = chi > 0
    assert on.sum() > 50
    assert np.allclose(us[:, on], ref[:, on], atol=1e-14)
    assert np.all(us[:, ~on] == 0)


def test_barycentric_reproduces_linear_velocity():
    """Vertex velocities linear in wing position (v = G x_w) are reproduced exactly
    at the closest point: above the plate interior that is the foot point."""
    n, L = 32, 4.0
    dx = L / n
    xw, _, tri, fr = inputs.plate(chord=0.3, span=1.0, nc=3, ns=5, pitch_deg=0.0)
    G = np.array([[0.1, 0.2, 0.0], [-0.3, 0.05, 0.0], [0.4, -0.1, 0.0]])
    vw = xw @ G.T
    chi, us, arg, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
    X = np.stack(inputs.grid(n, L))
    inside = (chi > 0) & (np.abs(X[0] - 2.0) < 0.14) & (np.abs(X[1] - 2.0) < 0.49)
    assert inside.sum() > 20
    foot_w = np.stack([X[0] - 2.0, X[1] - 2.0, np.zeros_like(X[0])])   # R = I, X_O = centre
    ref = np.einsum("ij,j...->i...", G, foot_w)
    assert np.allclose(us[:, inside], ref[:, inside], atol=1e-14)


def test_tanh_profile_dense():
    n, L = 16, 4.0
    dx = L / n
    xw, vw, tri, fr = inputs.plate()
    chi, us, arg, best = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, OM.PROFILE_TANH)
    assert np.all(arg >= 0)
    assert np.allclose(chi, 0.5 * (1 - np.tanh((best - 2 * dx) / (1.5 * dx))), atol=0)
    assert abs(OM.chi_tanh(2 * dx, 2 * dx, 1.5 * dx) - 0.5) < 1e-16


def test_revolving_startup_angle_and_rate():
    """phi(t) = tau e^{-t/tau} + t - tau: phi(0) = 0, phi'(0) = 0, the rate is
    its derivative, and for t >> tau the angle trails the constant-rate one
    by tau."""
    from paper_2002_08642_gb300 import inputs
    tau = 0.4
    assert inputs.revolving_angle(0.0, 1.0, tau) == (0.0, 0.0)
    for t in (0.1, 0.5, 2.0):
        h = 1e-6
        d = (inputs.revolving_angle(t + h, 1.0, tau)[0] - inputs.revolving_angle(t - h, 1.0, tau)[0]) / (2 * h)
        assert abs(d - inputs.revolving_angle(t, 1.0, tau)[1]) < 1e-8
    phi, rate = inputs.revolving_angle(20.0, 1.0, tau)
    assert abs(phi - (20.0 - tau)) < 1e-12 and abs(rate - 1.0) < 1e-12
    assert inputs.revolving_angle(3.0, 2.0, None) == (6.0, 2.0)
