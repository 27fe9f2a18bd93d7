"""Pins of the oracle pressure and pressure loads (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import pressure as OP
from oracle import step as S


def _grid(n, L):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, x, indexing="ij")


def test_taylor_green_2d_pressure_closed_form():
    """u = (sin x cos y, -cos x sin y, 0): p = (cos 2x + cos 2y)/4 up to the
    constant fixed by mean(Pi) = 0: -mean((1/2)|u|^2) = -1/4."""
    n, L = 16, 2 * math.pi
    p = S.Params(n=n, L=L, nu=0.01, eta=1.0, dt=1e-3)
    X, Y, Z = _grid(n, L)
    u = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y), np.zeros_like(X)])
    uh = S.to_spectral(u)
    pf = OP.static_pressure(p, uh, np.zeros((n, n, n)), np.zeros((3, n, n, n)))
    want = 0.25 * (np.cos(2 * X) + np.cos(2 * Y)) - 0.25
    assert np.max(np.abs(pf - want)) < 1e-13


def test_taylor_green_3d_pressure_closed_form():
    """u = (sin x cos y cos z, -cos x sin y cos z, 0): the classical
    p = (cos 2x + cos 2y)(cos 2z + 2)/16, shifted by -mean((1/2)|u|^2) = -1/8."""
    n, L = 16, 2 * math.pi
    p = S.Params(n=n, L=L, nu=0.01, eta=1.0, dt=1e-3)
    X, Y, Z = _grid(n, L)
    u = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), np.zeros_like(X)])
    pf = OP.static_pressure(p, S.to_spectral(u), np.zeros((n, n, n)), np.zeros((3, n, n, n)))
    want = (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0 - 0.125
    assert np.max(np.abs(pf - want)) < 1e-13


def test_penalization_gradient_gives_pressure():
    """u = 0, chi = c everywhere, u_s = grad phi: N = (c/eta) grad phi is a
    pure gradient, so Pi = (c/eta) phi (pins the sign of the penalization
    term and of Pi_hat = -i k.N/|k|^2)."""
    n, L, c, eta = 16, 2 * math.pi, 0.7, 0.05
    p = S.Params(n=n, L=L, nu=0.0, eta=eta, dt=1e-3)
    X, Y, Z = _grid(n, L)
    phi = np.sin(X) * np.cos(2 * Y) + 0.3 * np.cos(Z)
    us = np.stack([np.cos(X) * np.cos(2 * Y), -2 * np.sin(X) * np.sin(2 * Y), -0.3 * np.sin(Z)])
    uh = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    pf = OP.static_pressure(p, uh, np.full((n, n, n), c), us)
    assert np.max(np.abs(pf - (c / eta) * phi)) < 1e-12


@pytest.mark.parametrize("r", [0.0, 0.3, 0.5, 0.9, 1.5, 1.7, 2.2, 2.49, 2.6])
def test_smoothed_delta_is_the_box_convolution(r):
    got = float(OP.delta_smoothed(r))
    want, _ = integrate.quad(lambda s: float(OP.delta_cos4(s)), r - 0.5, r + 0.5, points=[-2.0, 2.0], epsabs=1e-14)
    assert abs(got - want) < 1e-12
    assert abs(float(OP.delta_smoothed(-r)) - got) < 1e-15


def test_smoothed_delta_partition_of_unity():
    rng = np.random.default_rng(3)
    for r in rng.uniform(0, 1, 50):
        j = np.arange(-4, 5)
        assert abs(np.sum(OP.delta_smoothed(r - j)) - 1.0) < 1e-14


def test_interpolation_of_constant_and_of_a_grid_mode():
    n, L = 12, 3.0
    pf = np.full((n, n, n), 2.5)
    X = np.random.default_rng(4).uniform(0, L, (20, 3))
    assert np.max(np.abs(OP.interpolate(pf, L, X) - 2.5)) < 1e-13
    # a slowly varying periodic field is reproduced to the kernel's accuracy
    n, L = 64, 1.0
    Xg, Yg, Zg = _grid(n, L)
    f = np.cos(2 * math.pi * Xg) + 0.5 * np.sin(2 * math.pi * Zg)
    got = OP.interpolate(f, L, X[:5] / 3.0)
    want = np.cos(2 * math.pi * X[:5, 0] / 3.0) + 0.5 * np.sin(2 * math.pi * X[:5, 2] / 3.0)
    assert np.max(np.abs(got - want)) < 2e-2


def test_node_loads_closed_surface_and_flat_triangle():
    # closed tetrahedron, outward-consistent orientation, uniform pressure
    xg = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    tri = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    F = OP.node_loads(np.full(4, 3.0), xg, tri)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-15
    # one triangle in the z = 0 plane, area 1/2, normal +z, p = 2: total -p A n
    F1 = OP.node_loads(np.full(3, 2.0), xg[:3], np.array([[0, 1, 2]]))
    assert np.allclose(F1.sum(axis=0), [0.0, 0.0, -1.0], atol=1e-15)
    assert np.allclose(F1, [[0, 0, -1.0 / 3]] * 3, atol=1e-15)
