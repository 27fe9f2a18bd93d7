"""Oracle pressure and pressure loads on the wing nodes.

Test infrastructure only (see ``oracle/__init__``).

Follows Sec. 4.1:

* Total pressure Pi = p + (1/2) u.u (the rotational form of the penalized
  Navier--Stokes equation). With div u = 0 the Leray projection removes
  exactly the gradient part -i k Pi_hat of the right-hand side, so
      Pi_hat = -i (k . N_hat) / |k|^2,   Pi_hat(0) = 0,
  with N_hat the truncated transform of u x omega - (chi/eta)(u - u_s) (the
  same term the step projects). The static pressure is p = Pi - (1/2)|u|^2.
  It is evaluated for the current state and the current mask (the paper
  computes p^{n+1} from u^{n+1} before the solid moves).
* Pressure at a mass point by discrete delta interpolation, product of one
  kernel per axis. The paper cites the smoothing technique of Yang et al.
  without printing a kernel; the reading here: the 4-point cosine kernel
      phi(r) = (1/4)(1 + cos(pi r / 2)),  |r| <= 2,
  convolved with the unit box, phi_s(r) = int_{r-1/2}^{r+1/2} phi(s) ds
  (support |r| < 5/2, five points per axis, periodic grid).
* Load on the mass points: every triangle gives each of its three vertices
  the force -p_v (A/3) n (n its unit normal from the vertex order, A its
  area), summed over the triangles of the vertex; p_v the interpolated
  pressure at that vertex.
"""
import math

import numpy as np

from . import fft as offt
from . import step as S


def total_pressure_hat(p, uh, chi, us):
    """Pi_hat (half spectrum, unnormalised DFT convention of ``oracle.step``)
    and the physical velocity of the state uh."""
    keep = S.dealias_mask(p.n, p.nz)
    wh = S.curl_hat(p, uh) * keep
    u = S.to_physical(uh, p.nz)
    w = S.to_physical(wh, p.nz)
    Nh = S.to_spectral(S.nonlinear_physical(u, w, chi, us, p.eta)) * keep
    kx, ky, kz = S.wavevectors(p)
    k2 = kx * kx + ky * ky + kz * kz
    k2_safe = np.where(k2 == 0.0, 1.0, k2)
    Pih = -1j * (kx * Nh[0] + ky * Nh[1] + kz * Nh[2]) / k2_safe
    Pih[0, 0, 0] = 0.0
    return Pih, u


def static_pressure(p, uh, chi, us):
    """p = Pi - (1/2)|u|^2 on the grid."""
    Pih, u = total_pressure_hat(p, uh, chi, us)
    return offt.irfft3(Pih, p.nz) - 0.5 * np.sum(u * u, axis=0)


def delta_cos4(r):
    r = np.abs(np.asarray(r, dtype=np.float64))
    return np.where(r <= 2.0, 0.25 * (1.0 + np.cos(0.5 * math.pi * r)), 0.0)


def delta_smoothed(r):
    """phi_s(r) = int_{r-1/2}^{r+1/2} phi(s) ds in closed form."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    c = 2.0 / math.pi
    inner = 0.25 * (1.0 + c * (np.sin(0.5 * math.pi * (r + 0.5)) - np.sin(0.5 * math.pi * (r - 0.5))))
    outer = 0.25 * ((2.5 - r) - c * np.sin(0.5 * math.pi * (r - 0.5)))
    return np.where(r <= 1.5, inner, np.where(r < 2.5, outer, 0.0))


def interpolate(pf, L, X):
    """Delta interpolation of the grid field pf (n x n x nz, periodic, grid
    spacing L/n on every axis) at points X (m, 3) with the smoothed kernel."""
    n = pf.shape[0]
    dims = pf.shape
    dx = L / n
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    for m in range(X.shape[0]):
        g = X[m] / dx
        lo = np.floor(g).astype(int) - 2
        idx = [np.arange(lo[a], lo[a] + 6) for a in range(3)]
        w = [delta_smoothed(g[a] - idx[a]) for a in range(3)]
        sub = pf[np.ix_(idx[0] % dims[0], idx[1] % dims[1], idx[2] % dims[2])]
        out[m] = np.einsum("i,j,k,ijk->", w[0], w[1], w[2], sub)
    return out


def node_loads(p_nodes, xg, tri):
    """Force on every node (global frame): sum over its triangles of
    -p_v (A/3) n = -p_v ((b - a) x (c - a)) / 6."""
    xg = np.asarray(xg, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    F = np.zeros_like(xg)
    for t in tri:
        a, b, c = xg[t[0]], xg[t[1]], xg[t[2]]
        nA6 = np.cross(b - a, c - a) / 6.0
        for v in t:
            F[v] -= p_nodes[v] * nA6
    return F


def pressure_loads(p, uh, chi, us, xw, tri, frame):
    """(p on the grid, p at the nodes, node forces) for the state uh, the
    mask (chi, us) and the wing nodes xw (wing frame) of ``frame``."""
    from . import mask as OM

    pf = static_pressure(p, uh, chi, us)
    xg = OM.global_nodes(xw, frame)
    pn = interpolate(pf, p.L, xg)
    return pf, pn, node_loads(pn, xg, tri)
