"""Oracle mask chi and solid velocity u_s from a triangulated wing.

Test infrastructure only (see ``oracle/__init__``).

Follows Sec. 4.1:

* Eq. (mask_function): chi(delta) = 1 for delta <= t_w - h,
  (1/2)(1 + cos(pi (delta - t_w + h) / (2h))) for t_w - h < delta < t_w + h,
  0 for delta >= t_w + h (t_w the wing semi-thickness, h the smoothing
  semi-width).
* delta(x) = min over triangles of the Euclidean distance from the grid point
  to the triangle; each triangle is only tested against the grid points of
  its bounding box (here dilated by t_w + h, the reach of the mask; no
  periodic images).
* u_s: on the closest triangle, the velocity of the closest point is the
  barycentric interpolation of the three vertex velocities; the frame
  transform of Eq. (relative_velocities) gives
      u_s = V_O + R v^(w) + Omega x (x - X_O)
  with the rigid term taken at the fluid node x itself (the paper's remark
  that the projected point and the fluid node share one velocity).
  Node global positions are X_O + R x^(w).

Readings: ties in delta go to the smallest triangle id;
u_s is set where chi > 0 in the banded (cosine) mode and is 0 elsewhere; the
alternative tanh profile chi = (1/2)(1 - tanh((delta - t_w)/h)) is evaluated
at every grid point with the minimum over all triangles.
"""
import math

import numpy as np

PROFILE_COS = 0
PROFILE_TANH = 1


def chi_cos(delta, tw, h):
    """Eq. (mask_function)."""
    delta = np.asarray(delta, dtype=np.float64)
    out = np.where(delta <= tw - h, 1.0, 0.0)
    ramp = (delta > tw - h) & (delta < tw + h)
    out = np.where(ramp, 0.5 * (1.0 + np.cos(math.pi * (delta - tw + h) / (2.0 * h))), out)
    return out


def chi_tanh(delta, tw, h):
    return 0.5 * (1.0 - np.tanh((np.asarray(delta, dtype=np.float64) - tw) / h))


def _closest_on_segment(P, A, B):
    """Closest point on segment AB to points P (..., 3); returns (t, point)."""
    AB = B - A
    t = np.sum((P - A) * AB, axis=-1) / np.dot(AB, AB)
    t = np.clip(t, 0.0, 1.0)
    return t, A + t[..., None] * AB


def closest_point_on_triangle(P, A, B, C):
    """Closest point of triangle ABC to each point P (..., 3).

    Returns (distance, beta) with beta (..., 3) the barycentric weights of the
    closest point on (A, B, C). Construction: solve for the orthogonal
    projection onto the plane in barycentric form; if all weights are >= 0 it
    is the answer, otherwise the closest point lies on the boundary, found as
    the nearest of the three clamped edge projections.
    """
    P = np.asarray(P, dtype=np.float64)
    e0 = B - A
    e1 = C - A
    d = P - A
    a00 = np.dot(e0, e0)
    a01 = np.dot(e0, e1)
    a11 = np.dot(e1, e1)
    b0 = np.sum(d * e0, axis=-1)
    b1 = np.sum(d * e1, axis=-1)
    det = a00 * a11 - a01 * a01
    s = (a11 * b0 - a01 * b1) / det
    t = (a00 * b1 - a01 * b0) / det
    inside = (s >= 0) & (t >= 0) & (s + t <= 1)

    proj = A + s[..., None] * e0 + t[..., None] * e1
    dist_in = np.linalg.norm(P - proj, axis=-1)
    beta_in = np.stack([1.0 - s - t, s, t], axis=-1)

    best_d = np.full(P.shape[:-1], np.inf)
    best_b = np.zeros(P.shape[:-1] + (3,))
    # edges (A,B), (B,C), (C,A) with their barycentric embeddings
    for (U, V, iu, iv) in ((A, B, 0, 1), (B, C, 1, 2), (C, A, 2, 0)):
        te, q = _closest_on_segment(P, U, V)
        de = np.linalg.norm(P - q, axis=-1)
        better = de < best_d
        bb = np.zeros(P.shape[:-1] + (3,))
        bb[..., iu] = 1.0 - te
        bb[..., iv] = te
        best_d = np.where(better, de, best_d)
        best_b = np.where(better[..., None], bb, best_b)

    dist = np.where(inside, dist_in, best_d)
    beta = np.where(inside[..., None], beta_in, best_b)
    return dist, beta


def global_nodes(xw, frame):
    R = np.asarray(frame["R"], dtype=np.float64).reshape(3, 3)
    return np.asarray(frame["X_O"], dtype=np.float64)[None] + np.asarray(xw) @ R.T


def rasterise(n, L, xw, vw, tri, frame, tw, h, profile=PROFILE_COS, nz=None):
    """chi [n,n,nz] and u_s [3,n,n,nz] (and the argmin triangle per point);
    grid points (i, j, k) L/n, nz = n unless given.

    xw, vw: (n_nodes, 3) wing-frame positions and velocities; tri: (n_tri, 3)
    vertex indices; frame: dict with R (3x3 row-major, wing -> global), X_O,
    V_O, Omega.
    """
    dx = L / n
    nz = n if nz is None else nz
    dims = np.array([n, n, nz])
    R = np.asarray(frame["R"], dtype=np.float64).reshape(3, 3)
    XO = np.asarray(frame["X_O"], dtype=np.float64)
    VO = np.asarray(frame["V_O"], dtype=np.float64)
    Om = np.asarray(frame["Omega"], dtype=np.float64)
    xg = global_nodes(xw, frame)
    vw = np.asarray(vw, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)

    best = np.full((n, n, nz), np.inf)
    arg = np.full((n, n, nz), -1, dtype=np.int64)
    beta = np.zeros((n, n, nz, 3))
    reach = tw + h
    for t_id in range(tri.shape[0]):
        A, B, C = xg[tri[t_id, 0]], xg[tri[t_id, 1]], xg[tri[t_id, 2]]
        if profile == PROFILE_COS:
            lo = np.minimum(np.minimum(A, B), C) - reach
            hi = np.maximum(np.maximum(A, B), C) + reach
            i0 = np.maximum(np.ceil(lo / dx).astype(int), 0)
            i1 = np.minimum(np.floor(hi / dx).astype(int), dims - 1)
            if np.any(i1 < i0):
                continue
        else:
            i0 = np.array([0, 0, 0])
            i1 = dims - 1
        gx = np.arange(i0[0], i1[0] + 1) * dx
        gy = np.arange(i0[1], i1[1] + 1) * dx
        gz = np.arange(i0[2], i1[2] + 1) * dx
        P = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), axis=-1)
        d, b = closest_point_on_triangle(P, A, B, C)
        sl = (slice(i0[0], i1[0] + 1), slice(i0[1], i1[1] + 1), slice(i0[2], i1[2] + 1))
        better = d < best[sl]          # strict: earlier (smaller) id wins ties
        best[sl] = np.where(better, d, best[sl])
        arg[sl] = np.where(better, t_id, arg[sl])
        beta[sl] = np.where(better[..., None], b, beta[sl])

    if profile == PROFILE_COS:
        chi = np.where(arg >= 0, chi_cos(np.where(arg >= 0, best, 0.0), tw, h), 0.0)
        active = chi > 0.0
    else:
        chi = chi_tanh(best, tw, h)
        active = arg >= 0

    # velocity of the closest point: barycentric blend of wing-frame vertex velocities
    safe = np.where(arg >= 0, arg, 0)
    tv = tri[safe]                                   # (n,n,n,3) vertex ids
    vloc = np.einsum("...v,...vc->...c", beta, vw[tv])
    vglob = vloc @ R.T
    X = np.arange(n) * dx
    XX = np.stack(np.meshgrid(X, X, np.arange(nz) * dx, indexing="ij"), axis=-1)
    r = XX - XO
    rot = np.cross(np.broadcast_to(Om, r.shape), r)
    us = VO + vglob + rot
    us = np.where(active[..., None], us, 0.0)
    return chi, np.moveaxis(us, -1, 0), np.where(active, arg, -1), best
