"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module builds inputs only: initial velocity fields, wing meshes, node
motions and frames. It holds none of the solver's arithmetic (no transform,
curl, projection, mask profile or force), so that the oracle and the CUDA path
both receive the same arrays and neither borrows the other's numerics.
Library routines (numpy's FFT, scipy's Delaunay) are used for synthesis.

Workload recipes (the configurations the solver is exercised on):

* Taylor--Green 3D: u = (sin x cos y cos z, -cos x sin y cos z, 0) on L = 2 pi.
* Taylor--Green 2D embedded in 3D: u = (sin x cos y, -cos x sin y, 0).
* Random turbulent-like field: complex Gaussian modes with 1 <= |m| < n/3,
  shell amplitudes giving E(k) ~ k^(-5/3), scaled so that after the solver's
  own projection each component has rms ~0.05 (the pre-projection field has
  rms 0.05 * sqrt(3/2); the projection removes one third of the energy of an
  isotropic field on average).
* Flat plate: chord 0.3 (wing x), span 1.0 (wing y), either 2 triangles or a
  structured nc x ns grid of quads split in two, centred at (2, 2, 2) in an
  L = 4 box and pitched 30 degrees about the global y axis; static.
* Elliptic revolving wing: full ellipse with semi-axes 0.175 (chord, wing x)
  and 0.5 (span, wing y), root at the hinge (wing y = 0), tip at y = 1;
  ``n_nodes`` nodes (boundary ring + Vogel-spiral interior, Delaunay
  triangulated); pitched 45 degrees about the span axis and revolving about
  global z at Omega about the hinge at the box centre. Seeded flapping
  displacement d_i(t) = a_i sin(2 pi t) along the wing-frame normal with
  a_i = 0.05 s_i^2 (0.9 + 0.1 zeta_i), zeta_i ~ U[-1, 1], s_i the spanwise
  coordinate.
"""
import math

import numpy as np


def grid(n, L):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, x, indexing="ij")


def taylor_green_3d(n, L=2.0 * math.pi):
    X, Y, Z = grid(n, L)
    return np.stack([np.sin(X) * np.cos(Y) * np.cos(Z),
                     -np.cos(X) * np.sin(Y) * np.cos(Z),
                     np.zeros_like(X)])


def taylor_green_2d(n, L=2.0 * math.pi):
    X, Y, Z = grid(n, L)
    return np.stack([np.sin(X) * np.cos(Y),
                     -np.cos(X) * np.sin(Y),
                     np.zeros_like(X)])


def random_field(n, L, seed=1234, rms=0.05, slope=-5.0 / 3.0, nz=None):
    """Band-limited Gaussian random vector field (not yet solenoidal) on the
    n x n x nz grid (nz = n by default; the spacing L/n on every axis, so a
    z mode m_z has the wavenumber (2 pi / L) m_z n / nz)."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    m = np.fft.fftfreq(n, 1.0 / n)
    mz = np.arange(nz // 2 + 1) * (n / nz)
    MX, MY, MZ = np.meshgrid(m, m, mz, indexing="ij")
    mag = np.sqrt(MX ** 2 + MY ** 2 + MZ ** 2)
    band = (mag >= 1.0) & (mag < n / 3.0)
    # E(k) dk ~ k^slope with ~k^2 modes per shell: |a|^2 ~ k^(slope-2)
    amp = np.where(band, np.power(np.where(band, mag, 1.0), 0.5 * (slope - 2.0)), 0.0)
    u = np.empty((3, n, n, nz))
    for c in range(3):
        z = rng.standard_normal(amp.shape) + 1j * rng.standard_normal(amp.shape)
        u[c] = np.fft.irfftn(z * amp, s=(n, n, nz), axes=(0, 1, 2))
    target = rms * math.sqrt(1.5)
    for c in range(3):
        u[c] *= target / np.sqrt(np.mean(u[c] ** 2))
    return u


def rot_y(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_z(rad):
    c, s = math.cos(rad), math.sin(rad)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def frame(R, X_O, V_O=(0.0, 0.0, 0.0), Omega=(0.0, 0.0, 0.0)):
    return {"R": np.asarray(R, dtype=np.float64).reshape(9),
            "X_O": np.asarray(X_O, dtype=np.float64),
            "V_O": np.asarray(V_O, dtype=np.float64),
            "Omega": np.asarray(Omega, dtype=np.float64)}


def plate(chord=0.3, span=1.0, nc=1, ns=1, centre=(2.0, 2.0, 2.0), pitch_deg=30.0):
    """Static flat plate: wing-frame nodes, zero velocities, triangles, frame."""
    xs = np.linspace(-0.5 * chord, 0.5 * chord, nc + 1)
    ys = np.linspace(-0.5 * span, 0.5 * span, ns + 1)
    XX, YY = np.meshgrid(xs, ys, indexing="ij")
    xw = np.stack([XX.ravel(), YY.ravel(), np.zeros(XX.size)], axis=1)
    tri = []
    for i in range(nc):
        for j in range(ns):
            a = i * (ns + 1) + j
            b = (i + 1) * (ns + 1) + j
            tri.append((a, b, b + 1))
            tri.append((a, b + 1, a + 1))
    tri = np.asarray(tri, dtype=np.int32)
    vw = np.zeros_like(xw)
    return xw, vw, tri, frame(rot_y(pitch_deg), centre)


def elliptic_wing_mesh(n_nodes=600, half_chord=0.175, half_span=0.5):
    """Wing-frame nodes (z = 0) and Delaunay triangles of the ellipse."""
    from scipy.spatial import Delaunay

    n_b = max(16, int(round(2.2 * math.sqrt(n_nodes))))
    n_i = n_nodes - n_b
    th = 2.0 * math.pi * np.arange(n_b) / n_b
    bx = half_chord * np.cos(th)
    by = half_span + half_span * np.sin(th)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    k = np.arange(n_i) + 0.5
    r = 0.93 * np.sqrt(k / n_i)
    ang = golden * k
    ix = half_chord * r * np.cos(ang)
    iy = half_span + half_span * r * np.sin(ang)
    x = np.concatenate([bx, ix])
    y = np.concatenate([by, iy])
    pts = np.stack([x, y], axis=1)
    tri = Delaunay(pts).simplices.astype(np.int32)
    xw = np.stack([x, y, np.zeros_like(x)], axis=1)
    return xw, tri


def flapping_amplitudes(xw, seed=42, amp=0.05):
    rng = np.random.default_rng(seed)
    zeta = rng.uniform(-1.0, 1.0, size=xw.shape[0])
    s = xw[:, 1]
    return amp * s * s * (0.9 + 0.1 * zeta)


def revolving_angle(t, omega=1.0, tau=None):
    """Rotation angle and rate of the revolving wing. tau None: constant rate
    omega. Otherwise the startup of Sec. 4.2 (rigid revolving wing),
    phi(t) = omega (tau e^{-t/tau} + t - tau), rate omega (1 - e^{-t/tau})."""
    if tau is None:
        return omega * t, omega
    e = math.exp(-t / tau)
    return omega * (tau * e + t - tau), omega * (1.0 - e)


def revolving_wing(t, xw0, a, centre=(2.0, 2.0, 2.0), omega=1.0, pitch_deg=45.0, tau=None):
    """Node positions/velocities in the wing frame and the frame at time t
    (tau: optional startup time of the rotation, see ``revolving_angle``)."""
    normal = np.array([0.0, 0.0, 1.0])
    xw = xw0 + (a * math.sin(2.0 * math.pi * t))[:, None] * normal[None]
    vw = (a * 2.0 * math.pi * math.cos(2.0 * math.pi * t))[:, None] * normal[None]
    phi, rate = revolving_angle(t, omega, tau)
    R = rot_z(phi) @ rot_y(pitch_deg)
    return xw, vw, frame(R, centre, (0.0, 0.0, 0.0), (0.0, 0.0, rate))


# Wing frame of the mass-spring wing: span along wing x (the bending angles
# of the network are measured in the x-y and x-z planes, so veins run along
# x), chord along wing y, normal along wing z. P maps the revolving wing's
# axes (span along y) to these; R_fsi = R P^T keeps the global placement.
_P_FSI = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, -1.0]])


def fsi_wing(ns=24, nc=8, span=1.0, half_chord=0.175, veins=(0, 4, 8), kb=1.1, ke=200.0, mass=0.281):
    """Structured mass-spring wing (synthetic recipe in the spirit of the
    vein/membrane model of Sec. 2.3): stations x_i = i span/ns (i = 0..ns),
    chordwise points y_ij = c(x_i) (2 j/nc - 1) (j = 0..nc) with
    c(x) = half_chord (0.35 + 0.65 sqrt(1 - (x/span)^2)); each quad split in
    two triangles. Membrane: an extension spring of stiffness ke on every
    triangle edge. Veins: the spanwise lines j in ``veins`` get bending
    springs of stiffness kb on consecutive triples (kb = 1.1 is what Eq.
    EI_k_relation gives for EI = 0.05 over 23 points of unit length; the
    caller converts). Stations 0 and 1 are clamped (the first two
    points of every vein, as in the cantilever of Sec. 2.3.1). The mass is
    spread equally over the nodes.
    Returns dict(x0, tri, ext, ke, bend, kb, mass, fixed)."""
    n_i, n_j = ns + 1, nc + 1
    xs = np.linspace(0.0, span, n_i)
    c = half_chord * (0.35 + 0.65 * np.sqrt(np.clip(1.0 - (xs / span) ** 2, 0.0, 1.0)))
    x0 = np.zeros((n_i * n_j, 3))
    for i in range(n_i):
        x0[i * n_j:(i + 1) * n_j, 0] = xs[i]
        x0[i * n_j:(i + 1) * n_j, 1] = c[i] * (2.0 * np.arange(n_j) / nc - 1.0)
    tri = []
    for i in range(ns):
        for j in range(nc):
            a, b = i * n_j + j, (i + 1) * n_j + j
            tri.append((a, b, b + 1))
            tri.append((a, b + 1, a + 1))
    tri = np.asarray(tri, dtype=np.int32)
    edges = set()
    for t in tri:
        for u, v in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            edges.add((min(u, v), max(u, v)))
    ext = np.asarray(sorted(edges), dtype=np.int32)
    bend = []
    for j in veins:
        bend += [(i * n_j + j, (i + 1) * n_j + j, (i + 2) * n_j + j) for i in range(ns - 1)]
    bend = np.asarray(bend, dtype=np.int32).reshape(-1, 3)
    fixed = np.zeros(n_i * n_j, dtype=bool)
    fixed[:2 * n_j] = True
    return {"x0": x0, "tri": tri, "ext": ext, "ke": np.full(len(ext), float(ke)), "bend": bend,
            "kb": np.full(len(bend), float(kb)), "mass": np.full(n_i * n_j, mass / (n_i * n_j)), "fixed": fixed}


def revolving_frames(t, centre=(2.0, 2.0, 2.0), omega=1.0, pitch_deg=45.0, tau=None):
    """Frames of the mass-spring wing revolving about global z through
    ``centre`` (the hinge) at angle phi(t) (``revolving_angle``), pitched
    about the span axis. Returns (frame for the rasteriser and the loads,
    frame of the network: A_O, Omega, dOmega in wing axes)."""
    phi, rate = revolving_angle(t, omega, tau)
    R = rot_z(phi) @ rot_y(pitch_deg) @ _P_FSI.T
    acc = 0.0 if tau is None else omega * math.exp(-t / tau) / tau
    Om = np.array([0.0, 0.0, rate])
    ms = {"A_O": (0.0, 0.0, 0.0), "Omega": R.T @ Om, "dOmega": R.T @ np.array([0.0, 0.0, acc])}
    return frame(R, centre, (0.0, 0.0, 0.0), Om), ms
