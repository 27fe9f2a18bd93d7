"""Oracle mass-spring network (Sec. 2 of the paper: extension and bending
springs, variable-step BDF2 with Newton--Raphson).

Test infrastructure only (see ``oracle/__init__``).

* Extension spring (i, j): energy (1/2) k^e (|x_j - x_i| - l_0)^2, whose
  gradient is the printed force k^e (|x_ij| - l_0) e_ij on i and its
  opposite on j.
* Bending spring (i, j, k): the two projected angles of Eq.
  (two_bending_angles),
      theta^y = atan2[(x_j-x_i)(y_k-y_j) - (x_k-x_j)(y_j-y_i), (x_j-x_i)(x_k-x_j) + (y_j-y_i)(y_k-y_j)],
      theta^z = the same with z for y,
  and the energy (1/2) k^b [(theta^y - theta^y_0)^2 + (theta^z - theta^z_0)^2].
  Reading: the printed force formula (k^b (theta - theta_0) times unit
  vectors) has no lever length and is not the gradient of any energy; the
  forces here are minus the gradient of this energy, which is what the
  k^b - EI relation of Eq. (EI_k_relation) assumes. Here the gradient is
  taken by central differences of the energy.
* Dynamics m_i dv_i/dt = F_int + F_ext (Eq. Newton_law), nodes flagged
  fixed do not move; in a moving frame each node also feels
  -m (A_O + dOmega x x + Omega x (Omega x x) + 2 Omega x v).
  Variable-step BDF2 (Eq. discretized_ODEs),
      q^{n+1} - (1+xi)^2/(1+2xi) q^n + xi^2/(1+2xi) q^{n-1} = (1+xi)/(1+2xi) dt f(q^{n+1}),
  xi = dt^n / dt^{n-1}; the first step is backward Euler (xi = 0). Newton on
  the positions (v eliminated), Jacobian by central differences, stopping at
  a relative or absolute L2 change below tol.
* Parity pinned: the extension force, the small-deflection beam, the
  static large-deflection table, BDF2 order, the backward-Euler start and
  the fictitious forces are each checked against a closed form or the
  paper's printed values in the tests.
"""
import math

import numpy as np


def _angles(xi, xj, xk):
    a = xj - xi
    b = xk - xj
    ty = math.atan2(a[0] * b[1] - b[0] * a[1], a[0] * b[0] + a[1] * b[1])
    tz = math.atan2(a[0] * b[2] - b[0] * a[2], a[0] * b[0] + a[2] * b[2])
    return ty, tz


class Network:
    def __init__(self, x0, mass, fixed, ext, ke, bend, kb):
        self.x0 = np.asarray(x0, dtype=np.float64).copy()
        self.mass = np.asarray(mass, dtype=np.float64)
        self.fixed = np.asarray(fixed, dtype=bool)
        self.ext = np.asarray(ext, dtype=np.int64).reshape(-1, 2)
        self.ke = np.asarray(ke, dtype=np.float64)
        self.bend = np.asarray(bend, dtype=np.int64).reshape(-1, 3)
        self.kb = np.asarray(kb, dtype=np.float64)
        self.l0 = np.array([np.linalg.norm(self.x0[j] - self.x0[i]) for i, j in self.ext])
        self.th0 = np.array([_angles(self.x0[i], self.x0[j], self.x0[k]) for i, j, k in self.bend]).reshape(-1, 2)

    def energy(self, x):
        """Total spring energy at positions x (..., n, 3); leading axes are a
        batch of configurations."""
        x = np.asarray(x, dtype=np.float64)
        e = np.zeros(x.shape[:-2])
        if len(self.ext):
            d = x[..., self.ext[:, 1], :] - x[..., self.ext[:, 0], :]
            e = e + 0.5 * np.sum(self.ke * (np.sqrt(np.sum(d * d, axis=-1)) - self.l0) ** 2, axis=-1)
        if len(self.bend):
            a = x[..., self.bend[:, 1], :] - x[..., self.bend[:, 0], :]
            b = x[..., self.bend[:, 2], :] - x[..., self.bend[:, 1], :]
            ax, ay, az = a[..., 0], a[..., 1], a[..., 2]
            bx, by, bz = b[..., 0], b[..., 1], b[..., 2]
            ty = np.arctan2(ax * by - bx * ay, ax * bx + ay * by)
            tz = np.arctan2(ax * bz - bx * az, ax * bx + az * bz)
            dy = np.angle(np.exp(1j * (ty - self.th0[:, 0])))   # angle change in (-pi, pi]
            dz = np.angle(np.exp(1j * (tz - self.th0[:, 1])))
            e = e + 0.5 * np.sum(self.kb * (dy ** 2 + dz ** 2), axis=-1)
        return e

    def forces(self, x, h=1e-7):
        """-grad energy by central differences (step h times the largest
        coordinate, at least h), all coordinates in one batch."""
        x = np.asarray(x, dtype=np.float64)
        n = x.shape[0]
        d = h * max(1.0, float(np.max(np.abs(x))))
        step = np.eye(3 * n).reshape(3 * n, n, 3) * d
        ep = self.energy(x[None] + step)
        em = self.energy(x[None] - step)
        return (-(ep - em) / (2 * d)).reshape(n, 3)


def _free_index(net):
    return np.repeat(~net.fixed, 3)


def equilibrium(net, f_ext, x_start=None, steps=10, tol=1e-10, max_iter=50):
    """Static equilibrium F_int(x) + f_ext = 0 with fixed nodes at x0, by
    Newton with load stepping (f_ext scaled by s/steps, s = 1..steps)."""
    x = (net.x0 if x_start is None else np.asarray(x_start)).copy()
    free = _free_index(net)
    f_ext = np.asarray(f_ext, dtype=np.float64)
    for s in range(1, steps + 1):
        fe = f_ext * (s / steps)
        for _ in range(max_iter):
            r = (net.forces(x) + fe).ravel()[free]
            J = _fd_jacobian(net, x, free)
            dx = np.linalg.solve(J, -r)
            xf = x.ravel().copy()
            xf[free] += dx
            x = xf.reshape(x.shape)
            if np.linalg.norm(dx) < tol * max(1.0, np.linalg.norm(xf[free])):
                break
    return x


def _fd_jacobian(net, x, free, h=1e-6):
    """d(F_int)/dx on the free coordinates by central differences."""
    idx = np.nonzero(free)[0]
    J = np.zeros((idx.size, idx.size))
    scale = max(1.0, float(np.max(np.abs(x))))
    for col, q in enumerate(idx):
        d = h * scale
        xp = x.ravel().copy(); xp[q] += d
        xm = x.ravel().copy(); xm[q] -= d
        J[:, col] = ((net.forces(xp.reshape(x.shape)) - net.forces(xm.reshape(x.shape))).ravel()[free]) / (2 * d)
    return J


def fictitious_forces(net, x, v, frame):
    """Forces of a moving frame on each node: -m (A_O + dOmega x x +
    Omega x (Omega x x) + 2 Omega x v), frame = dict(A_O, Omega, dOmega) in
    the frame's own axes (the wing frame of Sec. 4.1, Eq.
    relative_velocities, is such a frame)."""
    A = np.asarray(frame.get("A_O", (0.0, 0.0, 0.0)), dtype=np.float64)
    W = np.asarray(frame.get("Omega", (0.0, 0.0, 0.0)), dtype=np.float64)
    dW = np.asarray(frame.get("dOmega", (0.0, 0.0, 0.0)), dtype=np.float64)
    acc = A[None] + np.cross(dW[None], x) + np.cross(W[None], np.cross(W[None], x)) + 2.0 * np.cross(W[None], v)
    return -net.mass[:, None] * acc


def bdf2_step(net, x, v, xm1, vm1, dt, dt_prev, f_ext, tol=1e-10, max_iter=30, frame=None):
    """One variable-step BDF2 step (backward Euler when xm1 is None), in a
    moving frame when ``frame`` is given. Newton on the free positions y
    with v = (y - hx)/(c dt) eliminated; the Jacobian of the whole residual
    by central differences. Returns (x_new, v_new, iterations)."""
    xi = 0.0 if xm1 is None else dt / dt_prev
    a = (1 + xi) ** 2 / (1 + 2 * xi)
    b = xi * xi / (1 + 2 * xi)
    c = (1 + xi) / (1 + 2 * xi)
    xm1 = x if xm1 is None else xm1
    vm1 = v if vm1 is None else vm1
    free = _free_index(net)
    minv = np.repeat(1.0 / net.mass, 3)
    f_ext = np.asarray(f_ext, dtype=np.float64)
    hx = (a * x - b * xm1).ravel()
    hv = (a * v - b * vm1).ravel()

    def residual(yf):
        # velocity equation v(y) - hv - c dt f(y)/m on the free coordinates
        y = yf.reshape(x.shape)
        vy = (yf - hx) / (c * dt)
        F = net.forces(y) + f_ext
        if frame is not None:
            F = F + fictitious_forces(net, y, vy.reshape(x.shape), frame)
        return (vy - hv - c * dt * minv * F.ravel())[free]

    yf = x.ravel().copy()
    idx = np.nonzero(free)[0]
    it = 0
    for it in range(1, max_iter + 1):
        r = residual(yf)
        J = np.zeros((idx.size, idx.size))
        h = 1e-6 * max(1.0, float(np.max(np.abs(yf))))
        for col, q in enumerate(idx):
            yp = yf.copy(); yp[q] += h
            ym = yf.copy(); ym[q] -= h
            J[:, col] = (residual(yp) - residual(ym)) / (2 * h)
        dy = np.linalg.solve(J, -r)
        yf[free] += dy
        if np.linalg.norm(dy) < tol * max(1.0, np.linalg.norm(yf[free])):
            break
    y = yf.reshape(x.shape)
    vnew = ((yf - hx) / (c * dt)).reshape(x.shape)
    vnew[net.fixed] = 0.0
    return y, vnew, it


def kb_from_EI(EI, lb, n):
    """Eq. (EI_k_relation): k^b = (EI / l_b) n (2n + 1) / (2 (n + 1)) for a
    beam of n + 2 mass points (two clamped)."""
    return EI / lb * n * (2 * n + 1) / (2.0 * (n + 1))


def cantilever(L, EI, npts, ke):
    """Straight beam along x of npts points (first two fixed), extension
    springs between neighbours, bending springs on consecutive triples."""
    x0 = np.zeros((npts, 3))
    x0[:, 0] = np.linspace(0.0, L, npts)
    n = npts - 2
    ext = [(i, i + 1) for i in range(npts - 1)]
    bend = [(i, i + 1, i + 2) for i in range(npts - 2)]
    kb = kb_from_EI(EI, L, n)
    fixed = np.zeros(npts, dtype=bool)
    fixed[:2] = True
    return Network(x0, np.ones(npts), fixed, ext, np.full(len(ext), ke), bend, np.full(len(bend), kb))
