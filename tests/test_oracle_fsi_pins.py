"""Pins of the oracle's staggered coupling loop (oracle/fsi.py, Sec. 4.1,
coupling paragraph) against values that do not come from the loop itself.

1. Every node fixed: the network never moves, so the loop must reduce to the
   fluid step with the mask of the frame at t^n during step n (bit for bit
   against the oracle's Solver stepped by hand with masks rasterised at
   t0 + k dt). A mask taken from the frame at t^{n+1} fails it.
2. A free triangle (no springs) in a 2-D Taylor--Green flow whose
   penalization is negligible (eta = 1e300): the fluid decays exactly as
   exp(-2 nu t) under the integrating-factor scheme, so the static pressure
   after step n is the closed form p(t^{n+1}) = [(cos 2x + cos 2y)/4 - 1/4]
   exp(-4 nu t^{n+1}). With no internal or frame forces the BDF2 step of
   Eq. (discretized_ODEs) is explicit in the load, so the node trajectory is
   a recurrence written out here: loads of p(t^{n+1}) at the nodes as the
   fluid saw them (wing frame at t^n, translating with a constant velocity),
   rotated into wing axes by R^T, held over the step. Loads from p(t^n), from
   the frame at t^{n+1}, or rotated by R instead of R^T each move the nodes
   elsewhere (checked below by planting each mistake in a copy of the loop).
"""
import math

import numpy as np

from oracle import fsi as OF
from oracle import mask as OM
from oracle import massspring as OMS
from oracle import pressure as OP
from oracle import step as S


def _rotz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _tg2d(n, L):
    x = np.arange(n) * (L / n)
    X, Y = x[:, None, None], x[None, :, None]
    zero = np.zeros((n, n, n))
    return np.stack([np.sin(X) * np.cos(Y) + zero, -np.cos(X) * np.sin(Y) + zero, zero])


def test_all_nodes_fixed_reduces_to_step_and_rasterise_at_t_n():
    n, L = 16, 4.0
    dx = L / n
    p = S.Params(n=n, L=L, nu=2e-3, eta=2e-2, dt=1.0 / 64, x0=(2.0, 2.0, 2.0))   # dyadic times: t += dt is exact
    x0 = np.array([[0.0, 0.0, 0.0], [0.8, 0.0, 0.0], [0.0, 0.5, 0.0], [0.8, 0.5, 0.1]])
    tri = np.array([[0, 1, 2], [1, 3, 2]])
    net = OMS.Network(x0, np.ones(4), np.ones(4, dtype=bool), np.zeros((0, 2)), [], np.zeros((0, 3)), [])
    omega = 3.0

    def frames(t):
        R = _rotz(omega * t)
        fr = {"R": R.ravel(), "X_O": (2.0, 2.0, 2.0), "V_O": (0.0, 0.0, 0.0), "Omega": (0.0, 0.0, omega)}
        return fr, {"A_O": (0.0, 0.0, 0.0), "Omega": (0.0, 0.0, omega), "dOmega": (0.0, 0.0, 0.0)}

    rng = np.random.default_rng(3)
    u0 = 0.2 * rng.standard_normal((3, n, n, n))
    t0, K = 0.125, 3
    o = OF.Coupled(p, net, tri, frames, u0, 2 * dx, 1.5 * dx, t0=t0)
    o.step(K)

    ref = S.Solver(p)
    ref.set_velocity(u0)
    zero_v = np.zeros_like(x0)
    for k in range(K):
        fr, _ = frames(t0 + k * p.dt)
        chi, us, _, _ = OM.rasterise(n, L, x0, zero_v, tri, fr, 2 * dx, 1.5 * dx)
        ref.set_mask(chi, us)
        ref.step(1)
    assert np.array_equal(o.fluid.uh, ref.uh)
    assert np.array_equal(o.x, x0) and np.all(o.v == 0.0)
    # and the mask the loop holds afterwards is the frame at t0 + K dt
    fr, _ = frames(t0 + K * p.dt)
    chi, _, _, _ = OM.rasterise(n, L, x0, zero_v, tri, fr, 2 * dx, 1.5 * dx)
    assert np.array_equal(o.fluid.chi, chi)
    # a mask from the frame at t^{n+1} during step n would differ
    fr1, _ = frames(t0 + p.dt)
    chi1, _, _, _ = OM.rasterise(n, L, x0, zero_v, tri, fr1, 2 * dx, 1.5 * dx)
    fr0, _ = frames(t0)
    chi0, _, _, _ = OM.rasterise(n, L, x0, zero_v, tri, fr0, 2 * dx, 1.5 * dx)
    assert np.abs(chi1 - chi0).max() > 1e-2


class _Setup:
    n, L = 16, 2 * math.pi
    nu, dt, K = 0.5, 1.0 / 16, 4   # dyadic times: the loop's t += dt is exact
    t0 = 0.25
    R = _rotz(math.pi / 6)
    V = np.array([0.4, -0.3, 0.2])
    X0 = np.array([3.0, 2.9, 3.1])
    mass = np.array([0.02, 0.03, 0.025])
    xw0 = np.array([[0.0, 0.0, 0.0], [0.9, 0.1, 0.0], [0.2, 0.7, 0.15]])
    tri = np.array([[0, 1, 2]])

    def frames(self, t):
        fr = {"R": self.R.ravel(), "X_O": tuple(self.X0 + self.V * t), "V_O": tuple(self.V),
              "Omega": (0.0, 0.0, 0.0)}
        return fr, {"A_O": (0.0, 0.0, 0.0), "Omega": (0.0, 0.0, 0.0), "dOmega": (0.0, 0.0, 0.0)}

    def params(self):
        return S.Params(n=self.n, L=self.L, nu=self.nu, eta=1e300, dt=self.dt, x0=(3.0, 3.0, 3.0))

    def net(self):
        return OMS.Network(self.xw0, self.mass, np.zeros(3, dtype=bool), np.zeros((0, 2)), [], np.zeros((0, 3)),
                           [])

    def pressure_grid(self, t):
        x = np.arange(self.n) * (self.L / self.n)
        X, Y = x[:, None, None], x[None, :, None]
        # the flow starts as the Taylor--Green field at t0
        p = (0.25 * (np.cos(2 * X) + np.cos(2 * Y)) - 0.25) * math.exp(-4 * self.nu * (t - self.t0))
        return p + np.zeros((self.n, self.n, self.n))

    def loads_wing(self, x_wing, t_frame, t_pressure, rot_T=True):
        """Loads of p(t_pressure) on the triangle seen in the frame at
        t_frame, in wing axes."""
        xg = (self.X0 + self.V * t_frame)[None] + x_wing @ self.R.T
        pv = OP.interpolate(self.pressure_grid(t_pressure), self.L, xg)
        a, b, c = xg
        nA6 = np.cross(b - a, c - a) / 6.0
        fg = -pv[:, None] * nA6[None]
        return fg @ self.R if rot_T else fg @ self.R.T

    def trajectory(self, **mistake):
        """BDF2 of m dv/dt = f^n (loads held over the step), written out:
        backward Euler first, then constant-step BDF2 (xi = 1)."""
        x, v = self.xw0.copy(), np.zeros_like(self.xw0)
        xm1 = vm1 = None
        m = self.mass[:, None]
        out = []
        for k in range(self.K):
            tn = self.t0 + k * self.dt
            tf = tn + self.dt if mistake.get("frame_next") else tn
            tp = tn if mistake.get("pressure_old") else tn + self.dt
            f = self.loads_wing(x, tf, tp, rot_T=not mistake.get("rot_R"))
            if xm1 is None:
                vn = v + self.dt * f / m
                xn = x + self.dt * vn
            else:
                vn = (4 * v - vm1) / 3 + (2.0 / 3.0) * self.dt * f / m
                xn = (4 * x - xm1) / 3 + (2.0 / 3.0) * self.dt * vn
            xm1, vm1, x, v = x, v, xn, vn
            out.append(x.copy())
        return out


def test_free_triangle_follows_bdf2_with_loads_of_p_n_plus_1_at_frame_t_n():
    s = _Setup()
    p = s.params()
    dx = s.L / s.n
    o = OF.Coupled(p, s.net(), s.tri, s.frames, _tg2d(s.n, s.L), 2 * dx, 1.5 * dx, t0=s.t0, tol=1e-13)
    expect = s.trajectory()
    got = []
    for _ in range(s.K):
        o.step(1)
        got.append(o.x.copy())
    scale = max(np.abs(e - s.xw0).max() for e in expect)
    assert scale > 1e-3   # the loads move the nodes visibly
    for g, e in zip(got, expect):
        assert np.abs(g - e).max() < 1e-9 * scale, np.abs(g - e).max() / scale
    # the fluid itself is the exact Taylor--Green decay
    u = o.fluid.velocity()
    ref = _tg2d(s.n, s.L) * math.exp(-2 * s.nu * s.K * s.dt)
    assert np.abs(u - ref).max() < 1e-13


def test_free_triangle_pin_rejects_each_planted_timing_mistake():
    """Each plausible mistake in the loop's order moves the nodes by far more
    than the pin's tolerance: the pin can tell them apart."""
    s = _Setup()
    right = s.trajectory()
    scale = max(np.abs(e - s.xw0).max() for e in right)
    for mistake in ("frame_next", "pressure_old", "rot_R"):
        wrong = s.trajectory(**{mistake: True})
        dev = max(np.abs(w - r).max() for w, r in zip(wrong, right))
        assert dev > 1e-4 * scale, (mistake, dev / scale)
