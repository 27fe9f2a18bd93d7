"""Mass-spring network of the wing (Sec. 2.1-2.2) over the C ABI
(``ps_ms_*`` in include/ps.h): extension and bending springs, variable-step
BDF2 with Newton--Raphson, static equilibrium. Host arrays are numpy float64;
the solver itself is the library's native code.
"""
import ctypes

import numpy as np

from . import binding as B


def _ptr(a):
    return a.ctypes.data if a is not None else None


def kb_from_EI(EI, lb, n):
    """Eq. (EI_k_relation): bending stiffness of a vein of length l_b with
    n + 2 mass points (the first two clamped) that stores the energy of an
    Euler--Bernoulli beam of flexural rigidity EI under a tip load."""
    return EI / lb * n * (2 * n + 1) / (2.0 * (n + 1))


class MassSpring:
    """Owns one ``ps_ms`` network. Node arrays are (n, 3) float64."""

    def __init__(self, x0, mass, ext, ke, bend=(), kb=(), fixed=None, v0=None):
        self.x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 3)
        self.n = self.x0.shape[0]
        mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (self.n,)))
        ext = np.ascontiguousarray(ext, dtype=np.int32).reshape(-1, 2)
        ke = np.ascontiguousarray(np.broadcast_to(np.asarray(ke, np.float64), (ext.shape[0],)))
        bend = np.ascontiguousarray(bend, dtype=np.int32).reshape(-1, 3)
        kb = np.ascontiguousarray(np.broadcast_to(np.asarray(kb, np.float64), (bend.shape[0],)))
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
        self.mass = mass
        self.fixed = np.zeros(self.n, bool) if fixed is None else np.asarray(fixed, bool)
        self._m = B.ps_ms_create(self.n, _ptr(mass), _ptr(self.x0), _ptr(v0), _ptr(fx), ext.shape[0], _ptr(ext),
                                 _ptr(ke), bend.shape[0], _ptr(bend), _ptr(kb))

    def close(self):
        if getattr(self, "_m", None):
            B.ps_ms_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """(free nodes, node bandwidth of the Newton matrix, matrices factored)."""
        return B.ps_ms_info(self._m)

    def forces(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n, 3)
        f = np.empty_like(x)
        B.ps_ms_forces(self._m, _ptr(x), _ptr(f))
        return f

    def state(self):
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        B.ps_ms_state(self._m, _ptr(x), _ptr(v))
        return x, v

    def set_state(self, x, v=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        B.ps_ms_set_state(self._m, _ptr(x), _ptr(v))

    def save(self):
        """Time-stepping state (with the BDF2 history) as bytes."""
        return B.ps_ms_save(self._m)

    def restore(self, data):
        """Restore a state from ``save`` of a network built from the same inputs."""
        B.ps_ms_restore(self._m, data)

    def step(self, dt, f_ext=None, frame=None, tol=1e-10, max_iter=30):
        """One BDF2 step; frame = dict(A_O, Omega, dOmega) in the network's
        axes, or None for an inertial frame. Returns Newton iterations."""
        fe = None if f_ext is None else np.ascontiguousarray(f_ext, dtype=np.float64)
        fr = None if frame is None else B.make_ms_frame(**frame)
        return B.ps_ms_step(self._m, dt, _ptr(fe), fr, tol, max_iter)

    def equilibrium(self, f_ext, load_steps=10, tol=1e-10, max_iter=50):
        fe = np.ascontiguousarray(f_ext, dtype=np.float64)
        return B.ps_ms_equilibrium(self._m, _ptr(fe), load_steps, tol, max_iter)


def cantilever(L, EI, npts, ke, mass=1.0):
    """Straight vein along x of npts points on [0, L], the first two fixed,
    extension springs between neighbours and bending springs on consecutive
    triples with k^b from Eq. (EI_k_relation) (the Sec. 2.4.1 test beam)."""
    x0 = np.zeros((npts, 3))
    x0[:, 0] = np.linspace(0.0, L, npts)
    ext = [(i, i + 1) for i in range(npts - 1)]
    bend = [(i, i + 1, i + 2) for i in range(npts - 2)]
    fixed = np.zeros(npts, bool)
    fixed[:2] = True
    return MassSpring(x0, mass, ext, ke, bend, kb_from_EI(EI, L, npts - 2), fixed=fixed)
