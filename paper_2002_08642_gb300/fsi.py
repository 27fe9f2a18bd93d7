"""Staggered fluid-structure coupling of Sec. 4.1 (coupling paragraph):
per time step the fluid goes u^n -> u^{n+1} with the old mask chi^n and
solid velocity u_s^n (GPU step), the pressure p^{n+1} follows from u^{n+1}
(GPU), its loads on the wing's mass points drive the mass-spring network
from t^n to t^{n+1} in the wing frame (host, ps_ms_*), and the new node
positions and velocities give chi^{n+1}, u_s^{n+1} (GPU rasteriser, Eq.
relative_velocities for the solid velocity).

The loads are taken on the wing as the fluid saw it (nodes x^n, frame at
t^n), turned into wing axes, and held over the solid step; the network's
moving frame is the wing frame at t^{n+1}.
"""
import time

import numpy as np
import torch

from .massspring import MassSpring


class FSI:
    """Couples a ``Solver`` (GPU) and a ``MassSpring`` network (host).

    frames(t) -> (frame dict R, X_O, V_O, Omega for the rasteriser and the
    loads, frame dict A_O, Omega, dOmega of the network in wing axes).
    The node copies run on torch's current stream, which must be the
    solver's stream (the default). A solver created with keep_uw=True
    skips the x- and y-inverse passes of every step after the first."""

    def __init__(self, solver, ms: MassSpring, tri, frames, t0=0.0, tol=1e-8, max_iter=20):
        self.solver = solver
        self.ms = ms
        self.frames = frames
        self.t = float(t0)
        self.dt = float(solver.params.dt)
        self.tol, self.max_iter = tol, max_iter
        dev = solver.device
        self.tri = torch.as_tensor(np.ascontiguousarray(tri), dtype=torch.int32).to(dev).contiguous()
        n = ms.n
        self.xw = torch.empty((n, 3), dtype=torch.float64, device=dev)
        self.vw = torch.empty((n, 3), dtype=torch.float64, device=dev)
        self._host_x = torch.empty((2, n, 3), dtype=torch.float64).pin_memory() if dev.type == "cuda" else \
            torch.empty((2, n, 3), dtype=torch.float64)
        self._host_f = torch.empty((n, 3), dtype=torch.float64).pin_memory() if dev.type == "cuda" else \
            torch.empty((n, 3), dtype=torch.float64)
        self.p = None
        self.f_wing = np.zeros((n, 3))
        self.newton_iters = []
        self.host_solid_s = 0.0   # wall time spent in the network's steps
        self._upload_and_mask()

    def _upload_and_mask(self):
        x, v = self.ms.state()
        self._host_x[0].numpy()[:] = x
        self._host_x[1].numpy()[:] = v
        self.xw.copy_(self._host_x[0], non_blocking=True)
        self.vw.copy_(self._host_x[1], non_blocking=True)
        fr, _ = self.frames(self.t)
        self.solver.set_mask_from_nodes(self.xw, self.vw, self.tri, fr)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            fr_n, _ = self.frames(self.t)
            self.solver.step(1)
            self.p = self.solver.pressure(out=self.p)
            _, fn = self.solver.pressure_loads(self.p, self.xw, self.tri, fr_n)
            self._host_f.copy_(fn)   # synchronises: the solid step needs the loads
            R = np.asarray(fr_n["R"], dtype=np.float64).reshape(3, 3)
            self.f_wing = self._host_f.numpy() @ R   # rows R^T f
            _, ms_fr = self.frames(self.t + self.dt)
            t0 = time.perf_counter()
            self.newton_iters.append(self.ms.step(self.dt, self.f_wing, frame=ms_fr, tol=self.tol,
                                                  max_iter=self.max_iter))
            self.host_solid_s += time.perf_counter() - t0
            self.t += self.dt
            self._upload_and_mask()

    def state(self):
        """Wing-frame node positions and velocities (host)."""
        return self.ms.state()

    def save(self, path):
        """Checkpoint of the coupled state to a host file: the fluid's
        time-stepping state, the network's (with its BDF2 history) and the
        time. The mask is not stored: ``load`` rasterises it again from the
        restored nodes."""
        buf = self.solver.state_buffer()
        self.solver.save_state(buf)
        ms = np.frombuffer(self.ms.save(), dtype=np.uint8)
        np.savez(path, fluid=buf.cpu().numpy(), ms=ms, t=self.t, dt=self.dt)

    def load(self, path):
        """Resume from ``save`` (same solver parameters and network inputs):
        the coupled steps that follow give the same results as the run that
        was saved."""
        with np.load(path) as f:
            if float(f["dt"]) != self.dt:
                raise ValueError("checkpoint dt %s, coupling has %s" % (float(f["dt"]), self.dt))
            fluid = torch.from_numpy(np.ascontiguousarray(f["fluid"]))
            ms = f["ms"].tobytes()
            t = float(f["t"])
        buf = self.solver.state_buffer()
        buf.copy_(fluid)
        self.solver.restore_state(buf)
        self.ms.restore(ms)
        self.t = t
        self._upload_and_mask()
