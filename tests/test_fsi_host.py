"""Host logic of the coupling loop (paper_2002_08642_gb300/fsi.py) on the CPU:
the product's FSI class drives a stand-in fluid solver whose calls are the
oracle's routines and the product's host mass-spring network; the order of
its calls, the frames it passes and the load rotation R^T F must reproduce
the oracle's coupled loop (Sec. 4.1, coupling paragraph)."""
import types

import numpy as np
import torch

from oracle import fsi as OF
from oracle import mask as OM
from oracle import massspring as OMS
from oracle import pressure as OP
from oracle import step as S
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.fsi import FSI
from paper_2002_08642_gb300.massspring import MassSpring


class OracleFluid:
    """The Solver calls FSI makes, answered by the oracle on the CPU."""

    def __init__(self, p, u0, tw, h):
        self.p = p
        self.device = torch.device("cpu")
        self.params = types.SimpleNamespace(dt=p.dt)
        self.fluid = S.Solver(p)
        self.fluid.set_velocity(u0)
        self.tw, self.h = tw, h
        self.calls = []

    def set_mask_from_nodes(self, xw, vw, tri, frame):
        self.calls.append("mask")
        chi, us, _, _ = OM.rasterise(self.p.n, self.p.L, xw.numpy(), vw.numpy(), tri.numpy(), frame, self.tw,
                                     self.h)
        self.fluid.set_mask(chi, us)

    def step(self, k):
        self.calls.append("step")
        self.fluid.step(k)

    def pressure(self, out=None):
        self.calls.append("pressure")
        return torch.from_numpy(OP.static_pressure(self.p, self.fluid.uh, self.fluid.chi, self.fluid.us))

    def state_buffer(self):
        return torch.empty(2 * self.fluid.uh.nbytes + 8, dtype=torch.uint8)

    def save_state(self, buf):
        b = buf.numpy()
        nb = self.fluid.uh.nbytes
        b[:nb] = np.frombuffer(self.fluid.uh.tobytes(), dtype=np.uint8)
        b[nb:2 * nb] = np.frombuffer(self.fluid.Nprev.tobytes(), dtype=np.uint8)
        b[2 * nb:] = np.frombuffer(np.int64(self.fluid.nstep).tobytes(), dtype=np.uint8)

    def restore_state(self, buf):
        b = buf.numpy()
        nb = self.fluid.uh.nbytes
        shape = self.fluid.uh.shape
        self.fluid.uh = np.frombuffer(b[:nb].tobytes(), dtype=np.complex128).reshape(shape).copy()
        self.fluid.Nprev = np.frombuffer(b[nb:2 * nb].tobytes(), dtype=np.complex128).reshape(shape).copy()
        self.fluid.nstep = int(np.frombuffer(b[2 * nb:].tobytes(), dtype=np.int64)[0])

    def pressure_loads(self, pf, xw, tri, frame):
        self.calls.append("loads")
        xg = OM.global_nodes(xw.numpy(), frame)
        pn = OP.interpolate(pf.numpy(), self.p.L, xg)
        return torch.from_numpy(pn), torch.from_numpy(OP.node_loads(pn, xg, tri.numpy()))


def test_coupling_order_frames_and_load_rotation():
    pbuild.build()
    n, L, nu, eta, dt = 16, 4.0, 1.527e-4, 1e-2, 2e-3
    w = inputs.fsi_wing(ns=4, nc=2, veins=(0, 2), kb=0.05, ke=20.0, mass=0.05)

    def frames(t):
        return inputs.revolving_frames(t, tau=0.05)

    u0 = inputs.random_field(n, L, seed=5, rms=0.3)
    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0))
    tw, h = 2 * L / n, 1.5 * L / n
    net = OMS.Network(w["x0"], w["mass"], w["fixed"], w["ext"], w["ke"], w["bend"], w["kb"])
    o = OF.Coupled(p, net, w["tri"], frames, u0, tw, h, tol=1e-12)
    o.step(2)
    fake = OracleFluid(p, u0, tw, h)
    ms = MassSpring(w["x0"], w["mass"], w["ext"], w["ke"], w["bend"], w["kb"], fixed=w["fixed"])
    c = FSI(fake, ms, w["tri"], frames, tol=1e-12)
    c.step(2)
    assert fake.calls == ["mask"] + ["step", "pressure", "loads", "mask"] * 2
    x, v = c.state()
    assert np.max(np.abs(o.x - w["x0"])) > 1e-7
    assert np.max(np.abs(x - o.x)) < 1e-8 * np.max(np.abs(o.x - w["x0"])) + 1e-14
    assert np.max(np.abs(v - o.v)) < 1e-6 * np.max(np.abs(o.v))
    assert abs(c.t - 2 * dt) < 1e-15


def test_coupled_checkpoint_resume(tmp_path):
    """FSI.save / FSI.load: a coupled run resumed from a checkpoint file
    (fluid state, network state with its BDF2 history, time; the mask
    rasterised again from the restored nodes) continues with the same
    results as the run that was saved."""
    pbuild.build()
    n, L, nu, eta, dt = 16, 4.0, 1.527e-4, 1e-2, 2e-3
    w = inputs.fsi_wing(ns=4, nc=2, veins=(0, 2), kb=0.05, ke=20.0, mass=0.05)

    def frames(t):
        return inputs.revolving_frames(t, tau=0.05)

    u0 = inputs.random_field(n, L, seed=6, rms=0.3)
    p = S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0))
    tw, h = 2 * L / n, 1.5 * L / n

    def make():
        ms = MassSpring(w["x0"], w["mass"], w["ext"], w["ke"], w["bend"], w["kb"], fixed=w["fixed"])
        fake = OracleFluid(p, u0, tw, h)
        return fake, FSI(fake, ms, w["tri"], frames, tol=1e-12)

    fa, a = make()
    a.step(1)
    a.save(tmp_path / "fsi.npz")
    a.step(2)
    fb, b = make()
    b.load(tmp_path / "fsi.npz")
    b.step(2)
    xa, va = a.state()
    xb, vb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(fa.fluid.uh, fb.fluid.uh) and b.t == a.t
