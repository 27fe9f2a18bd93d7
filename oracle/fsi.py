"""Oracle staggered fluid-structure coupling (Sec. 4.1, coupling
paragraph), composed from the other oracle modules.

Test infrastructure only (see ``oracle/__init__``).

One coupled step, in the paper's order:
1. fluid u^n -> u^{n+1} with the old mask chi^n, u_s^n (``step``);
2. pressure p^{n+1} from u^{n+1} (``pressure.static_pressure``, same mask);
3. its loads on the wing's mass points (``pressure.interpolate`` and
   ``pressure.node_loads``), on the wing as the fluid saw it: nodes x^n,
   frame at t^n; turned into wing axes (R^T F);
4. the mass-spring network advances t^n -> t^{n+1} in the wing frame with
   those loads held over the step (``massspring.bdf2_step``; the frame's
   fictitious forces at t^{n+1});
5. the new nodes give chi^{n+1}, u_s^{n+1} (``mask.rasterise``, the frame at
   t^{n+1}).
"""
import numpy as np

from . import mask as OM
from . import massspring as MS
from . import pressure as OP
from . import step as S


class Coupled:
    """frames(t) -> (rasteriser frame dict, network frame dict), as in the
    product's coupling loop."""

    def __init__(self, params, net, tri, frames, u0, tw, h, t0=0.0, tol=1e-10):
        self.p = params
        self.net = net
        self.tri = np.asarray(tri)
        self.frames = frames
        self.tw, self.h, self.tol = tw, h, tol
        self.t = float(t0)
        self.fluid = S.Solver(params)
        self.fluid.set_velocity(u0)
        self.x = net.x0.copy()
        self.v = np.zeros_like(self.x)
        self.xm1 = self.vm1 = None
        self.dt_prev = None
        self._mask()

    def _mask(self):
        fr, _ = self.frames(self.t)
        chi, us, _, _ = OM.rasterise(self.p.n, self.p.L, self.x, self.v, self.tri, fr, self.tw, self.h,
                                     nz=self.p.nz)
        self.fluid.set_mask(chi, us)

    def step(self, nsteps=1):
        dt = self.p.dt
        for _ in range(nsteps):
            fr_n, _ = self.frames(self.t)
            self.fluid.step(1)
            pf = OP.static_pressure(self.p, self.fluid.uh, self.fluid.chi, self.fluid.us)
            xg = OM.global_nodes(self.x, fr_n)
            fg = OP.node_loads(OP.interpolate(pf, self.p.L, xg), xg, self.tri)
            R = np.asarray(fr_n["R"], dtype=np.float64).reshape(3, 3)
            fw = fg @ R
            _, ms_fr = self.frames(self.t + dt)
            xn, vn, _ = MS.bdf2_step(self.net, self.x, self.v, self.xm1, self.vm1, dt, self.dt_prev, fw,
                                     tol=self.tol, frame=ms_fr)
            self.xm1, self.vm1, self.x, self.v, self.dt_prev = self.x, self.v, xn, vn, dt
            self.t += dt
            self._mask()
