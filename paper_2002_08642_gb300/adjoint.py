"""Gradients of the time-averaged penalization force and moment with respect
to the wing's node positions, through the library's discrete adjoint
(ps_adjoint_step, ps_mask_nodes_vjp) with checkpointed recompute.

The objective over a window of K steps is
    J = sum_c g_c * mean_n F^n_c + sum_c h_c * mean_n M^n_c
(g, h the incoming gradient of the 6-vector output). Node positions enter
through the mask and solid velocity rasterised at every step from
x^(w)_n = x^(w)_0 + d_n (d_n the prescribed deformation of step n), so
dJ/dx^(w)_0 = sum_n dJ/dx^(w)_n.
"""
import torch


class WingWindow:
    """The prescribed part of a window: per-step deformations, node
    velocities and frames, the triangle list, the initial velocity."""

    def __init__(self, tri, disp, vw, frames, u0):
        self.tri = tri          # (n_tri, 3) int32 cuda
        self.disp = disp        # list of (n_nodes, 3) float64 cuda
        self.vw = vw            # list of (n_nodes, 3) float64 cuda
        self.frames = frames    # list of frame dicts
        self.u0 = u0            # (3, n, n, nz) cuda, solver dtype
        self.steps = len(frames)


class TimeAveragedForce(torch.autograd.Function):
    """forward(xw0, solver, window, every) -> (mean F, mean M) as a 6-vector;
    backward gives dJ/dxw0. ``every`` is the checkpoint interval in steps."""

    @staticmethod
    def forward(ctx, xw0, solver, win, every):
        K = win.steps
        solver.set_velocity(win.u0)
        ckpts = {}
        acc = torch.zeros(6, dtype=torch.float64)
        for k in range(K):
            if k % every == 0:
                buf = solver.state_buffer()
                solver.save_state(buf)
                ckpts[k] = buf
            solver.set_mask_from_nodes((xw0 + win.disp[k]).contiguous(), win.vw[k], win.tri, win.frames[k])
            solver.step(1)
            F, M = solver.forces()
            acc += torch.tensor(list(F) + list(M), dtype=torch.float64)
        ctx.solver, ctx.win, ctx.every, ctx.ckpts = solver, win, every, ckpts
        ctx.save_for_backward(xw0)
        return (acc / K).to(xw0.device)

    @staticmethod
    def backward(ctx, gout):
        (xw0,) = ctx.saved_tensors
        solver, win, every, ckpts = ctx.solver, ctx.win, ctx.every, ctx.ckpts
        K = win.steps
        g = gout.detach().double().cpu().numpy() / K
        a, b = g[:3], g[3:]
        n, nz = solver.n, solver.nz
        gchi = torch.empty((n, n, nz), dtype=solver.dtype, device=solver.device)
        gus = torch.empty((3, n, n, nz), dtype=solver.dtype, device=solver.device)
        gxw = torch.zeros_like(xw0, dtype=torch.float64)
        solver.adjoint_reset()
        starts = sorted(ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + every, K)
            solver.restore_state(ckpts[s0])
            states = []
            for k in range(s0, s1):
                buf = solver.state_buffer()
                solver.save_state(buf)
                states.append(buf)
                if k < s1 - 1:
                    solver.set_mask_from_nodes((xw0 + win.disp[k]).contiguous(), win.vw[k], win.tri, win.frames[k])
                    solver.step(1)
            for k in range(s1 - 1, s0 - 1, -1):
                solver.restore_state(states[k - s0])
                xk = (xw0 + win.disp[k]).contiguous()
                solver.set_mask_from_nodes(xk, win.vw[k], win.tri, win.frames[k])
                solver.adjoint_step(a, b, k == 0, gchi, gus)
                solver.mask_nodes_vjp(gchi, gus, gxw)
        torch.cuda.synchronize(solver.device)
        return gxw.to(xw0.dtype), None, None, None
