"""Python face of libps: a Solver owning one context, its workspace tensor
and its stream. Tensors are checked and their device pointers handed to the
C ABI; nothing is computed here.
"""
import math

import numpy as np
import torch

from . import binding as B

_PREC = {"fp32": B.PS_FP32, "fp64": B.PS_FP64}
_PROFILE = {"cos": B.PS_MASK_COS, "tanh": B.PS_MASK_TANH}
_MEAN = {"fixed": B.PS_MEAN_FIXED, "free": B.PS_MEAN_FREE}


def make_params(n, L, nu, eta, dt, precision="fp32", mask_profile="cos", mean_mode="fixed",
                tw=None, h=None, x0=None, with_adjoint=False, keep_uw=False, nz=None):
    """nz: points along z (None: n); the box is [0, L)^2 x [0, L nz / n)."""
    dx = L / n
    p = B.PsParams()
    p.n = int(n)
    p.nz = int(n if nz is None else nz)
    p.precision = _PREC[precision]
    p.mask_profile = _PROFILE[mask_profile]
    p.mean_mode = _MEAN[mean_mode]
    p.with_adjoint = 1 if with_adjoint else 0
    p.keep_uw = 1 if keep_uw else 0
    p.L, p.nu, p.eta, p.dt = float(L), float(nu), float(eta), float(dt)
    p.tw = float(2.0 * dx if tw is None else tw)
    p.h = float(1.5 * dx if h is None else h)
    Lz = L * p.nz / p.n
    x0 = (0.5 * L, 0.5 * L, 0.5 * Lz) if x0 is None else x0
    for i in range(3):
        p.x0[i] = float(x0[i])
    return p


class Solver:
    """One penalized pseudo-spectral solver on one CUDA device."""

    def __init__(self, n, L, nu, eta, dt, precision="fp32", mask_profile="cos", mean_mode="fixed",
                 tw=None, h=None, x0=None, device=None, stream=None, with_adjoint=False, keep_uw=False,
                 nz=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libps needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.params = make_params(n, L, nu, eta, dt, precision, mask_profile, mean_mode, tw, h, x0, with_adjoint,
                                  keep_uw, nz)
        self.n = int(n)
        self.nz = int(self.params.nz)
        self.L = float(L)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.precision = precision
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            nbytes = B.ps_workspace_size(self.params)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = B.ps_init(self.params, self.stream.cuda_stream, self.workspace.data_ptr(), nbytes)

    def close(self):
        if getattr(self, "ctx", None):
            B.ps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- checks
    def _field(self, t, comps, name):
        n, nz = self.n, self.nz
        shape = (comps, n, n, nz) if comps > 1 else (n, n, nz)
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype:
            raise ValueError("%s must be a %s tensor on %s" % (name, self.dtype, self.device))
        if tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError("%s must be contiguous with shape %s" % (name, shape))
        return t.data_ptr()

    # ---------------------------------------------------------------- API
    def set_velocity(self, u):
        B.ps_set_velocity(self.ctx, self._field(u, 3, "u"))

    def velocity(self, out=None):
        n, nz = self.n, self.nz
        if out is None:
            out = torch.empty((3, n, n, nz), dtype=self.dtype, device=self.device)
        B.ps_get_velocity(self.ctx, self._field(out, 3, "out"))
        return out

    def set_mask(self, chi, us):
        B.ps_set_mask(self.ctx, self._field(chi, 1, "chi"), self._field(us, 3, "us"))

    def mask(self):
        n, nz = self.n, self.nz
        chi = torch.empty((n, n, nz), dtype=self.dtype, device=self.device)
        us = torch.empty((3, n, n, nz), dtype=self.dtype, device=self.device)
        B.ps_get_mask(self.ctx, chi.data_ptr(), us.data_ptr())
        return chi, us

    def set_mask_from_nodes(self, xw, vw, tri, frame):
        for t, nm, dt in ((xw, "xw", torch.float64), (vw, "vw", torch.float64), (tri, "tri", torch.int32)):
            if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dt or not t.is_contiguous():
                raise ValueError("%s must be a contiguous %s tensor on %s" % (nm, dt, self.device))
            if t.dim() != 2 or t.shape[1] != 3:
                raise ValueError("%s must have shape (k, 3)" % nm)
        if xw.shape != vw.shape:
            raise ValueError("xw and vw must have the same shape")
        B.ps_set_mask_from_nodes(self.ctx, xw.data_ptr(), vw.data_ptr(), xw.shape[0], tri.data_ptr(),
                                 tri.shape[0], B.make_frame(frame))

    def step(self, nsteps=1):
        B.ps_step(self.ctx, int(nsteps))

    def forces(self):
        return B.ps_forces(self.ctx)

    def set_sponge(self, chi_sp, c_sp=1.0):
        """Turn the sponge term on with mask chi_sp (kept referenced: the
        library reads it every step) or off with None."""
        if chi_sp is None:
            B.ps_set_sponge(self.ctx, 0, 0.0)
            self._sponge = None
            return
        B.ps_set_sponge(self.ctx, self._field(chi_sp, 1, "chi_sp"), c_sp)
        self._sponge = chi_sp

    def pressure(self, out=None):
        """Static pressure p = Pi - (1/2)|u|^2 of the current state and mask."""
        n, nz = self.n, self.nz
        if out is None:
            out = torch.empty((n, n, nz), dtype=self.dtype, device=self.device)
        B.ps_pressure(self.ctx, self._field(out, 1, "out"))
        return out

    def pressure_loads(self, p, xw, tri, frame):
        """(p at the nodes, node forces (global frame)) from the pressure p."""
        for t, nm, dt in ((xw, "xw", torch.float64), (tri, "tri", torch.int32)):
            if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dt or not t.is_contiguous():
                raise ValueError("%s must be a contiguous %s tensor on %s" % (nm, dt, self.device))
            if t.dim() != 2 or t.shape[1] != 3:
                raise ValueError("%s must have shape (k, 3)" % nm)
        pn = torch.empty(xw.shape[0], dtype=torch.float64, device=self.device)
        fn = torch.empty((xw.shape[0], 3), dtype=torch.float64, device=self.device)
        B.ps_pressure_loads(self.ctx, self._field(p, 1, "p"), xw.data_ptr(), xw.shape[0], tri.data_ptr(),
                            tri.shape[0], B.make_frame(frame), pn.data_ptr(), fn.data_ptr())
        return pn, fn

    def diagnostics(self):
        return B.ps_diagnostics(self.ctx)

    def clear_error(self):
        """Reset the sticky device error flag (see ps_clear_error)."""
        B.ps_clear_error(self.ctx)

    def adjoint_reset(self):
        B.ps_adjoint_reset(self.ctx)

    def adjoint_step(self, dJdF, dJdM, first, grad_chi, grad_us):
        """Reverse one step (see include/ps.h); grad_chi, grad_us are overwritten."""
        B.ps_adjoint_step(self.ctx, dJdF, dJdM, first, self._field(grad_chi, 1, "grad_chi"),
                          self._field(grad_us, 3, "grad_us"))

    def mask_nodes_vjp(self, grad_chi, grad_us, grad_xw):
        """Add dJ/dx^(w) of the last rasterised wing to grad_xw (n_nodes x 3 float64)."""
        if grad_xw.dtype != torch.float64 or grad_xw.device != self.device or not grad_xw.is_contiguous():
            raise ValueError("grad_xw must be a contiguous float64 tensor on %s" % self.device)
        B.ps_mask_nodes_vjp(self.ctx, self._field(grad_chi, 1, "grad_chi"), self._field(grad_us, 3, "grad_us"),
                            grad_xw.data_ptr())

    def timing(self, on=True):
        B.ps_timing_enable(self.ctx, on)

    def timing_read(self):
        return B.ps_timing_read(self.ctx)

    def state_buffer(self):
        return torch.empty(B.ps_state_size(self.ctx), dtype=torch.uint8, device=self.device)

    def save_state(self, buf):
        B.ps_save_state(self.ctx, buf.data_ptr())

    def restore_state(self, buf):
        B.ps_restore_state(self.ctx, buf.data_ptr())

    def save_checkpoint(self, path):
        """Write the time-stepping state (spectral velocity, AB2 history,
        step counter) and the parameters it belongs to to a host file."""
        buf = self.state_buffer()
        self.save_state(buf)
        p = self.params
        np.savez(path, state=buf.cpu().numpy(), n=p.n, precision=p.precision, L=p.L, nu=p.nu, eta=p.eta,
                 dt=p.dt)

    def load_checkpoint(self, path):
        """Restore a state written by ``save_checkpoint`` of a solver with the
        same grid, precision and parameters (ValueError otherwise)."""
        with np.load(path) as f:
            p = self.params
            for k in ("n", "precision", "L", "nu", "eta", "dt"):
                if float(f[k]) != float(getattr(p, k)):
                    raise ValueError("checkpoint %s = %s, solver has %s" % (k, f[k], getattr(p, k)))
            state = torch.from_numpy(np.ascontiguousarray(f["state"]))
        buf = self.state_buffer()
        if state.numel() != buf.numel():
            raise ValueError("checkpoint state size does not match")
        buf.copy_(state)
        self.restore_state(buf)
