"""ctypes binding of libps (include/ps.h): the same entry points, argument
marshalling only. Every computation runs in the CUDA library; there is no
fallback path. PyTorch supplies device memory (the workspace, fields) and the
CUDA stream.
"""
import ctypes
import os
import re

from . import build as _build

c_int32 = ctypes.c_int32
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p

PS_OK, PS_EINVAL, PS_ENOMEM, PS_ECUDA, PS_ESTATE, PS_EUNSUPPORTED, PS_ENUMERIC = range(7)
PS_FP32, PS_FP64 = 0, 1
PS_MASK_COS, PS_MASK_TANH = 0, 1
PS_MEAN_FIXED, PS_MEAN_FREE = 0, 1

STATUS_NAMES = {0: "PS_OK", 1: "PS_EINVAL", 2: "PS_ENOMEM", 3: "PS_ECUDA", 4: "PS_ESTATE",
                5: "PS_EUNSUPPORTED", 6: "PS_ENUMERIC"}


class PsParams(ctypes.Structure):
    _fields_ = [("n", c_int32), ("precision", c_int32), ("mask_profile", c_int32), ("mean_mode", c_int32),
                ("with_adjoint", c_int32), ("L", c_double), ("nu", c_double), ("eta", c_double), ("dt", c_double),
                ("tw", c_double), ("h", c_double), ("x0", c_double * 3), ("keep_uw", c_int32),
                ("nz", c_int32)]


class PsFrame(ctypes.Structure):
    _fields_ = [("R", c_double * 9), ("X_O", c_double * 3), ("V_O", c_double * 3), ("Omega", c_double * 3)]


class PsMsFrame(ctypes.Structure):
    _fields_ = [("A_O", c_double * 3), ("Omega", c_double * 3), ("dOmega", c_double * 3)]


class PsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_P = ctypes.POINTER
_SIGS = {
    "ps_supported_n": (c_int32, [_P(c_int32), c_int32, _P(c_int32)]),
    "ps_workspace_size": (c_int32, [_P(PsParams), _P(c_size_t)]),
    "ps_init": (c_int32, [_P(PsParams), c_void_p, c_void_p, c_size_t, _P(c_void_p)]),
    "ps_destroy": (c_int32, [c_void_p]),
    "ps_set_velocity": (c_int32, [c_void_p, c_void_p]),
    "ps_get_velocity": (c_int32, [c_void_p, c_void_p]),
    "ps_set_mask": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ps_get_mask": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ps_set_mask_from_nodes": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32, _P(PsFrame)]),
    "ps_step": (c_int32, [c_void_p, c_int32]),
    "ps_forces": (c_int32, [c_void_p, _P(c_double), _P(c_double)]),
    "ps_diagnostics": (c_int32, [c_void_p, _P(c_double), _P(c_double)]),
    "ps_clear_error": (c_int32, [c_void_p]),
    "ps_grid_info": (c_int32, [c_void_p, _P(c_int32), _P(c_int32), _P(c_int32)]),
    "ps_slab_set": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32]),
    "ps_slab_phase": (c_int32, [c_void_p, c_int32]),
    "ps_slab_buffer": (c_int32, [c_void_p, _P(c_void_p), _P(c_size_t)]),
    "ps_debug_wait_timeout": (c_int32, [c_void_p, c_int32]),
    "ps_pressure": (c_int32, [c_void_p, c_void_p]),
    "ps_set_sponge": (c_int32, [c_void_p, c_void_p, c_double]),
    "ps_pressure_loads": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32, _P(PsFrame),
                                    c_void_p, c_void_p]),
    "ps_state_size": (c_int32, [c_void_p, _P(c_size_t)]),
    "ps_save_state": (c_int32, [c_void_p, c_void_p]),
    "ps_restore_state": (c_int32, [c_void_p, c_void_p]),
    "ps_adjoint_reset": (c_int32, [c_void_p]),
    "ps_adjoint_step": (c_int32, [c_void_p, _P(c_double), _P(c_double), c_int32, c_void_p, c_void_p]),
    "ps_mask_nodes_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ps_timing_enable": (c_int32, [c_void_p, c_int32]),
    "ps_timing_read": (c_int32, [c_void_p, _P(c_double), _P(ctypes.c_int64), c_int32, _P(c_int32)]),
    "ps_timing_name": (ctypes.c_char_p, [c_int32]),
    "ps_last_error": (ctypes.c_char_p, [c_void_p]),
    "ps_penalization_force_noalloc": (c_int32, [c_int32, c_int32, c_double, c_double, _P(c_double), c_void_p,
                                                c_void_p, c_void_p, c_void_p, c_void_p]),
    "ps_ms_create": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                               c_int32, c_void_p, c_void_p, _P(c_void_p)]),
    "ps_ms_destroy": (c_int32, [c_void_p]),
    "ps_ms_info": (c_int32, [c_void_p, _P(c_int32), _P(c_int32), _P(ctypes.c_int64)]),
    "ps_ms_forces": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ps_ms_state": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ps_ms_set_state": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ps_ms_step": (c_int32, [c_void_p, c_double, c_void_p, _P(PsMsFrame), c_double, c_int32, _P(c_int32)]),
    "ps_ms_equilibrium": (c_int32, [c_void_p, c_void_p, c_int32, c_double, c_int32, _P(c_int32)]),
    "ps_ms_last_error": (ctypes.c_char_p, [c_void_p]),
    "ps_ms_state_size": (c_int32, [c_void_p, _P(c_size_t)]),
    "ps_ms_save": (c_int32, [c_void_p, c_void_p]),
    "ps_ms_restore": (c_int32, [c_void_p, c_void_p]),
}

_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libps.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libps.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def header_symbols(header=None):
    """Names of the functions declared in include/ps.h."""
    header = header or os.path.join(_build.INCLUDE, "ps.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", text)))


def check(status, ctx=None):
    if status != PS_OK:
        msg = ""
        if ctx:
            raw = lib().ps_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise PsError(status, msg)


# ------------------------------------------------------------------ thin calls
def ps_supported_n():
    L = lib()
    cnt = c_int32(0)
    check(L.ps_supported_n(None, 0, ctypes.byref(cnt)))
    arr = (c_int32 * cnt.value)()
    check(L.ps_supported_n(arr, cnt.value, ctypes.byref(cnt)))
    return list(arr)


def ps_workspace_size(params):
    out = c_size_t(0)
    check(lib().ps_workspace_size(ctypes.byref(params), ctypes.byref(out)))
    return out.value


def ps_init(params, stream_ptr, workspace_ptr, workspace_bytes):
    ctx = c_void_p(0)
    check(lib().ps_init(ctypes.byref(params), c_void_p(stream_ptr), c_void_p(workspace_ptr),
                        workspace_bytes, ctypes.byref(ctx)))
    return ctx


def ps_destroy(ctx):
    check(lib().ps_destroy(ctx))


def ps_set_velocity(ctx, u_ptr):
    check(lib().ps_set_velocity(ctx, c_void_p(u_ptr)), ctx)


def ps_get_velocity(ctx, u_ptr):
    check(lib().ps_get_velocity(ctx, c_void_p(u_ptr)), ctx)


def ps_set_mask(ctx, chi_ptr, us_ptr):
    check(lib().ps_set_mask(ctx, c_void_p(chi_ptr), c_void_p(us_ptr)), ctx)


def ps_get_mask(ctx, chi_ptr, us_ptr):
    check(lib().ps_get_mask(ctx, c_void_p(chi_ptr), c_void_p(us_ptr)), ctx)


def ps_set_mask_from_nodes(ctx, xw_ptr, vw_ptr, n_nodes, tri_ptr, n_tri, frame):
    check(lib().ps_set_mask_from_nodes(ctx, c_void_p(xw_ptr), c_void_p(vw_ptr), n_nodes, c_void_p(tri_ptr),
                                       n_tri, ctypes.byref(frame)), ctx)


def ps_step(ctx, nsteps):
    check(lib().ps_step(ctx, nsteps), ctx)


def ps_forces(ctx):
    F = (c_double * 3)()
    M = (c_double * 3)()
    check(lib().ps_forces(ctx, F, M), ctx)
    return list(F), list(M)


def ps_set_sponge(ctx, chi_sp_ptr, c_sp):
    check(lib().ps_set_sponge(ctx, c_void_p(chi_sp_ptr) if chi_sp_ptr else None, float(c_sp)), ctx)


def ps_pressure(ctx, p_ptr):
    check(lib().ps_pressure(ctx, c_void_p(p_ptr)), ctx)


def ps_pressure_loads(ctx, p_ptr, xw_ptr, n_nodes, tri_ptr, n_tri, frame, pn_ptr, fn_ptr):
    check(lib().ps_pressure_loads(ctx, c_void_p(p_ptr), c_void_p(xw_ptr), n_nodes, c_void_p(tri_ptr), n_tri,
                                  ctypes.byref(frame), c_void_p(pn_ptr), c_void_p(fn_ptr)), ctx)


def ps_diagnostics(ctx):
    e = c_double(0)
    d = c_double(0)
    st = lib().ps_diagnostics(ctx, ctypes.byref(e), ctypes.byref(d))
    check(st, ctx)
    return e.value, d.value


def ps_grid_info(ctx):
    K, Kz, Kzp = c_int32(0), c_int32(0), c_int32(0)
    check(lib().ps_grid_info(ctx, ctypes.byref(K), ctypes.byref(Kz), ctypes.byref(Kzp)), ctx)
    return K.value, Kz.value, Kzp.value


def ps_slab_set(ctx, x0, x1, ky0, ky1):
    check(lib().ps_slab_set(ctx, int(x0), int(x1), int(ky0), int(ky1)), ctx)


def ps_slab_phase(ctx, phase):
    check(lib().ps_slab_phase(ctx, int(phase)), ctx)


def ps_slab_buffer(ctx):
    ptr, nb = c_void_p(0), c_size_t(0)
    check(lib().ps_slab_buffer(ctx, ctypes.byref(ptr), ctypes.byref(nb)), ctx)
    return ptr.value, nb.value


def ps_clear_error(ctx):
    check(lib().ps_clear_error(ctx), ctx)


def ps_debug_wait_timeout(ctx, cap):
    check(lib().ps_debug_wait_timeout(ctx, int(cap)), ctx)


def ps_state_size(ctx):
    out = c_size_t(0)
    check(lib().ps_state_size(ctx, ctypes.byref(out)), ctx)
    return out.value


def ps_save_state(ctx, buf_ptr):
    check(lib().ps_save_state(ctx, c_void_p(buf_ptr)), ctx)


def ps_restore_state(ctx, buf_ptr):
    check(lib().ps_restore_state(ctx, c_void_p(buf_ptr)), ctx)


def ps_adjoint_reset(ctx):
    check(lib().ps_adjoint_reset(ctx), ctx)


def ps_adjoint_step(ctx, dJdF, dJdM, first, gchi_ptr, gus_ptr):
    F = (c_double * 3)(*[float(v) for v in dJdF])
    M = (c_double * 3)(*[float(v) for v in dJdM])
    check(lib().ps_adjoint_step(ctx, F, M, 1 if first else 0, c_void_p(gchi_ptr), c_void_p(gus_ptr)), ctx)


def ps_mask_nodes_vjp(ctx, gchi_ptr, gus_ptr, gxw_ptr):
    check(lib().ps_mask_nodes_vjp(ctx, c_void_p(gchi_ptr), c_void_p(gus_ptr), c_void_p(gxw_ptr)), ctx)


def ps_timing_enable(ctx, on):
    check(lib().ps_timing_enable(ctx, 1 if on else 0), ctx)


def ps_timing_read(ctx):
    """{pass name: (total ms, launches)} since ps_timing_enable."""
    cnt = c_int32(0)
    check(lib().ps_timing_read(ctx, None, None, 0, ctypes.byref(cnt)), ctx)
    ms = (c_double * cnt.value)()
    ln = (ctypes.c_int64 * cnt.value)()
    check(lib().ps_timing_read(ctx, ms, ln, cnt.value, ctypes.byref(cnt)), ctx)
    return {lib().ps_timing_name(i).decode(): (ms[i], ln[i]) for i in range(cnt.value)}


def ps_last_error(ctx):
    raw = lib().ps_last_error(ctx)
    return raw.decode() if raw else ""


def ps_penalization_force_noalloc(n, precision, L, eta, x0, u_ptr, chi_ptr, us_ptr, fm_ptr, stream_ptr):
    """Allocation-free force/moment of caller fields into fm (6 device doubles)."""
    x = (c_double * 3)(*[float(v) for v in x0])
    check(lib().ps_penalization_force_noalloc(int(n), int(precision), float(L), float(eta), x, c_void_p(u_ptr),
                                              c_void_p(chi_ptr), c_void_p(us_ptr), c_void_p(fm_ptr),
                                              c_void_p(stream_ptr)))


def make_frame(fr):
    """PsFrame from a dict with R (9 or 3x3), X_O, V_O, Omega."""
    f = PsFrame()
    R = [float(v) for v in (fr["R"].reshape(-1) if hasattr(fr["R"], "reshape") else fr["R"])]
    for i in range(9):
        f.R[i] = R[i]
    for i in range(3):
        f.X_O[i] = float(fr["X_O"][i])
        f.V_O[i] = float(fr.get("V_O", (0, 0, 0))[i])
        f.Omega[i] = float(fr.get("Omega", (0, 0, 0))[i])
    return f


def ms_check(status, m):
    if status != PS_OK:
        raw = lib().ps_ms_last_error(m) if m else None
        raise PsError(status, raw.decode() if raw else "")


def ps_ms_create(n_nodes, mass_ptr, x0_ptr, v0_ptr, fixed_ptr, n_ext, ext_ptr, ke_ptr, n_bend, bend_ptr, kb_ptr):
    m = c_void_p(0)
    check(lib().ps_ms_create(int(n_nodes), c_void_p(mass_ptr), c_void_p(x0_ptr), c_void_p(v0_ptr),
                             c_void_p(fixed_ptr), int(n_ext), c_void_p(ext_ptr), c_void_p(ke_ptr), int(n_bend),
                             c_void_p(bend_ptr), c_void_p(kb_ptr), ctypes.byref(m)))
    return m


def ps_ms_destroy(m):
    check(lib().ps_ms_destroy(m))


def ps_ms_info(m):
    nf, bw, nfac = c_int32(0), c_int32(0), ctypes.c_int64(0)
    ms_check(lib().ps_ms_info(m, ctypes.byref(nf), ctypes.byref(bw), ctypes.byref(nfac)), m)
    return nf.value, bw.value, nfac.value


def ps_ms_forces(m, x_ptr, f_ptr):
    ms_check(lib().ps_ms_forces(m, c_void_p(x_ptr), c_void_p(f_ptr)), m)


def ps_ms_state(m, x_ptr, v_ptr):
    ms_check(lib().ps_ms_state(m, c_void_p(x_ptr), c_void_p(v_ptr)), m)


def ps_ms_set_state(m, x_ptr, v_ptr):
    ms_check(lib().ps_ms_set_state(m, c_void_p(x_ptr), c_void_p(v_ptr)), m)


def ps_ms_step(m, dt, fext_ptr, frame, tol, max_iter):
    it = c_int32(0)
    fr = ctypes.byref(frame) if frame is not None else None
    ms_check(lib().ps_ms_step(m, float(dt), c_void_p(fext_ptr), fr, float(tol), int(max_iter), ctypes.byref(it)), m)
    return it.value


def ps_ms_equilibrium(m, fext_ptr, load_steps, tol, max_iter):
    it = c_int32(0)
    ms_check(lib().ps_ms_equilibrium(m, c_void_p(fext_ptr), int(load_steps), float(tol), int(max_iter),
                                     ctypes.byref(it)), m)
    return it.value


def make_ms_frame(A_O=(0.0, 0.0, 0.0), Omega=(0.0, 0.0, 0.0), dOmega=(0.0, 0.0, 0.0)):
    f = PsMsFrame()
    for i in range(3):
        f.A_O[i], f.Omega[i], f.dOmega[i] = float(A_O[i]), float(Omega[i]), float(dOmega[i])
    return f


def ps_ms_save(m):
    """The network's state as bytes."""
    nb = c_size_t(0)
    ms_check(lib().ps_ms_state_size(m, ctypes.byref(nb)), m)
    buf = ctypes.create_string_buffer(nb.value)
    ms_check(lib().ps_ms_save(m, buf), m)
    return buf.raw


def ps_ms_restore(m, data):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    ms_check(lib().ps_ms_restore(m, buf), m)
