"""Benchmark of the penalized pseudo-spectral step (Sec. 4.1) on one GB300.

One step = rasterise the wing mask and solid velocity from the node
positions of that step (Sec. 4.1, Eq. mask_function / relative_velocities)
+ one integrating-factor AB2 step of the penalized Navier--Stokes equations
with the FP64 force/moment reduction. Metric: Mpts*steps/s = n^3 * steps /
seconds. Inputs are synthetic (seeded revolving elliptic wing, see
paper_2002_08642_gb300/inputs.py) and resident in HBM before timing; the
fields (tens of GB) are far larger than the 129 MB L2, so no flush is needed.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
(test infrastructure, the only other use of ``oracle/`` here) on a bounded
sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # revolving flexible elliptic wing, FP32 bulk, mask rasterised every step
    "wing768": dict(n=768, L=4.0, nodes=2000, nu=1.527e-4, eta=1e-3, dt=5e-4, precision="fp32"),
    "wing384": dict(n=384, L=4.0, nodes=2000, nu=1.527e-4, eta=1e-3, dt=5e-4, precision="fp32"),
    "wing256": dict(n=256, L=4.0, nodes=600, nu=1.527e-4, eta=1e-3, dt=5e-4, precision="fp32"),
    "wing128": dict(n=128, L=4.0, nodes=600, nu=1.527e-4, eta=1e-3, dt=5e-4, precision="fp32"),
    # the paper's revolving-wing box (Sec. 4.2): 4 x 4 x 2 with N x N x N/2 points
    "wing768x384": dict(n=768, nz=384, L=4.0, nodes=2000, nu=1.527e-4, eta=1e-3, dt=5e-4, precision="fp32"),
}

CPU_SAMPLE_N = 48



def fma_peak(precision, iters, stream_ptr):
    """Measured FMA rate (FLOP/s) of the current device from the bench-only
    probe library libps_bench.so; precision 0 = FP32, 1 = FP64."""
    import ctypes

    from paper_2002_08642_gb300 import build as pbuild

    lib = ctypes.CDLL(pbuild.BENCH_LIB)
    fn = lib.bench_fma_peak
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double(0.0)
    st = fn(int(precision), int(iters), ctypes.c_void_p(stream_ptr), ctypes.byref(out))
    if st != 0:
        raise RuntimeError("bench_fma_peak failed with status %d" % st)
    return out.value

def algorithmic_bytes(n, elem_complex, flagged_lines=0, elem_real=4, nz=None):
    """Bytes each pass must move per step with the 2/3-truncated storage
    (reads + writes of the kept modes only) on the n x n x nz grid, keyed
    by pass name."""
    nz = n if nz is None else nz
    mm = (n - 1) // 3
    K, Kz = 2 * mm + 1, (nz - 1) // 3 + 1
    kk = K * K * Kz
    nk = n * K * Kz
    nn = n * n * Kz
    e = elem_complex
    mask = flagged_lines * nz * 4 * elem_real + n * n  # chi + u_s on flagged lines, flags
    return {
        "x_inverse_curl": (3 * kk + 6 * nk) * e,
        "y_inverse": (6 * nk + 6 * nn) * e,
        "z_c2r_nonlinear_r2c": (6 * nn + 3 * nn) * e + mask,
        "y_forward": (3 * nn + 3 * nk) * e,
        "x_forward_project_ab2": (3 * nk + 3 * kk + 6 * kk) * e,   # reads N, Q; writes U, Q
    }


def adjoint_bytes(n, elem_complex, elem_real):
    """Algorithmic bytes of one reversed step (ps_adjoint_step, FP32 or
    FP64 storage), per kernel family; the checkpoint recompute of the
    forward steps and the rasteriser VJP (band points only) are not counted.
    State arrays are 3 x K^2 Kz (lam, mu, G, Ub, Wb), z-spectral 3 x n^2 Kz,
    physical 3 x n^3."""
    mm = (n - 1) // 3
    K, Kz = 2 * mm + 1, mm + 1
    kk, nk, nn = K * K * Kz, n * K * Kz, n * n * Kz
    e, r_ = elem_complex, elem_real
    n3 = n ** 3
    return {
        "spectral_1": 5 * 3 * kk * e,                                # lam, mu in; G, lam, mu out
        "inverse_u_omega": (3 * kk + 6 * nk) * e + (6 * nk + 6 * nn) * e + 6 * nn * e + 6 * n3 * r_,
        "inverse_G": (3 * kk + 3 * nk) * e + (3 * nk + 3 * nn) * e + 3 * nn * e + 3 * n3 * r_,
        "pointwise": 23 * n3 * r_,                                   # u, w, nbar, chi, u_s in; ubar, wbar, grads out
        "forward_2x3": 2 * (3 * n3 * r_ + 3 * nn * e + (3 * nn + 3 * nk) * e + (3 * nk + 3 * kk) * e),
        "spectral_2": 12 * kk * e,                                   # lam, Ub, Wb in; lam out
    }


def host_info():
    """CPU model, logical cores and RAM of this host (for the CPU baseline)."""
    import platform

    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    ram = None
    try:
        with open("/proc/meminfo") as f:
            ram = round(int(f.readline().split()[1]) / 1024 ** 2, 1)
    except (OSError, ValueError, IndexError):
        pass
    return {"cpu_model": model, "arch": platform.machine(), "nproc": os.cpu_count(), "ram_gib": ram}


def step_flops(n):
    """Model of the arithmetic of one step: 5 m log2(m) real FLOPs per
    complex length-m line transform (the usual FFT count) for every line the
    five passes transform, plus 15 FLOPs per point for u x omega and the
    penalization term. Lines: x-inverse 5 per kept (ky, kz) (three velocity
    components and two kx-derivative transforms), y-inverse 6 per (x, kz),
    z pass 4.5 per (x, y) (three complex inverse, one and a half forward by
    two-for-one packing), y-forward 3 per (x, kz), x-forward 3 per (ky, kz)."""
    mm = (n - 1) // 3
    K, Kz = 2 * mm + 1, mm + 1
    per_line = 5.0 * n * math.log2(n)
    lines = 5 * K * Kz + 6 * n * Kz + 4.5 * n * n + 3 * n * Kz + 3 * K * Kz
    return lines * per_line + 15.0 * n ** 3


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, world):
    """Max of a per-rank float over the process group (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


TRAFFIC_SOURCES = ("ps_kernels.cuh", "ps_fft.cuh", "ps_async.cuh", "ps_engine.cuh")


def sources_sha256():
    import hashlib

    return hashlib.sha256(b"".join(open(os.path.join(ROOT, "paper_2002_08642_gb300", "csrc", f), "rb").read()
                                   for f in TRAFFIC_SOURCES)).hexdigest()


def measured_traffic(kernel, npts):
    """DRAM bytes per launch of pass `kernel` on a grid of npts points,
    scaled from the ncu figure in profiles/traffic.txt (a capture on a
    smaller grid: every z line moves the same bytes per point) by the grid
    points; None if the kernel sources changed since the counters were
    taken, or no figure exists."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                k, v = line.split(None, 1)
                kv[k] = v.strip()
    except OSError:
        return None
    if kv.get("sources_sha256") != sources_sha256() or kernel not in kv:
        return None
    return float(kv[kernel]) * npts / float(kv["measured_points"])


def wing_inputs(cfg, steps):
    """Revolving-wing node positions, velocities and frames of `steps` steps,
    hinge at the box centre."""
    from paper_2002_08642_gb300 import inputs

    L = cfg["L"]
    Lz = L * cfg.get("nz", cfg["n"]) / cfg["n"]
    xw0, tri = inputs.elliptic_wing_mesh(cfg["nodes"])
    amp = inputs.flapping_amplitudes(xw0)
    seq = [inputs.revolving_wing(k * cfg["dt"], xw0, amp, centre=(L / 2, L / 2, Lz / 2)) for k in range(steps)]
    return tri, seq


def timed_leg(cfg, precision, steps, warmup, dev):
    """Rasterise + step of a revolving-wing workload on a fresh context:
    ms per step (CUDA events around `steps` steps after `warmup`), the
    per-pass times, the flagged z lines and the step's algorithmic bytes."""
    import torch

    from paper_2002_08642_gb300.solver import Solver

    n, nz, L = cfg["n"], cfg.get("nz", cfg["n"]), cfg["L"]
    tri, seq = wing_inputs(cfg, warmup + steps)
    g = Solver(n, L, cfg["nu"], cfg["eta"], cfg["dt"], precision=precision, device=dev, nz=nz)
    dt_ = torch.float64 if precision == "fp64" else torch.float32
    g.set_velocity(torch.zeros((3, n, n, nz), dtype=dt_, device=dev))
    tri_d = torch.from_numpy(tri).to(dev, torch.int32)
    xs = [torch.from_numpy(q[0]).to(dev, torch.float64) for q in seq]
    vs = [torch.from_numpy(q[1]).to(dev, torch.float64) for q in seq]
    for k in range(warmup):
        g.set_mask_from_nodes(xs[k], vs[k], tri_d, seq[k][2])
        g.step(1)
    torch.cuda.synchronize()
    flagged = int(g.mask()[0].reshape(n * n, nz).gt(0).any(dim=1).sum().item())
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.timing(True)
    e0.record(stream)
    for k in range(warmup, warmup + steps):
        g.set_mask_from_nodes(xs[k], vs[k], tri_d, seq[k][2])
        g.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    passes = {k: v[0] / max(v[1], 1) for k, v in g.timing_read().items()}
    g.timing(False)
    del g
    torch.cuda.empty_cache()
    ab = algorithmic_bytes(n, 8 if precision == "fp32" else 16, flagged, 4 if precision == "fp32" else 8, nz)
    return ms, passes, flagged, ab


def roofline_of(passes, ab, peak, src, ms_step):
    """Dominant transform pass against the HBM peak, and the whole step."""
    fft = {k: v for k, v in passes.items() if k in ab}
    top = max(fft, key=lambda k: fft[k])
    ach = ab[top] / (fft[top] / 1e3) / 1e9
    sb = sum(ab.values())
    return ({"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
             "peak_source": src, "algorithmic_bytes_per_launch": ab[top]},
            {"algorithmic_bytes_per_step": sb, "achieved_GBs": sb / (ms_step / 1e3) / 1e9,
             "frac": sb / (ms_step / 1e3) / 1e9 / peak,
             "passes": {k: {"ms": fft[k], "GBs": ab[k] / (fft[k] / 1e3) / 1e9,
                            "frac": ab[k] / (fft[k] / 1e3) / 1e9 / peak} for k in fft}})


def cpu_oracle_rate(cfg, budget_s=12.0, n=CPU_SAMPLE_N, min_steps=2):
    """The oracle stepping the same workload recipe at n^3 for about budget_s
    seconds (at least min_steps steps): (Mpts*steps/s, steps, n)."""
    from oracle import mask as OM
    from oracle import step as S
    from paper_2002_08642_gb300 import inputs

    L = cfg["L"]
    dx = L / n
    o = S.Solver(S.Params(n=n, L=L, nu=cfg["nu"], eta=cfg["eta"], dt=cfg["dt"], x0=(L / 2,) * 3))
    o.set_velocity(inputs.random_field(n, L, seed=1234))
    tri, seq = wing_inputs(cfg, 64)
    t0 = time.perf_counter()
    k = 0
    while k < min_steps or (time.perf_counter() - t0 < budget_s and k < len(seq)):
        xw, vw, fr = seq[k]
        chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx)
        o.set_mask(chi, us)
        o.step(1)
        k += 1
    el = time.perf_counter() - t0
    return n ** 3 * k / el / 1e6, k, n


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    for _ in range(args.warmup):
        cpu_oracle_rate(cfg, budget_s=0.0)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, k, n = cpu_oracle_rate(cfg, budget_s=5.0)
        rates.append(r)
    el = time.perf_counter() - t0
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": "Mpts*steps/s", "value": value, "unit": "Mpts*steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_n": CPU_SAMPLE_N},
        "cpu_baseline": {"value": value, "unit": "Mpts*steps/s", "cores": 1, "kind": "oracle",
                         "sample": "FP64 numpy oracle stepping the same revolving-wing recipe at %d^3 "
                                   "(rasterise + step), ~5 s per bench step" % CPU_SAMPLE_N,
                         "host": host_info()},
        "e2e": {"value": value, "unit": "Mpts*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist

    from paper_2002_08642_gb300 import build as pbuild
    from paper_2002_08642_gb300 import inputs
    from paper_2002_08642_gb300.forces import lift_drag
    from paper_2002_08642_gb300.solver import Solver

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pbuild.build()

    n, L = cfg["n"], cfg["L"]
    nz = cfg.get("nz", n)
    total = args.warmup + args.steps
    tri, seq = wing_inputs(cfg, total + args.steps)
    g = Solver(n, L, cfg["nu"], cfg["eta"], cfg["dt"], precision=cfg["precision"], device=dev, nz=nz)
    # the revolving-wing configurations start from rest (u^0 = 0)
    u = torch.zeros((3, n, n, nz), dtype=g.dtype, device=dev)
    g.set_velocity(u)
    del u
    tri_d = torch.from_numpy(tri).to(dev, torch.int32)
    xw_d = [torch.from_numpy(s[0]).to(dev, torch.float64) for s in seq[:total]]
    vw_d = [torch.from_numpy(s[1]).to(dev, torch.float64) for s in seq[:total]]
    frames = [s[2] for s in seq]

    def one(k):
        g.set_mask_from_nodes(xw_d[k], vw_d[k], tri_d, frames[k])
        g.step(1)

    for k in range(args.warmup):
        one(k)
    torch.cuda.synchronize()
    flagged = int(g.mask()[0].reshape(n * n, nz).gt(0).any(dim=1).sum().item())

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-timed region
    clocks = Clocks(local)
    clocks.start()
    g.timing(True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.warmup, total):
        one(k)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    passes = g.timing_read()
    g.timing(False)
    clk = clocks.stop()
    F, M = g.forces()
    ms = max_over_ranks(ms, world)
    npts = n * n * nz
    value = npts * args.steps * world / (ms / 1e3) / 1e6

    # ---- end to end through the public API with host buffers
    xw_h = [torch.from_numpy(s[0]).pin_memory() for s in seq[total:total + args.steps]]
    vw_h = [torch.from_numpy(s[1]).pin_memory() for s in seq[total:total + args.steps]]
    fr_h = frames[total:total + args.steps]
    xw_s = torch.empty_like(xw_d[0])
    vw_s = torch.empty_like(vw_d[0])
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        xw_s.copy_(xw_h[k], non_blocking=True)
        vw_s.copy_(vw_h[k], non_blocking=True)
        g.set_mask_from_nodes(xw_s, vw_s, tri_d, fr_h[k])
        g.step(1)
        g.forces()  # device -> host read of F, M (synchronises)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = npts * args.steps * world / e2e_s / 1e6
    h2d = 2 * xw_h[0].numel() * 8
    d2h = 6 * 8

    # ---- roofline of the dominant pass
    ab = algorithmic_bytes(n, 8 if cfg["precision"] == "fp32" else 16, flagged,
                           4 if cfg["precision"] == "fp32" else 8, nz)
    fft_passes = {k: v for k, v in passes.items() if k in ab}
    top = max(fft_passes, key=lambda k: fft_passes[k][0])
    tms, tl = fft_passes[top]
    peak, src = peaks()
    achieved = ab[top] / (tms / tl / 1e3) / 1e9
    step_bytes = sum(ab.values())
    # five passes + rasteriser (clear with node positions, triangle boxes,
    # prefix sum, pair pass, evaluate; FP64 adds a second pair pass)
    kernels_per_step = 5 + (5 if cfg["precision"] == "fp32" else 6)
    # the z pass against the FP32 FMA rate: its line transforms (4.5 complex
    # length-n transforms per (x, y) line, 5 n log2 n FLOPs each) and the
    # pointwise term; it is bound by instruction issue, not by FMA throughput
    z_ms = passes["z_c2r_nonlinear_r2c"][0] / max(passes["z_c2r_nonlinear_r2c"][1], 1)
    peak32 = fma_peak(0 if cfg["precision"] == "fp32" else 1, 200000, stream.cuda_stream)
    z_fl = 4.5 * n * n * 5.0 * n * math.log2(n) + 15.0 * n ** 3
    z_pass_alu = {"bound": "alu", "achieved": z_fl / (z_ms / 1e3) / 1e12, "peak": peak32 / 1e12,
                  "unit": "TFLOP/s", "frac": z_fl / (z_ms / 1e3) / peak32, "flops_per_launch": z_fl,
                  "peak_source": "measured FMA rate of the path's precision"}
    out = {
        "metric": "Mpts*steps/s", "value": value, "unit": "Mpts*steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if cfg["precision"] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "L": L, "nodes": cfg["nodes"],
                   "precision": cfg["precision"], "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": src, "traffic": measured_traffic(top, npts),
                     "algorithmic_bytes_per_launch": ab[top]},
        "step_roofline": {"algorithmic_bytes_per_step": step_bytes,
                          "achieved_GBs": step_bytes / (ms / args.steps / 1e3) / 1e9,
                          "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
                          "passes": {k: {"ms": fft_passes[k][0] / max(fft_passes[k][1], 1),
                                         "algorithmic_bytes": ab[k],
                                         "GBs": ab[k] / (fft_passes[k][0] / max(fft_passes[k][1], 1) / 1e3) / 1e9,
                                         "frac": ab[k] / (fft_passes[k][0] / max(fft_passes[k][1], 1) / 1e3)
                                                 / 1e9 / peak,
                                         "traffic": measured_traffic(k, npts)} for k in fft_passes}},
        "z_pass_alu": z_pass_alu,
        "passes_ms": {k: v[0] / max(v[1], 1) for k, v in passes.items()},
        "e2e": {"value": e2e, "unit": "Mpts*steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": kernels_per_step * args.steps,
        "forces_last": {"F": F, "M": M, "lift_drag": lift_drag(F, frames[total - 1]["R"])},
    }
    if clk:
        out["clocks"] = clk
    # pressure of the stepped state and its loads on the nodes (the coupling
    # step that follows every fluid step), same workload
    pfield = torch.empty((n, n, nz), dtype=g.dtype, device=dev)
    for _ in range(2):
        g.pressure(pfield)
        g.pressure_loads(pfield, xw_d[0], tri_d, frames[0])
    torch.cuda.synchronize()
    kp_ = max(3, args.steps // 4)
    e0.record(stream)
    for _ in range(kp_):
        g.pressure(pfield)
        g.pressure_loads(pfield, xw_d[0], tri_d, frames[0])
    e1.record(stream)
    torch.cuda.synchronize()
    msp = e0.elapsed_time(e1) / kp_
    out["pressure_loads"] = {"value": npts / (msp / 1e3) / 1e6, "unit": "Mpts/s", "ms_per_call": msp,
                             "calls": kp_, "nodes": int(xw_d[0].shape[0]),
                             "note": "static pressure of the state (passes 1-4, Pi_hat, one inverse field) "
                                     "+ delta interpolation and p A/3 loads on the nodes"}
    del pfield
    cubic = nz == n
    if args.fsi and world == 1 and cubic:
        # staggered FSI step (fluid step, pressure, loads, host mass-spring
        # step, rasterised mask of the new nodes) with an 833-node network
        from paper_2002_08642_gb300.fsi import FSI
        from paper_2002_08642_gb300.massspring import MassSpring

        # a context with keep_uw: the step after each pressure skips passes 1-2
        uf = g.velocity()
        del g
        torch.cuda.empty_cache()
        g = Solver(n, L, cfg["nu"], cfg["eta"], cfg["dt"], precision=cfg["precision"], device=dev, keep_uw=True)
        g.set_velocity(uf)
        del uf
        wf = inputs.fsi_wing(ns=48, nc=16, veins=(0, 4, 8, 12, 16))
        msn = MassSpring(wf["x0"], wf["mass"], wf["ext"], wf["ke"], wf["bend"], wf["kb"], fixed=wf["fixed"])
        cpl = FSI(g, msn, wf["tri"], lambda t: inputs.revolving_frames(t, centre=(L / 2, L / 2, L / 2)),
                  tol=1e-8)
        cpl.step(2)
        torch.cuda.synchronize()
        kf = max(3, args.steps // 4)
        cpl.host_solid_s = 0.0
        it0 = len(cpl.newton_iters)
        t0 = time.perf_counter()
        cpl.step(kf)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / kf
        out["fsi_step"] = {"value": n ** 3 / wall / 1e6, "unit": "Mpts*steps/s", "ms_per_step": wall * 1e3,
                           "steps": kf, "nodes": msn.n, "bandwidth": msn.info()[1], "factorizations": msn.info()[2],
                           "host_solid_ms_per_step": cpl.host_solid_s * 1e3 / kf,
                           "newton_iters": cpl.newton_iters[it0:],
                           "keep_uw": True,
                           "note": "wall clock per coupled step: GPU step (resumed at its z pass) + pressure + "
                                   "loads (D2H) + host mass-spring BDF2/Newton + H2D nodes + GPU rasterise"}
        del cpl, msn
    del g
    torch.cuda.empty_cache()
    if args.fp64 and world == 1 and cubic:
        g64 = Solver(n, L, cfg["nu"], cfg["eta"], cfg["dt"], precision="fp64", device=dev)
        g64.set_velocity(torch.zeros((3, n, n, n), dtype=torch.float64, device=dev))
        k64 = max(2, args.steps // 4)
        for k in range(2):
            g64.set_mask_from_nodes(xw_d[k], vw_d[k], tri_d, frames[k])
            g64.step(1)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(k64):
            g64.set_mask_from_nodes(xw_d[k], vw_d[k], tri_d, frames[k])
            g64.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        v64 = n ** 3 * k64 / (ms64 / 1e3) / 1e6
        peak64 = fma_peak(1, 20000, stream.cuda_stream)
        fl = step_flops(n)
        out["fp64_step"] = {"value": v64, "unit": "Mpts*steps/s", "steps": k64, "ms_per_step": ms64 / k64,
                            "fp32_speedup": value / v64,
                            "alu_roofline": {"bound": "alu", "achieved": fl / (ms64 / k64 / 1e3) / 1e12,
                                             "peak": peak64 / 1e12, "unit": "TFLOP/s",
                                             "frac": fl / (ms64 / k64 / 1e3) / peak64,
                                             "flops_per_step": fl, "peak_source": "measured FP64 FMA rate"}}
        del g64
        torch.cuda.empty_cache()
    if args.small and world == 1 and n != 256:
        # the 256^3 revolving-wing configuration (600 nodes), FP32 and FP64
        # steps, with the per-pass breakdown and the step's HBM roofline
        c2 = WORKLOADS["wing256"]
        ms32, pass32, fl32, ab32 = timed_leg(c2, "fp32", 20, 3, dev)
        ms64_, _, _, _ = timed_leg(c2, "fp64", 8, 3, dev)
        pk, src_ = peaks()
        top2, step2 = roofline_of(pass32, ab32, pk, src_, ms32)
        v32, v64_ = c2["n"] ** 3 / (ms32 / 1e3) / 1e6, c2["n"] ** 3 / (ms64_ / 1e3) / 1e6
        out["wing256_step"] = {"value": v32, "unit": "Mpts*steps/s", "ms_per_step": ms32, "steps": 20,
                               "fp64_value": v64_, "fp64_ms_per_step": ms64_, "fp64_steps": 8,
                               "fp32_speedup": v32 / v64_, "passes_ms": pass32, "roofline": top2,
                               "step_roofline": step2, "flagged_lines": fl32,
                               "note": "256^3 revolving wing, 600 nodes, rasterise + step, inputs resident"}
    if args.aniso and world == 1 and cubic:
        # the paper's 4 x 4 x 2 box at 768 x 768 x 384 (Sec. 4.2 grids), FP32
        ca = WORKLOADS["wing768x384"]
        msa_, passa, fla, aba = timed_leg(ca, "fp32", 10, 3, dev)
        pk, src_ = peaks()
        topa, stepa = roofline_of(passa, aba, pk, src_, msa_)
        na3 = ca["n"] * ca["n"] * ca["nz"]
        out["aniso_step"] = {"value": na3 / (msa_ / 1e3) / 1e6, "unit": "Mpts*steps/s", "ms_per_step": msa_,
                             "steps": 10, "grid": [ca["n"], ca["n"], ca["nz"]], "box": [4.0, 4.0, 2.0],
                             "passes_ms": passa, "roofline": topa, "step_roofline": stepa,
                             "note": "revolving wing, 2000 nodes, rasterise + step, FP32, inputs resident"}
    if args.adjoint and world == 1:
        # adjoint step throughput at 512^3 (FP32): one reversed step per call,
        # on the state and mask reached by a few forward steps
        na = args.adjoint_n
        ga = Solver(na, L, cfg["nu"], cfg["eta"], cfg["dt"], precision="fp32", device=dev, with_adjoint=True)
        ga.set_velocity(torch.zeros((3, na, na, na), dtype=torch.float32, device=dev))
        ga.set_mask_from_nodes(xw_d[0], vw_d[0], tri_d, frames[0])
        ga.step(2)
        gc = torch.empty((na, na, na), dtype=torch.float32, device=dev)
        gs = torch.empty((3, na, na, na), dtype=torch.float32, device=dev)
        gx = torch.zeros_like(xw_d[0])
        ga.adjoint_reset()
        for _ in range(2):
            ga.adjoint_step((0, 0, 1.0), (0, 0, 0), False, gc, gs)
            ga.mask_nodes_vjp(gc, gs, gx)
        ka = max(3, args.steps // 4)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ka):
            ga.adjoint_step((0, 0, 1.0), (0, 0, 0), False, gc, gs)
            ga.mask_nodes_vjp(gc, gs, gx)
        e1.record(stream)
        torch.cuda.synchronize()
        msa = e0.elapsed_time(e1)
        adj_b = adjoint_bytes(na, 8, 4)
        pk, src_ = peaks()
        adj_tot = sum(adj_b.values())
        out["adjoint_step"] = {"value": na ** 3 * ka / (msa / 1e3) / 1e6, "unit": "Mpts*steps/s", "n": na,
                               "precision": "fp32", "steps": ka, "ms_per_step": msa / ka,
                               "roofline": {"bound": "hbm", "algorithmic_bytes_per_step": adj_tot,
                                            "bytes_by_kernel_family": adj_b,
                                            "achieved": adj_tot / (msa / ka / 1e3) / 1e9, "peak": pk,
                                            "unit": "GB/s", "frac": adj_tot / (msa / ka / 1e3) / 1e9 / pk,
                                            "peak_source": src_},
                               "note": "reversed step + rasteriser VJP, excluding the checkpoint recompute "
                                       "(the byte model leaves out the VJP, which touches the band points only)"}
        del ga
        torch.cuda.empty_cache()
    if rank == 0 and args.cpu_baseline:
        r, k, cn = cpu_oracle_rate(cfg)
        # the configurations' own small sizes: median of three runs each
        by_n = {}
        for nn_, steps_ in ((32, 4), (128, 1)):
            rr = [cpu_oracle_rate(cfg, budget_s=0.0, n=nn_, min_steps=steps_)[0] for _ in range(3)]
            by_n[str(nn_)] = {"value": statistics.median(rr), "runs": rr, "steps_per_run": steps_}
        out["cpu_baseline"] = {"value": r, "unit": "Mpts*steps/s", "cores": 1, "kind": "oracle",
                               "sample": "FP64 numpy oracle, same revolving-wing recipe at %d^3, "
                                         "%d steps (rasterise + step), single-threaded numpy" % (cn, k),
                               "by_n": by_n, "host": host_info()}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="wing768", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false")
    ap.add_argument("--no-256", dest="small", action="store_false")
    ap.add_argument("--no-fsi", dest="fsi", action="store_false")
    ap.add_argument("--no-aniso", dest="aniso", action="store_false")
    ap.add_argument("--adjoint-n", type=int, default=512, help="grid of the adjoint-step leg")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
