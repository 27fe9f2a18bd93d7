"""Host-side pieces of bench.py: the byte model, the traffic figure's source
check and the max-over-ranks timing reduction (two gloo ranks on CPU)."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_algorithmic_bytes_model():
    ab = bench.algorithmic_bytes(768, 8)
    total = sum(ab.values())
    # kept modes only: K = 511 x/y modes, Kz = 256 z modes; per step the five
    # passes move 12 K^2 Kz + 18 n K Kz + 18 n^2 Kz complex values (the AB2
    # update reads one history array) plus the n^2 line flags
    K, Kz, n = 511, 256, 768
    assert total == (12 * K * K * Kz + 18 * n * K * Kz + 18 * n * n * Kz) * 8 + n * n
    # ~94 bytes per grid point per step
    assert 93 < total / 768 ** 3 < 96
    assert max(ab, key=ab.get) == "y_inverse"


def test_step_flop_model():
    """5 m log2 m FLOPs per complex line transform: at 64^3 (K = 43, Kz = 22)
    the passes transform 5*43*22 + 6*64*22 + 4.5*64^2 + 3*64*22 + 3*43*22
    lines of length 64 (5*64*6 = 1920 FLOPs each), plus 15 FLOPs per point."""
    lines = 5 * 43 * 22 + 6 * 64 * 22 + 4.5 * 64 * 64 + 3 * 64 * 22 + 3 * 43 * 22
    assert bench.step_flops(64) == pytest.approx(lines * 1920 + 15 * 64 ** 3, rel=1e-12)
    # about 460 FLOPs per point at 768^3: FP64 at ~1 TFLOP/s is far from HBM-bound
    assert 440 < bench.step_flops(768) / 768 ** 3 < 480


def test_traffic_figure_tracks_kernel_sources(monkeypatch):
    # the figure is scaled by grid points: ~10.5 GB per 768^3 z pass
    npts = 768 ** 3
    got = bench.measured_traffic("z_c2r_nonlinear_r2c", npts)
    assert got is None or 1e10 < got < 1.2e10
    assert bench.measured_traffic("no_such_kernel", npts) is None
    # a figure taken on other kernel sources is not used
    monkeypatch.setattr(bench, "sources_sha256", lambda: "0" * 64)
    assert bench.measured_traffic("z_c2r_nonlinear_r2c", npts) is None


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(10.0 + rank, world)
    out[rank] = v
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    port = 29500 + os.getpid() % 1000
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == 11.0 and out[1] == 11.0


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on a bounded sample)
    runs without a GPU and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_adjoint_bytes_model():
    """The reversed step's byte model, kernel by kernel: each kernel reads and
    writes whole arrays of four kinds (spectral state K^2 Kz, x-physical
    n K Kz, z-spectral n^2 Kz complex; physical n^3 real). At 512^3 the
    families are the totals of the per-kernel launch list (one reversed step:
    two z c2r for u and omega, one for nbar, two forward passes)."""
    n = 512
    K, Kz = 341, 171
    spec, xphys, zspec, phys = K * K * Kz * 8, n * K * Kz * 8, n * n * Kz * 8, n ** 3 * 4
    xinv = lambda f_in, f_out: f_in * spec + f_out * xphys
    yinv = lambda f: f * xphys + f * zspec
    zc2r = 3 * zspec + 3 * phys
    fwd = 3 * phys + 3 * zspec + (3 * zspec + 3 * xphys) + (3 * xphys + 3 * spec)
    ab = bench.adjoint_bytes(n, 8, 4)
    assert ab["spectral_1"] == 15 * spec                       # lam, mu in; G, lam, mu out
    assert ab["inverse_u_omega"] == xinv(3, 6) + yinv(6) + 2 * zc2r
    assert ab["inverse_G"] == xinv(3, 3) + yinv(3) + zc2r
    assert ab["pointwise"] == 23 * phys                        # 13 physical fields in, 10 out
    assert ab["forward_2x3"] == 2 * fwd
    assert ab["spectral_2"] == 12 * spec                       # lam, Ub, Wb in; lam out
    # the figures of the 512^3 launch list, in GB
    got = {k: round(v / 1e9, 2) for k, v in ab.items()}
    assert got == {"spectral_1": 2.39, "inverse_u_omega": 10.87, "inverse_G": 5.67, "pointwise": 12.35,
                   "forward_2x3": 11.35, "spectral_2": 1.91}
