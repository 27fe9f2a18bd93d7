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


def test_traffic_figure_tracks_kernel_sources(monkeypatch):
    got = bench.measured_traffic("z_c2r_nonlinear_r2c", 768)
    assert got is None or got > 1e10
    assert bench.measured_traffic("no_such_kernel", 768) is None


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
