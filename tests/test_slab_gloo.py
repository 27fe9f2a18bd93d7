"""Slab decomposition of the step (paper_2002_08642_gb300/slab.py) on CPU
processes with gloo: the two exchanges against the global arrays, and a
distributed 3-D forward transform (z and y on x-slabs, exchange, x on
ky-slabs) against the oracle's transform with the 2/3 truncation."""
import datetime
import os
import socket
import traceback

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import fft as offt
from paper_2002_08642_gb300.slab import SlabPlan, balanced


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    try:
        _work(rank, world, port, n, q)
    except Exception:
        q.put((rank, False, False, False, traceback.format_exc()))


def _work(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        mm = (n - 1) // 3
        K, Kz = 2 * mm + 1, mm + 1
        plan = SlabPlan(n, K, None)
        rng = np.random.default_rng(11)
        # 1) exchanges against the global array
        G = rng.normal(size=(3, K, n, 5)) + 1j * rng.normal(size=(3, K, n, 5))
        x0, x1 = plan.x_range()
        k0, k1 = plan.ky_range()
        a = torch.from_numpy(G[:, :, x0:x1].copy())
        b = plan.x_to_ky(a)
        ok1 = np.array_equal(b.numpy(), G[:, k0:k1])
        back = plan.ky_to_x(b)
        ok2 = np.array_equal(back.numpy(), G[:, :, x0:x1])
        # 2) distributed forward transform of a real field (one component)
        u = rng.normal(size=(n, n, n))
        loc = u[x0:x1]                                   # x-slab [x][y][z]
        zt = np.fft.rfft(loc, axis=2)[:, :, :Kz]         # z r2c, kz < Kz
        yt = np.fft.fft(zt, axis=1)                      # y
        my = np.r_[0:mm + 1, n - mm:n]                   # kept ky, FFT order
        yt = yt[:, my]                                   # [x][ky][kz]
        A = torch.from_numpy(np.ascontiguousarray(np.transpose(yt, (1, 0, 2))[None]))   # [1][K][x][kz]
        B = plan.x_to_ky(A)                              # [1][ky][x = all][kz]
        xt = np.fft.fft(B.numpy()[0], axis=1)[:, my]     # x, kept kx -> [ky][kx][kz]
        want = offt.rfft3(u)[np.ix_(my, my, np.arange(Kz))]   # [kx][ky][kz]
        ok3 = np.allclose(np.transpose(xt, (1, 0, 2)), want[:, k0:k1], atol=1e-9)
        FM = torch.full((6,), float(rank + 1), dtype=torch.float64)
        ok4 = float(plan.sum_forces(FM)[0]) == world * (world + 1) / 2
        q.put((rank, ok1, ok2, ok3, ok4))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 12), (3, 16)])
def test_slab_exchanges_and_distributed_transform(world, n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=120) for _ in range(world)]
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for r, ok1, ok2, ok3, ok4 in res:
        assert ok1 and ok2 and ok3 and ok4, (r, ok1, ok2, ok3, ok4)


def test_balanced_split():
    assert balanced(10, 3) == [0, 4, 7, 10]
    assert balanced(511, 8)[-1] == 511 and max(np.diff(balanced(511, 8))) - min(np.diff(balanced(511, 8))) <= 1
