"""The sharded step's decomposition (paper_2002_08642_gb300/slab.py) on
gloo CPU ranks: two IF-AB2 steps with a mask, each rank doing the x passes
(curl, projection, update) on its ky rows and the y/z passes and the
pointwise term on its x-planes, joined by the plan's two exchanges and the
force all-reduce, reproduce the oracle's global step. The per-slab
arithmetic here is the oracle's (test code); the exchanges are the
product's."""
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
from oracle import step as S
from paper_2002_08642_gb300.slab import SlabPlan


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(n):
    rng = np.random.default_rng(5)
    p = S.Params(n=n, L=2 * np.pi, nu=0.02, eta=0.5, dt=0.01, x0=(1.0, 2.0, 3.0))
    X, Y, Z = S.grid_coords(p)
    shape = (n, n, n)
    u = np.stack([np.broadcast_to(c, shape) for c in
                  (np.sin(Y + 0.3) + 0.2 * np.cos(2 * Z), np.sin(Z) * np.cos(X), np.cos(X + Y))])
    chi = np.zeros((n, n, n))
    chi[2:6, 3:7, 1:5] = 1.0
    chi[6, 3:7, 1:5] = 0.5
    us = np.zeros((3, n, n, n))
    us[0] = 0.3 * chi
    us[2] = -0.1 * chi
    return p, u, chi, us


def _rank_step(plan, p, uh, nprev, nstep, chi_s, us_s, my, kz_keep):
    """One step on this rank: uh, nprev are ky-slabs [3][kx][ky_loc][kz]."""
    n = p.n
    k0, k1 = plan.ky_range()
    x0, x1 = plan.x_range()
    ks = 2 * np.pi / p.L
    kx = (ks * S.mode_numbers(n))[:, None, None]
    ky = (ks * S.mode_numbers(n)[my[k0:k1]])[None, :, None]
    kz = (ks * np.arange(n // 2 + 1))[None, None, :]
    keep = S.dealias_mask(n)[:, my[k0:k1], :]
    ux, uy, uz = uh
    wh = np.stack([1j * (ky * uz - kz * uy), 1j * (kz * ux - kx * uz), 1j * (kx * uy - ky * ux)]) * keep
    six = np.concatenate([uh, wh])                                   # [6][kx][kyl][kz]
    a = offt.ifft(six, axis=1)                                       # x-inverse -> [6][x][kyl][kz]
    a = torch.from_numpy(np.ascontiguousarray(np.transpose(a, (0, 2, 1, 3))))   # [6][kyl][x][kz]
    b = plan.ky_to_x(a).numpy()                                      # [6][K][xl][kz]
    full = np.zeros((6, n, x1 - x0, n // 2 + 1), dtype=np.complex128)
    full[:, my] = b
    yinv = offt.ifft(full, axis=1)                                   # [6][y][xl][kz]
    yinv = np.transpose(yinv, (0, 2, 1, 3))                          # [6][xl][y][kz]
    phys = np.fft.irfft(yinv, n=n, axis=3)                           # [6][xl][y][z]
    u, w = phys[:3], phys[3:]
    # pointwise term and force partials on the x-slab
    nl = S.nonlinear_physical(u, w, chi_s, us_s, p.eta)
    pen = chi_s[None] * (u - us_s)
    dx = p.L / n
    X = (np.arange(x0, x1) * dx)[:, None, None]
    Y = (np.arange(n) * dx)[None, :, None]
    Zc = (np.arange(n) * dx)[None, None, :]
    r = [np.broadcast_to(c - o, pen.shape[1:]) for c, o in zip((X, Y, Zc), p.x0)]
    mom = [r[1] * pen[2] - r[2] * pen[1], r[2] * pen[0] - r[0] * pen[2], r[0] * pen[1] - r[1] * pen[0]]
    FM = torch.tensor([pen[c].sum() for c in range(3)] + [mom[c].sum() for c in range(3)], dtype=torch.float64)
    FM = plan.sum_forces(FM) * dx ** 3 / p.eta
    # forward: z, y on the x-slab, exchange, x on the ky-slab
    zf = np.fft.rfft(nl, axis=3)                                     # [3][xl][y][kz]
    yf = offt.fft(zf, axis=2)[:, :, my]                              # [3][xl][K][kz]
    a2 = torch.from_numpy(np.ascontiguousarray(np.transpose(yf, (0, 2, 1, 3))))   # [3][K][xl][kz]
    b2 = plan.x_to_ky(a2).numpy()                                    # [3][kyl][x][kz]
    Nh = np.transpose(offt.fft(b2, axis=2), (0, 2, 1, 3)) * keep     # [3][kx][kyl][kz]
    k2 = kx * kx + ky * ky + kz * kz
    k2s = np.where(k2 == 0.0, 1.0, k2)
    kd = kx * Nh[0] + ky * Nh[1] + kz * Nh[2]
    PN = np.stack([Nh[0] - kx * kd / k2s, Nh[1] - ky * kd / k2s, Nh[2] - kz * kd / k2s])
    if k0 == 0:                                                      # the k = 0 mode (ky = 0 is row 0)
        PN[:, 0, 0, 0] = 0.0
    E = np.exp(-p.nu * k2 * p.dt)
    if nstep == 0:
        new = E * (uh + p.dt * PN)
    else:
        new = E * uh + 0.5 * p.dt * (3.0 * E * PN - E * E * nprev)
    return new, PN, FM.numpy()


def _worker(rank, world, port, n, q):
    try:
        _work(rank, world, port, n, q)
    except Exception:
        q.put((rank, float("inf"), traceback.format_exc()))


def _work(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        p, u, chi, us = _case(n)
        mm = (n - 1) // 3
        my = np.r_[0:mm + 1, n - mm:n]
        plan = SlabPlan(n, 2 * mm + 1, None)
        o = S.Solver(p)
        o.set_velocity(u)
        o.set_mask(chi, us)
        k0, k1 = plan.ky_range()
        x0, x1 = plan.x_range()
        uh = o.uh[:, :, my[k0:k1]].copy()
        nprev = np.zeros_like(uh)
        errs, ferrs = [], []
        for step in range(2):
            uh, nprev, FM = _rank_step(plan, p, uh, nprev, step, chi[x0:x1], us[:, x0:x1], my, None)
            o.step(1)
            errs.append(np.max(np.abs(uh - o.uh[:, :, my[k0:k1]])) / np.max(np.abs(o.uh)))
            ferrs.append(np.max(np.abs(FM - np.r_[o.F, o.M])) / np.max(np.abs(np.r_[o.F, o.M])))
        q.put((rank, max(errs), max(ferrs)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_step_matches_global_oracle_step(world):
    n = 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    try:
        res = [q.get(timeout=180) for _ in range(world)]
    finally:
        for pr in procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.kill()
    for r, e, ef in res:
        assert e < 1e-13 and ef < 1e-12, (r, e, ef)
