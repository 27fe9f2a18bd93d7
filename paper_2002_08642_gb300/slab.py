"""Slab decomposition of the pseudo-spectral step over P ranks (the MPI
slabs of the paper's solver, Sec. 4.1, mapped to one process per GPU).

Rank r holds the x-planes [x0_r, x1_r) for the y and z passes, the
pointwise term and the rasteriser, and the kept ky rows [k0_r, k1_r) for
the x passes (x-inverse with the curl, x-forward with the projection and
the update). Two exchanges per step move the spectral data between the two
partitions, both all-to-alls of [field][ky block][x block][kz] tiles in the
layout of the x-pass array A ([field][ky][x][kz]):

* ``ky_to_x`` after the x-inverse (six fields): rank r sends to rank d its
  ky rows [k0_r, k1_r) for d's x-planes;
* ``x_to_ky`` after the y-forward (three fields): rank r sends to rank d its
  x-planes [x0_r, x1_r) for d's ky rows.

Both use one ``all_to_all_single`` on a packed buffer (NCCL between GPUs,
gloo between CPU processes); splits are balanced (sizes differ by at most
one). Forces and moments are summed with one all-reduce of 6 doubles.
"""
import torch
import torch.distributed as dist


def balanced(total, parts):
    """Start offsets (parts + 1) of a balanced split of range(total)."""
    q, r = divmod(total, parts)
    off = [0]
    for i in range(parts):
        off.append(off[-1] + q + (1 if i < r else 0))
    return off


class SlabPlan:
    """Partition of n x-planes and K kept ky rows over the ranks of ``group``."""

    def __init__(self, n, K, group=None):
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.n, self.K = n, K
        self.xo = balanced(n, self.world)
        self.ko = balanced(K, self.world)

    def x_range(self, r=None):
        r = self.rank if r is None else r
        return self.xo[r], self.xo[r + 1]

    def ky_range(self, r=None):
        r = self.rank if r is None else r
        return self.ko[r], self.ko[r + 1]

    @staticmethod
    def _flat(t):
        return torch.view_as_real(t).reshape(-1) if t.is_complex() else t.reshape(-1)

    def _exchange(self, send_blocks, recv_shapes, like):
        send = torch.cat([self._flat(b.contiguous()) for b in send_blocks])
        per = 2 if like.is_complex() else 1
        in_splits = [b.numel() * per for b in send_blocks]
        out_splits = []
        for s in recv_shapes:
            c = per
            for d in s:
                c *= d
            out_splits.append(c)
        real = torch.float64 if like.dtype in (torch.complex128, torch.float64) else torch.float32
        recv = torch.empty(sum(out_splits), dtype=real, device=like.device)
        dist.all_to_all_single(recv, send, out_splits, in_splits, group=self.group)
        out, o = [], 0
        for s, c in zip(recv_shapes, out_splits):
            piece = recv[o:o + c]
            o += c
            if like.is_complex():
                piece = torch.view_as_complex(piece.reshape(*s, 2))
            else:
                piece = piece.reshape(*s)
            out.append(piece)
        return out

    def x_to_ky(self, a):
        """a: this rank's x-slab [F][K][x1 - x0][C] -> its ky-slab [F][k1 - k0][n][C]."""
        F, K, xs, C = a.shape
        assert K == self.K and xs == self.x_range()[1] - self.x_range()[0]
        k0, k1 = self.ky_range()
        send = [a[:, self.ko[d]:self.ko[d + 1]] for d in range(self.world)]
        shapes = [(F, k1 - k0, self.xo[s + 1] - self.xo[s], C) for s in range(self.world)]
        return torch.cat(self._exchange(send, shapes, a), dim=2)

    def ky_to_x(self, b):
        """b: this rank's ky-slab [F][k1 - k0][n][C] -> its x-slab [F][K][x1 - x0][C]."""
        F, ks, n, C = b.shape
        assert n == self.n and ks == self.ky_range()[1] - self.ky_range()[0]
        x0, x1 = self.x_range()
        send = [b[:, :, self.xo[d]:self.xo[d + 1]] for d in range(self.world)]
        shapes = [(F, self.ko[s + 1] - self.ko[s], x1 - x0, C) for s in range(self.world)]
        return torch.cat(self._exchange(send, shapes, b), dim=1)

    def sum_forces(self, FM):
        """All-reduce of the 6 force/moment partial sums (a float64 tensor)."""
        dist.all_reduce(FM, group=self.group)
        return FM
