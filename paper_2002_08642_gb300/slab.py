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


class SlabContexts:
    """P slabs of the sharded step as P contexts on one GPU (each with its
    own workspace): every pass of the step runs as the slabs' share of it
    (ps_slab_phase), the two exchanges are device-to-device block copies
    between the slabs' x-pass arrays A in the layout of ``SlabPlan``, and the
    force is the host sum of the slabs' partial forces. It exercises the
    per-slab GPU passes and the exchange pattern of the multi-GPU step
    without a second GPU.

    ``solvers``: P ``Solver`` objects of the same grid and parameters, in
    slab order; ``x_off``, ``ky_off``: P + 1 start offsets of the x-plane and
    kept-ky-row partitions (``balanced``)."""

    def __init__(self, solvers, x_off, ky_off):
        from . import binding as B

        self.B = B
        self.s = list(solvers)
        self.P = len(self.s)
        self.xo, self.ko = list(x_off), list(ky_off)
        self.A = []
        for r, g in enumerate(self.s):
            B.ps_slab_set(g.ctx, self.xo[r], self.xo[r + 1], self.ko[r], self.ko[r + 1])
            K, _, Kzp = B.ps_grid_info(g.ctx)
            ptr, nbytes = B.ps_slab_buffer(g.ctx)
            off = ptr - g.workspace.data_ptr()
            cdt = torch.complex128 if g.dtype == torch.float64 else torch.complex64
            self.A.append(g.workspace[off:off + nbytes].view(cdt).view(6, K, g.n, Kzp))
        self.K = K

    def _phase(self, ph):
        for g in self.s:
            self.B.ps_slab_phase(g.ctx, ph)

    def ky_to_x(self):
        """After the x-inverse: slab r gets rows ky in slab s's range at its
        own x-planes from slab s (six fields)."""
        for r in range(self.P):
            x0, x1 = self.xo[r], self.xo[r + 1]
            for s in range(self.P):
                if s != r:
                    k0, k1 = self.ko[s], self.ko[s + 1]
                    self.A[r][:, k0:k1, x0:x1].copy_(self.A[s][:, k0:k1, x0:x1])

    def x_to_ky(self):
        """After the y-forward: slab r gets its ky rows at slab s's x-planes
        from slab s (three fields)."""
        for r in range(self.P):
            k0, k1 = self.ko[r], self.ko[r + 1]
            for s in range(self.P):
                if s != r:
                    x0, x1 = self.xo[s], self.xo[s + 1]
                    self.A[r][:3, k0:k1, x0:x1].copy_(self.A[s][:3, k0:k1, x0:x1])

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self._phase(0)
            self.ky_to_x()
            self._phase(1)
            self.x_to_ky()
            self._phase(2)

    def forces(self):
        """F and M of the last step: the sum of the slabs' shares (host, double)."""
        F = [0.0, 0.0, 0.0]
        M = [0.0, 0.0, 0.0]
        for g in self.s:
            f, m = g.forces()
            F = [a + b for a, b in zip(F, f)]
            M = [a + b for a, b in zip(M, m)]
        return F, M

    def state(self):
        """The global spectral state (U, H) assembled from the slabs' ky rows,
        as a state buffer of the first slab's size (ps_save_state layout)."""
        K, n = self.K, self.s[0].n
        bufs = []
        for g in self.s:
            b = g.state_buffer()
            g.save_state(b)
            bufs.append(b)
        out = bufs[0].clone()
        cdt = torch.complex128 if self.s[0].dtype == torch.float64 else torch.complex64
        es = torch.finfo(self.s[0].dtype).bits // 4   # bytes per complex
        nb = (out.numel() - 256) // 2                   # bytes of U (and of H)
        Kzp = nb // (3 * K * K * es)

        def view(b, which):
            o = 256 + which * nb
            return b[o:o + nb].view(cdt).view(3, K, K, Kzp)

        for r in range(1, self.P):
            k0, k1 = self.ko[r], self.ko[r + 1]
            for which in (0, 1):
                view(out, which)[:, k0:k1].copy_(view(bufs[r], which)[:, k0:k1])
        return out
