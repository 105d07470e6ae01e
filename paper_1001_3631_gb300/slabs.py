"""r* slab decomposition of one grid over ranks (the data-parallel split of the (r*, theta)
grid, Sec. 3): partition of the interior columns, the halo exchange between neighbouring
ranks, and a driver that steps a slab instance of the library one step at a time.

Each rank owns a run of interior r* columns and holds one more column on each side (a
halo, or the grid's own end column).  The stencil of one Lax-Wendroff step (Eqs. 13-14)
reaches one column in r*, so after every step a rank sends its first owned column to the
left neighbour and its last to the right neighbour and receives their columns into its
halos; the grid's end columns stay zero (the radial boundary condition).  The exchange is
the only collective of the step; it moves 2 x n_theta x 32 bytes per rank and step
(FP64 state), point to point."""
from __future__ import annotations


def partition(n_rstar, n_slabs):
    """(col0, ncols) of each slab: the interior columns 1 .. n_rstar-2 in n_slabs runs
    whose lengths differ by at most one."""
    cols = n_rstar - 2
    if n_slabs < 1 or cols < 2 * n_slabs:
        raise ValueError("need at least two interior columns per slab")
    base, extra = divmod(cols, n_slabs)
    out, c0 = [], 1
    for k in range(n_slabs):
        n = base + (1 if k < extra else 0)
        out.append((c0, n))
        c0 += n
    return out


def exchange(send_left, send_right, recv_left, recv_right, rank, world):
    """Point-to-point halo exchange over torch.distributed: send_left (this rank's first
    owned column) to rank - 1 and send_right (its last) to rank + 1; receive recv_left
    from rank - 1 and recv_right from rank + 1.  Tensors live where the process group's
    backend wants them (host for gloo, device for NCCL)."""
    import torch.distributed as dist
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(send_left, rank - 1))
        reqs.append(dist.irecv(recv_left, rank - 1))
    if rank < world - 1:
        reqs.append(dist.isend(send_right, rank + 1))
        reqs.append(dist.irecv(recv_right, rank + 1))
    for r in reqs:
        r.wait()


class SlabStepper:
    """One slab of a grid on this rank: a library context whose instance is the slab
    (teuk_params.slab_col0 / slab_ncols), stepped one step at a time with the halo
    exchange between steps.  host_exchange: move the halo columns through host memory
    (a gloo process group); otherwise device tensors go to the process group directly."""

    def __init__(self, params, rank, world, host_exchange=False, stream=None):
        import torch

        from .solver import TeukSolver
        self.rank, self.world = rank, world
        self.col0, self.ncols = partition(params["n_rstar"], world)[rank]
        self.solver = TeukSolver(dict(params, slab_col0=self.col0, slab_ncols=self.ncols), stream=stream)
        nb = self.solver.halo_bytes()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dbuf = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(4)]   # sendL, sendR, recvL, recvR
        self.host = host_exchange
        if host_exchange:
            self.hbuf = [torch.empty(nb, dtype=torch.uint8) for _ in range(4)]

    def step(self, n):
        import torch
        s = self.solver
        for _ in range(n):
            s.step(1)
            if self.world == 1:
                continue
            if self.rank > 0:
                s.slab_export(0, self.dbuf[0].data_ptr())
            if self.rank < self.world - 1:
                s.slab_export(1, self.dbuf[1].data_ptr())
            torch.cuda.current_stream().synchronize()
            if self.host:
                for k in (0, 1):
                    self.hbuf[k].copy_(self.dbuf[k])
                exchange(*self.hbuf, self.rank, self.world)
                for k in (2, 3):
                    self.dbuf[k].copy_(self.hbuf[k])
            else:
                exchange(*self.dbuf, self.rank, self.world)
            if self.rank > 0:
                s.slab_import(0, self.dbuf[2].data_ptr())
            if self.rank < self.world - 1:
                s.slab_import(1, self.dbuf[3].data_ptr())

    def owned(self, u):
        """The owned columns of a slab state [4][n_theta][ncols + 2]."""
        return u[:, :, 1:1 + self.ncols]
