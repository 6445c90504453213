"""z-slab solves over several GPUs (the paper's P-TDMA, Sec. 2.2.3): one rank
per GPU holds whole x-y planes of a field; a solve is the library's reduce
call, one all-gather of the boundary buffers, and the finish call.

Every arithmetic step runs in the library's CUDA kernels
(cfs_slab_poisson_reduce / _finish, cfs_slab_helmholtz_reduce / _finish);
this module only moves the boundary buffers between ranks (2 values per
column per rank: the only data the decomposition exchanges) with
torch.distributed -- NCCL between GPUs.  With a single rank (no process
group) the exchange is the buffer itself.
"""

from __future__ import annotations

from . import chanfs


def gather_boundaries(bnd, group=None):
    """All ranks' boundary buffers concatenated rank-major (rank r's buffer at
    offset r * bnd.numel()): the layout the finish calls read."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return bnd
    world = dist.get_world_size(group)
    if world == 1:
        return bnd
    parts = [torch.empty_like(bnd) for _ in range(world)]
    dist.all_gather(parts, bnd.contiguous(), group=group)
    return torch.cat(parts)


class SlabSolver:
    """This rank's slab of an nx x ny x nz grid split along z over the ranks of
    `group` (all of torch.distributed's default group if None); fields are
    the rank's planes, shape (z1 - z0, ny, nx), float64 on its GPU."""

    def __init__(self, nx, ny, nz, lx, ly, dz, bc=chanfs.NEUMANN, group=None, nranks=None,
                 rank=None):
        import torch.distributed as dist
        if nranks is None or rank is None:
            if dist.is_available() and dist.is_initialized():
                nranks, rank = dist.get_world_size(group), dist.get_rank(group)
            else:
                nranks, rank = 1, 0
        self.group = group
        self.slab = chanfs.Slab(nx, ny, nz, lx, ly, dz, bc, nranks, rank)
        self.shape = self.slab.shape
        self.z0, self.z1 = self.slab.z0, self.slab.z1

    def close(self):
        self.slab.close()

    def _buffers(self, kind, like):
        import torch
        n = self.slab.boundary_doubles(kind)
        return torch.empty(n, dtype=like.dtype, device=like.device)

    def poisson_solve(self, f, out=None, work=None):
        import torch
        out = torch.empty_like(f) if out is None else out
        work = out if work is None else work
        bnd = self._buffers(chanfs.REQ_POISSON, f)
        self.slab.poisson_reduce(f, work, bnd)
        bnd_all = gather_boundaries(bnd, self.group)
        self.slab.poisson_finish(bnd_all, work, out)
        return out

    def helmholtz_solve(self, c, rhs, loc=chanfs.CENTER, out=None, work=None):
        import torch
        out = torch.empty_like(rhs) if out is None else out
        work = torch.empty_like(rhs) if work is None else work
        bnd = self._buffers(chanfs.REQ_HELMHOLTZ, rhs)
        self.slab.helmholtz_reduce(c, loc, rhs, work, bnd)
        bnd_all = gather_boundaries(bnd, self.group)
        self.slab.helmholtz_finish(c, loc, bnd_all, work, out)
        return out
