"""How one cell's path shards over several GPUs (one rank per GPU), as the
paper distributes it over MPI ranks (Sec. 4, last paragraphs: the density
kernel's columns are distributed, and communication is limited to the
Fermi-level search; Sec. 5 runs on CPU clusters).  This module holds the
partitioning and the exchange steps, written against torch.distributed so
that the same code runs on NCCL ranks (one GPU each) or on gloo ranks
(the CPU tests):

* grid slabs: rank r owns whole z-planes [z0, z1) of the grid, so the
  Gram matrix X^T X and the projection X^T (H X) are sums of per-slab
  products, all-reduced (Ns^2 words); the stencil needs R planes of each
  neighbouring slab per filter step (halo_planes);
* column blocks: rank r owns columns [j0, j1) of the T_j of the
  Chebyshev recurrence (Hhat replicated): T_{j+1}[:, cols] =
  2 Hhat T_j[:, cols] - T_{j-1}[:, cols] needs no exchange, and the
  moments m_j = tr T_j are all-reduced (npl + 1 words), the only
  communication of the Fermi-level search;
* the density kernel's column blocks are all-gathered before the slab-local
  density rho = 2 rowdot(X, X Ds) / dV.

On one GPU the path runs unsharded; this module is the partitioning,
exercised by two and three gloo ranks on the CPU (tests/test_sharding_gloo.py).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _split(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [a, b) of n items for `rank`: the first n % world
    ranks take one item more."""
    q, r = divmod(n, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def grid_slab(nz: int, world: int, rank: int) -> tuple[int, int]:
    """z-planes [z0, z1) of this rank's slab."""
    if nz < world:
        raise ValueError("fewer planes than ranks")
    return _split(nz, world, rank)


def column_block(Ns: int, world: int, rank: int) -> tuple[int, int]:
    """Columns [j0, j1) of the density-kernel matrices on this rank."""
    return _split(Ns, world, rank)


def allreduce_sum(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks (the Gram / projection matrix, the moments)."""
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def gram_slabs(X_local: torch.Tensor, Y_local: torch.Tensor) -> torch.Tensor:
    """X^T Y summed over the slabs: the local block product, all-reduced.
    X_local, Y_local: (Ns, n_local) rows of this rank's grid points (the
    library's column-major N x Ns block restricted to the slab)."""
    return allreduce_sum(X_local @ Y_local.T)


def moments_columns(T_cols: list[torch.Tensor], j0: int) -> torch.Tensor:
    """m_j = tr T_j from this rank's columns [j0, j0 + w) of every T_j
    (T_cols[j] is Ns x w), all-reduced."""
    m = torch.stack([torch.diagonal(Tj[j0:j0 + Tj.shape[1], :]).sum() for Tj in T_cols])
    return allreduce_sum(m)


def gather_columns(D_cols: torch.Tensor, Ns: int) -> torch.Tensor:
    """The full Ns x Ns matrix from every rank's column block (all-gather)."""
    world = dist.get_world_size() if dist.is_initialized() else 1
    if world == 1:
        return D_cols
    parts = [torch.empty((Ns, b - a), dtype=D_cols.dtype, device=D_cols.device)
             for a, b in (column_block(Ns, world, r) for r in range(world))]
    dist.all_gather(parts, D_cols.contiguous())
    return torch.cat(parts, dim=1)


def halo_planes(slab: torch.Tensor, R: int) -> tuple[torch.Tensor, torch.Tensor]:
    """The R planes below and above this rank's slab, from the neighbouring
    ranks (periodic in z): slab is (..., planes, ny, nx); returns
    (below, above), each (..., R, ny, nx).  Each rank sends its first R
    planes down and its last R planes up."""
    world = dist.get_world_size() if dist.is_initialized() else 1
    if slab.shape[-3] < R:
        raise ValueError("slab thinner than the stencil radius")
    first = slab[..., :R, :, :].contiguous()
    last = slab[..., -R:, :, :].contiguous()
    if world == 1:
        return last, first
    rank = dist.get_rank()
    up, down = (rank + 1) % world, (rank - 1) % world
    below = torch.empty_like(first)
    above = torch.empty_like(last)
    # a rank's first planes become the lower neighbour's `above` (tag 1),
    # its last planes the upper neighbour's `below` (tag 2).  With two ranks
    # both neighbours are the same rank; backends that match messages of a
    # pair in issue order (NCCL ignores tags) then need the receives in the
    # order of the peer's sends: first `above`, then `below`.
    ops = [dist.P2POp(dist.isend, first, down, tag=1), dist.P2POp(dist.isend, last, up, tag=2),
           dist.P2POp(dist.irecv, above, up, tag=1), dist.P2POp(dist.irecv, below, down, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return below, above
