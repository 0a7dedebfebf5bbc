"""The sharded form of one cell's path (paper_2112_08639_gb300.sharding) on
two and three gloo ranks on the CPU, against the same computation on one
rank:

* grid slabs: the Gram matrix X^T X and the projection X^T (H X) as
  all-reduced sums of per-slab products, H X computed on each slab with
  the stencil planes of the neighbouring slabs from the halo exchange
  (periodic in z);
* column blocks: the Chebyshev recurrence T_{j+1} = 2 Hhat T_j - T_{j-1}
  on each rank's columns with no exchange, the moments all-reduced, and
  the density kernel all-gathered for the slab-local density.

The per-rank arithmetic here is float64 torch on the CPU, standing in for
the library's kernels; what is tested is the partitioning and the exchange
steps.  No GPU is used."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_GRID, NS, R, NPL = 8, 12, 2, 9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    g = torch.Generator().manual_seed(3)
    X = torch.randn(NS, N_GRID, N_GRID, N_GRID, generator=g, dtype=torch.float64)
    V = torch.randn(N_GRID, N_GRID, N_GRID, generator=g, dtype=torch.float64)
    w = torch.tensor([-2.5, 1.333, -0.0833], dtype=torch.float64)   # a radius-2 star
    A = torch.randn(NS, NS, generator=g, dtype=torch.float64)
    Hs = 0.5 * (A + A.T) / NS
    return X, V, w, Hs


def _stencil(Xp, V, w, z_lo):
    """H x = -1/2 star(x) + V x on planes z_lo .. of a padded slab Xp
    (..., planes + 2R, ny, nx): x and y periodic, z from the padding."""
    out = torch.zeros_like(Xp[..., R:-R, :, :])
    core = Xp[..., R:-R, :, :]
    acc = 3 * w[0] * core
    for p in range(1, R + 1):
        acc = acc + w[p] * (torch.roll(core, p, -1) + torch.roll(core, -p, -1) +
                            torch.roll(core, p, -2) + torch.roll(core, -p, -2) +
                            Xp[..., R - p:Xp.shape[-3] - R - p, :, :] +
                            Xp[..., R + p:Xp.shape[-3] - R + p, :, :])
    out = -0.5 * acc + V[z_lo:z_lo + core.shape[-3]] * core
    return out


def _reference():
    X, V, w, Hs = _data()
    Xp = torch.cat([X[..., -R:, :, :], X, X[..., :R, :, :]], dim=-3)
    HX = _stencil(Xp, V, w, 0)
    Xf, HXf = X.reshape(NS, -1), HX.reshape(NS, -1)
    T = [torch.eye(NS, dtype=torch.float64), Hs.clone()]
    for _ in range(1, NPL):
        T.append(2 * Hs @ T[-1] - T[-2])
    m = torch.stack([torch.trace(t) for t in T])
    return Xf @ Xf.T, Xf @ HXf.T, m, T[-1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    from paper_2112_08639_gb300 import sharding
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, V, w, Hs = _data()
        z0, z1 = sharding.grid_slab(N_GRID, world, rank)
        slab = X[..., z0:z1, :, :].contiguous()
        below, above = sharding.halo_planes(slab, R)
        HX = _stencil(torch.cat([below, slab, above], dim=-3), V, w, z0)
        S = sharding.gram_slabs(slab.reshape(NS, -1), slab.reshape(NS, -1))
        Hsl = sharding.gram_slabs(slab.reshape(NS, -1), HX.reshape(NS, -1))
        j0, j1 = sharding.column_block(NS, world, rank)
        I = torch.eye(NS, dtype=torch.float64)
        T = [I[:, j0:j1].clone(), Hs[:, j0:j1].clone()]
        for _ in range(1, NPL):
            T.append(2 * Hs @ T[-1] - T[-2])
        m = sharding.moments_columns(T, j0)
        Tlast = sharding.gather_columns(T[-1], NS)
        out[rank] = (S.numpy(), Hsl.numpy(), m.numpy(), Tlast.numpy(), (z0, z1), (j0, j1))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gram_projection_and_moments_equal_one_rank(world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    S_ref, Hs_ref, m_ref, T_ref = (t.numpy() for t in _reference())
    # the slabs and column blocks tile the grid and the columns exactly
    assert sorted(r[4] for r in res.values())[0][0] == 0
    assert sum(r[4][1] - r[4][0] for r in res.values()) == N_GRID
    assert sum(r[5][1] - r[5][0] for r in res.values()) == NS
    for r in range(world):
        S, Hs, m, T, _, _ = res[r]
        np.testing.assert_allclose(S, S_ref, rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(Hs, Hs_ref, rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(m, m_ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(T, T_ref, rtol=1e-13, atol=1e-13)


def test_partitions_on_one_rank_and_uneven_sizes():
    sys.path.insert(0, ROOT)
    from paper_2112_08639_gb300 import sharding
    blocks = [sharding.column_block(10, 4, r) for r in range(4)]
    assert blocks == [(0, 3), (3, 6), (6, 8), (8, 10)]
    assert sharding.grid_slab(72, 1, 0) == (0, 72)
    with pytest.raises(ValueError):
        sharding.grid_slab(2, 3, 0)
