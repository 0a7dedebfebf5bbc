"""Batched filtering of uneven cells (sq3_batch_*) against the single-cell
FP32 filter of the same library (sq3_cheb_filter, SQ3_MIXED, no
projectors) and against the oracle's filter by its plain definition.

The batched launch computes each cell with the single-cell ring stencil's
tiling in FP32; its taps are summed per axis with the weights as constants
and scaled by the spacings afterwards (the single-cell step multiplies each
tap by its own rounded coefficient), so the two agree to FP32 rounding of
the whole filter: 1e-5 of the block's largest value after up to 12 steps
(a few ulps per step, carried along by the recurrence).  Against the FP64
oracle the FP32 filter of degree <= 12 stays within 1e-5 relative (L2).  Cells of different grids (cubic and not), numbers of vectors and
degrees share the launches; the autotuner keeps the results unchanged."""
import numpy as np
import pytest
import torch

from oracle import chebyshev, hamiltonian
from paper_2112_08639_gb300 import inputs

from gpu_common import need_gpu, sq3

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CELLS = [  # (grid, lengths, Ns, degree, seed)
    ((24, 24, 24), (7.78, 7.78, 7.78), 20, 10, 0),
    ((32, 24, 20), (10.0, 7.78, 6.5), 12, 7, 1),
    ((16, 16, 16), (5.2, 5.2, 5.2), 9, 12, 2),
]


def _cell(n, L, seed):
    pos = inputs.fcc_positions(1, disp_sigma=0.3, seed=seed) * np.array(L) / inputs.A0_FCC
    # the periodic local potential of the inputs module on a cubic grid of
    # the cell's largest side, sampled on this grid
    g = np.random.default_rng(seed)
    k = np.arange(np.prod(n))
    x, y, z = k % n[0], (k // n[0]) % n[1], k // (n[0] * n[1])
    V = np.zeros(np.prod(n))
    for R in pos:
        dx = np.minimum(np.abs(x * L[0] / n[0] - R[0]), L[0] - np.abs(x * L[0] / n[0] - R[0]))
        dy = np.minimum(np.abs(y * L[1] / n[1] - R[1]), L[1] - np.abs(y * L[1] / n[1] - R[1]))
        dz = np.minimum(np.abs(z * L[2] / n[2] - R[2]), L[2] - np.abs(z * L[2] / n[2] - R[2]))
        V -= 1.5 * np.exp(-(dx * dx + dy * dy + dz * dz) / 1.5)
    return V + 0.1 * g.normal(size=V.size)


def _bounds(V, n, L):
    hi = 0.5 * sum(7.0729 / (L[a] / n[a]) ** 2 for a in range(3)) + V.max()
    a0 = V.min() - 0.1
    return a0 + 0.1 * (hi - a0), hi, a0


def test_batched_filter_matches_single_cell_filter_and_oracle():
    m = sq3()
    batch = m.Batch(0)
    blocks, refs = [], []
    for (n, L, Ns, deg, seed) in CELLS:
        V = _cell(n, L, seed)
        N = int(np.prod(n))
        X0 = inputs.random_block(N, Ns, seed=seed).astype(np.float32)
        Xb = torch.from_numpy(X0).cuda()
        idx = batch.add_cell(n, L, torch.from_numpy(V), Xb, deg)
        a, b, a0 = _bounds(V, n, L)
        batch.set_bounds(idx, a, b, a0)
        # the single-cell filter of the same library on a copy
        ctx = m.Context(0)
        ctx.setup_grid(*n, *L, 12)
        ctx.set_potential(torch.from_numpy(V))
        Xs = torch.from_numpy(X0).cuda()
        ctx.cheb_filter(Xs, deg, a, b, a0, m.MIXED)
        blocks.append(Xb)
        refs.append((Xs.cpu().numpy(), X0, V, n, L, deg, (a, b, a0)))
    batch.filter()
    for Xb, (Xs, X0, V, n, L, deg, (a, b, a0)) in zip(blocks, refs):
        got = Xb.cpu().numpy()
        assert np.max(np.abs(got - Xs)) <= 1e-5 * np.max(np.abs(Xs))
    # the cubic cell against the oracle's plain filter in FP64
    Xs, X0, V, n, L, deg, (a, b, a0) = refs[0]
    parts = hamiltonian.hamiltonian_sparse(n[0], L[0], V)
    ref = chebyshev.filter_plain(lambda Z: hamiltonian.apply(parts, Z), X0.T.astype(np.float64),
                                 deg, a, b, a0).T
    got = blocks[0].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) < 1e-5 * np.linalg.norm(ref)


def test_autotune_keeps_the_results_and_new_bounds_reuse_the_graph():
    m = sq3()
    batch = m.Batch(0)
    blocks = []
    for (n, L, Ns, deg, seed) in CELLS:
        V = _cell(n, L, seed)
        X0 = inputs.random_block(int(np.prod(n)), Ns, seed=seed).astype(np.float32)
        Xb = torch.from_numpy(X0).cuda()
        batch.set_bounds(batch.add_cell(n, L, torch.from_numpy(V), Xb, deg), *_bounds(V, n, L))
        blocks.append((Xb, X0))
    saved = [X.clone() for X, _ in blocks]
    ctas, div = batch.autotune()
    assert ctas in (1, 2) and div in (1, 2)
    for (X, _), s in zip(blocks, saved):
        assert torch.equal(X, s)                     # the blocks were put back
    batch.filter()
    first = [X.clone() for X, _ in blocks]
    # a second filter with other bounds (same graph) from the same blocks
    for i, ((X, X0), (n, L, Ns, deg, seed)) in enumerate(zip(blocks, CELLS)):
        X.copy_(torch.from_numpy(X0))
        a, b, a0 = _bounds(_cell(n, L, seed), n, L)
        batch.set_bounds(i, a + 0.5, b, a0)
    batch.filter()
    for (X, _), f in zip(blocks, first):
        assert not torch.equal(X, f)                 # the new bounds were used
    for i, ((X, X0), (n, L, Ns, deg, seed)) in enumerate(zip(blocks, CELLS)):
        X.copy_(torch.from_numpy(X0))
        batch.set_bounds(i, *_bounds(_cell(n, L, seed), n, L))
    batch.filter()
    for (X, _), f in zip(blocks, first):
        assert torch.equal(X, f)                     # and reproducibly


def test_batch_error_paths():
    m = sq3()
    batch = m.Batch(0)
    with pytest.raises(m.SQ3Error):
        batch.filter()                               # no cells
    X = torch.zeros((4, 12 * 12 * 12), dtype=torch.float32, device="cuda")
    with pytest.raises(m.SQ3Error):                  # nx below 16
        batch.add_cell((12, 12, 12), (4.0, 4.0, 4.0), torch.zeros(1728, dtype=torch.float64), X, 5)
