"""Failure detection on the device without a fault: a kernel waits on an
mbarrier that nothing completes, through the library's bounded wait; the
wait runs out after about a second, the kernel records a timeout and
returns, the host reads SQ3_ETIMEOUT, and the same context then computes
correctly.  Nothing traps, faults or hangs."""
import time

import numpy as np
import pytest
import torch

from paper_2112_08639_gb300 import inputs

from gpu_common import (c1_cell, context_for, from_gpu_block, need_gpu, oracle_parts, sq3,
                        to_gpu_block)
from oracle import hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    cell = c1_cell()
    ctx = context_for(cell)
    m = sq3()
    t0 = time.perf_counter()
    rc = ctx.selftest_timeout()
    dt = time.perf_counter() - t0
    assert rc == m.ETIMEOUT
    assert 0.5 < dt < 30.0                       # about one second of waiting, bounded
    # the status word was cleared: the next call on the context succeeds
    X = inputs.random_block(cell.cfg.N, 5, seed=4).T
    Y = ctx.hamiltonian_apply(to_gpu_block(X))
    ref = hamiltonian.apply(oracle_parts(cell), X)
    assert np.linalg.norm(from_gpu_block(Y) - ref) < 1e-12 * np.linalg.norm(ref)
    assert ctx.selftest_timeout() == m.ETIMEOUT  # and the path repeats


def _usable(ctx, cell):
    """The context still applies H correctly."""
    X = inputs.random_block(cell.cfg.N, 3, seed=9).T
    Y = ctx.hamiltonian_apply(to_gpu_block(X))
    ref = hamiltonian.apply(oracle_parts(cell), X)
    return np.linalg.norm(from_gpu_block(Y) - ref) < 1e-12 * np.linalg.norm(ref)


def test_nan_in_the_potential_is_reported_and_the_context_recovers():
    """A NaN planted on the host in V: sq3_set_potential returns
    SQ3_ENONFINITE (the range check of the potential), and setting a
    finite potential again makes the context usable."""
    m = sq3()
    cell = c1_cell()
    ctx = context_for(cell)
    V = cell.V.copy()
    V[123] = np.nan
    with pytest.raises(m.SQ3Error) as e:
        ctx.set_potential(torch.from_numpy(V))
    assert e.value.code == m.ENONFINITE
    ctx.set_potential(torch.from_numpy(cell.V))
    assert _usable(ctx, cell)


def test_corrupted_projector_table_is_rejected():
    """A NaN among the projector values, a NaN energy and an index outside
    the grid are rejected with SQ3_EINVAL before any device work; a
    duplicated grid index inside one projector is legal (its values add)
    and gives the same H as the summed value."""
    from gpu_common import small_proj_cell
    m = sq3()
    cell = small_proj_cell()
    ctx = context_for(cell)
    pr = cell.proj
    bad = pr.val.copy()
    bad[7] = np.nan
    with pytest.raises(m.SQ3Error) as e:
        ctx.set_projectors(pr.ptr, pr.idx, bad, pr.gamma)
    assert e.value.code == m.EINVAL
    g = pr.gamma.copy()
    g[2] = np.inf
    with pytest.raises(m.SQ3Error) as e:
        ctx.set_projectors(pr.ptr, pr.idx, pr.val, g)
    assert e.value.code == m.EINVAL
    idx = pr.idx.copy()
    idx[5] = cell.cfg.N
    with pytest.raises(m.SQ3Error) as e:
        ctx.set_projectors(pr.ptr, idx, pr.val, pr.gamma)
    assert e.value.code == m.EINVAL
    # a duplicated index: projector 0's first entry split into two halves
    a, b = int(pr.ptr[0]), int(pr.ptr[1])
    idx2 = np.concatenate([pr.idx[a:a + 1], pr.idx[a:b], pr.idx[b:]])
    val2 = np.concatenate([0.5 * pr.val[a:a + 1], np.r_[0.5 * pr.val[a], pr.val[a + 1:b]],
                           pr.val[b:]])
    ptr2 = pr.ptr.copy()
    ptr2[1:] += 1
    ctx2 = context_for(cell)
    ctx2.set_projectors(ptr2, idx2, val2, pr.gamma)
    X = to_gpu_block(inputs.random_block(cell.cfg.N, 4, seed=2).T)
    ctx.set_projectors(pr.ptr, pr.idx, pr.val, pr.gamma)     # the rejected tables left no trace
    Y1 = ctx.hamiltonian_apply(X)
    Y2 = ctx2.hamiltonian_apply(X)
    assert torch.allclose(Y1, Y2, rtol=0, atol=1e-12 * float(Y1.abs().max()))


def test_nan_in_the_block_or_the_kernel_is_reported():
    """A NaN planted in the block: the Cholesky of its Gram matrix meets a
    non-finite pivot (SQ3_ENOTPD); a NaN in Ds reaches rho and
    sq3_density returns SQ3_ENONFINITE; N_e >= 2 Ns is SQ3_EINVAL.  The
    context computes correctly afterwards."""
    m = sq3()
    cell = c1_cell()
    ctx = context_for(cell)
    X = to_gpu_block(inputs.random_block(cell.cfg.N, 16, seed=3).T)
    X[4, 17] = float("nan")
    with pytest.raises(m.SQ3Error) as e:
        ctx.orthonormalise(X)
    assert e.value.code == m.ENOTPD
    X = to_gpu_block(inputs.random_block(cell.cfg.N, 16, seed=3).T)
    ctx.orthonormalise(X)
    D = torch.eye(16, dtype=torch.float64, device="cuda") * 0.5
    D[3, 3] = float("nan")
    with pytest.raises(m.SQ3Error) as e:
        ctx.density(X, D)
    assert e.value.code == m.ENONFINITE
    with pytest.raises(m.SQ3Error) as e:
        ctx.density_kernel(X, 20, cell.cfg.sigma, 32.0)
    assert e.value.code == m.EINVAL
    assert _usable(ctx, cell)
