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
