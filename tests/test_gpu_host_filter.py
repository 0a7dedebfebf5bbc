"""sq3_cheb_filter_from_host: the Chebyshev filter of a block held in host
memory, uploaded in two chunks of vectors (the first eighth, then the rest),
the second overlapping the filtering of the first.  The result must be the
filter of sq3_cheb_filter (the same kernels on each chunk of vectors) and
the oracle's filter; uneven chunks (Ns = 7: 1 + 6, 13: 2 + 11, 3: 1 + 2)
are covered.
"""
import numpy as np
import pytest
import torch

from oracle import chebyshev
from paper_2112_08639_gb300 import inputs

from gpu_common import (apply_fn, c1_cell, context_for, from_gpu_block, need_gpu, oracle_parts,
                        small_proj_cell, sq3, to_gpu_block)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cellf,Ns,m", [(c1_cell, 7, 12), (small_proj_cell, 13, 16),
                                        (small_proj_cell, 3, 10)])
def test_filter_from_host_matches_device_filter_and_oracle(prec, cellf, Ns, m):
    cell = cellf()
    ctx = context_for(cell)
    p = sq3().FP64 if prec == "fp64" else sq3().MIXED
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = inputs.random_block(cell.cfg.N, Ns, seed=11).T
    X = X.astype(np.float32).astype(np.float64) if prec == "mixed" else X
    a0, a, b = -1.8, 2.0, 60.0
    Xd = to_gpu_block(X, dt)
    Xh = Xd.cpu().pin_memory()
    ctx.cheb_filter(Xd, m, a, b, a0, prec=p)
    Xo = torch.empty_like(Xh, device="cuda:0")
    ctx.cheb_filter_from_host(Xh, Xo, m, a, b, a0, prec=p)
    ref = chebyshev.filter_plain(apply_fn(oracle_parts(cell)), X, m, a, b, a0)
    got = from_gpu_block(Xo)
    # same kernels per vector; only the order of the projection atomics differs
    assert _rel(got, from_gpu_block(Xd)) < (1e-12 if prec == "fp64" else 1e-6)
    assert _rel(got, ref) < (1e-12 if prec == "fp64" else 1e-5)


def test_filter_from_host_rejects_device_source():
    cell = c1_cell()
    ctx = context_for(cell)
    Xd = to_gpu_block(inputs.random_block(cell.cfg.N, 4, seed=2).T)
    with pytest.raises(ValueError):
        ctx.cheb_filter_from_host(Xd, torch.empty_like(Xd), 4, 2.0, 60.0, -1.8)
