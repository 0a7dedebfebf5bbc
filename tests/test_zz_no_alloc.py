"""The allocation-free spectral-bounds entry point.

sq3_lanczos_bounds_noalloc serves callers that cannot let a library allocate
device memory (a process that reserves HBM for its own arena, or a loop in
which a device allocation would stall other streams): it keeps its scratch
in a fixed device array inside the library.  These tests call it through the
C ABI and check that it returns the same chi and xi as the Lanczos step of
sq3_kernel_from_hs, on two calls in a row (the array keeps the previous
call's contents, which must not leak into the next result).  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch
from scipy.stats import ortho_group

from gpu_common import c1_cell, context_for, need_gpu, sq3

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _hs(Ns, seed):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(-1.2, 3.5, Ns))
    Q = ortho_group.rvs(Ns, random_state=seed)
    return (Q * lam) @ Q.T


def test_noalloc_bounds_match_context_entry_point_twice():
    m = sq3()
    ctx = context_for(c1_cell())
    for Ns, seed in ((300, 1), (64, 2)):            # a larger call, then a smaller one
        Hs = torch.from_numpy(_hs(Ns, seed)).cuda()
        _, ref = ctx.kernel_from_hs(Hs, 20, 0.3675, 0.4 * Ns, want_D=False)
        for _ in range(2):
            b = m.lanczos_bounds_noalloc(Hs).cpu().numpy()
            assert abs(b[0] - ref["chi"]) <= 1e-12 * max(1.0, abs(ref["chi"]))
            assert abs(b[1] - ref["xi"]) <= 1e-12 * ref["xi"]
        lam = np.linalg.eigvalsh(Hs.cpu().numpy())
        assert b[0] - b[1] <= lam[0] + 1e-12 and b[0] + b[1] >= lam[-1] - 1e-12


def test_noalloc_rejects_sizes_beyond_its_array():
    m = sq3()
    Hs = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    rc = m.lib.sq3_lanczos_bounds_noalloc(m._ptr(Hs), m.NOALLOC_MAX_NS + 1, m._ptr(out), None)
    assert rc == m.EINVAL
    rc = m.lib.sq3_lanczos_bounds_noalloc(None, 4, m._ptr(out), None)
    assert rc == m.EINVAL
