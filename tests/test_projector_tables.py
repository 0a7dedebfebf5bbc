"""CPU checks of the host side of the Kleinman-Bylander projector tables
(sq3_projector_table_info: the tables sq3_set_projectors builds, computed on
the host without a device).

Pins, each independent of the library's arithmetic:
* the Gershgorin bounds enclose every eigenvalue of V_nl = sum_p gamma_p
  c_p c_p^T (Sec. 2, Eq. (nonlocaloperator)), assembled densely and
  diagonalised by numpy, and its largest eigenvalue is within the bound's
  width of the bound (the bound is not vacuous);
* the number of (point, ball) entries, of balls and the largest number of
  entries and balls in one 8 x 8 x 4 brick equal a plain numpy count;
* a grid index repeated inside a projector (its values split in two) gives
  the same counts and bounds as the merged table;
* malformed tables are rejected."""
import numpy as np
import pytest

from paper_2112_08639_gb300 import inputs

N_GRID = 16
L = 7.78


def _sq3():
    from paper_2112_08639_gb300 import build
    build.build()
    from paper_2112_08639_gb300 import sq3
    return sq3


def _table(seed=0, natoms_cells=1, n=N_GRID):
    pos = inputs.fcc_positions(natoms_cells, disp_sigma=0.3, seed=seed) * (L / inputs.A0_FCC)
    return inputs.projectors(n, L * natoms_cells, pos, seed=seed), pos


def _dense_vnl(pr, N, dV):
    V = np.zeros((N, N))
    for p in range(pr.n_proj):
        c = np.zeros(N)
        np.add.at(c, pr.idx[pr.ptr[p]:pr.ptr[p + 1]], pr.val[pr.ptr[p]:pr.ptr[p + 1]] * np.sqrt(dV))
        V += pr.gamma[p] * np.outer(c, c)
    return V


@pytest.mark.parametrize("seed", [0, 3])
def test_gershgorin_bounds_enclose_the_spectrum_of_vnl(seed):
    sq3 = _sq3()
    pr, _ = _table(seed)
    N = N_GRID ** 3
    dV = (L / N_GRID) ** 3
    info = sq3.projector_table_info((N_GRID,) * 3, dV, pr.ptr, pr.idx, pr.val, pr.gamma)
    lam = np.linalg.eigvalsh(_dense_vnl(pr, N, dV))
    lo, hi = info["vnl_lo"], info["vnl_hi"]
    assert lo <= lam.min() + 1e-12 and lam.max() <= hi + 1e-12
    assert lo <= 0.0 <= hi
    # the upper bound is a Gershgorin bound of Gamma S, not a loose guess
    assert hi - lam.max() <= hi - lo


def test_brick_counts_equal_a_plain_count():
    sq3 = _sq3()
    pr, _ = _table(1)
    n = N_GRID
    dV = (L / n) ** 3
    info = sq3.projector_table_info((n, n, n), dV, pr.ptr, pr.idx, pr.val, pr.gamma)
    # balls: the 4 projectors of an atom share one index list
    assert info["balls"] == pr.n_proj // 4
    pts = [pr.idx[pr.ptr[4 * a]:pr.ptr[4 * a + 1]] for a in range(pr.n_proj // 4)]
    assert info["entries"] == sum(len(np.unique(p)) for p in pts)
    brick = lambda k: (k % n) // 8 + ((n + 7) // 8) * (((k // n) % n) // 8 +
                                                          ((n + 7) // 8) * ((k // (n * n)) // 4))
    nb = ((n + 7) // 8) ** 2 * ((n + 3) // 4)
    ent = np.zeros(nb, int)
    balls = [set() for _ in range(nb)]
    for a, p in enumerate(pts):
        for b in brick(np.unique(p)):
            ent[b] += 1
            balls[b].add(a)
    assert info["bricks"] == nb
    assert info["max_brick_entries"] == ent.max()
    assert info["max_brick_balls"] == max(len(s) for s in balls)
    assert info["smem_bytes"] > 0


def test_repeated_indices_are_merged():
    sq3 = _sq3()
    pr, _ = _table(2)
    dV = (L / N_GRID) ** 3
    ref = sq3.projector_table_info((N_GRID,) * 3, dV, pr.ptr, pr.idx, pr.val, pr.gamma)
    # every projector's first entry split into two halves, listed twice
    ptr, idx, val = [0], [], []
    for p in range(pr.n_proj):
        a, b = pr.ptr[p], pr.ptr[p + 1]
        idx += [pr.idx[a], pr.idx[a]] + list(pr.idx[a + 1:b])
        val += [0.5 * pr.val[a], 0.5 * pr.val[a]] + list(pr.val[a + 1:b])
        ptr.append(len(idx))
    got = sq3.projector_table_info((N_GRID,) * 3, dV, ptr, idx, val, pr.gamma)
    for k in ("balls", "entries", "bricks", "max_brick_balls", "max_brick_entries"):
        assert got[k] == ref[k], k
    assert got["vnl_lo"] == pytest.approx(ref["vnl_lo"], abs=1e-12)
    assert got["vnl_hi"] == pytest.approx(ref["vnl_hi"], rel=1e-12)


def test_malformed_tables_are_rejected():
    sq3 = _sq3()
    pr, _ = _table(0)
    dV = (L / N_GRID) ** 3
    g = (N_GRID,) * 3
    bad = pr.val.copy()
    bad[3] = np.nan
    for args in ((pr.ptr, pr.idx, bad, pr.gamma),
                 (pr.ptr, np.where(np.arange(len(pr.idx)) == 5, N_GRID ** 3, pr.idx), pr.val,
                  pr.gamma),
                 (pr.ptr, pr.idx, pr.val, np.where(np.arange(pr.n_proj) == 1, np.inf,
                                                   pr.gamma))):
        with pytest.raises(sq3.SQ3Error) as e:
            sq3.projector_table_info(g, dV, *args)
        assert e.value.code == sq3.EINVAL
    with pytest.raises(sq3.SQ3Error):
        sq3.projector_table_info(g, -1.0, pr.ptr, pr.idx, pr.val, pr.gamma)
    empty = sq3.projector_table_info(g, dV, [0], [], [], [])
    assert empty["balls"] == 0 and empty["vnl_lo"] == 0.0 and empty["vnl_hi"] == 0.0
