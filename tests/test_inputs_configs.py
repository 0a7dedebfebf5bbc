"""CPU checks of the workload table: the batched workload C4 spans its
recipe (uneven FCC cells of 4 to 32 atoms on 0.324-bohr grids, Ns = 20 per
atom, kT from 5 to 20 eV) and C5 is the 32-atom cell's QMD run at kT = 10 eV
(116,045 K: the temperature of Sec. 5's Al runs)."""
import numpy as np

from paper_2112_08639_gb300 import inputs


def test_c4_batch_cells_span_the_recipe():
    cells = inputs.batch_cells(64, seed=0)
    assert len(cells) == 64
    atoms = {c["natoms"] for c in cells}
    assert atoms <= {4, 8, 16, 32} and len(atoms) >= 3
    for c in cells:
        L, n = np.array(c["L"]), np.array(c["n"])
        assert np.allclose(L / n, inputs.A0_FCC / 24)            # 0.324 bohr
        assert set(c["n"]) <= {24, 48}
        assert c["Ns"] == 20 * c["natoms"] and 80 <= c["Ns"] <= 640
        assert 5.0 <= c["kT"] <= 20.0 and c["m"] == 20
        assert np.all(c["pos"] >= 0) and np.all(c["pos"] < L)
    # seeded: the same cells again, other cells for another seed
    again = inputs.batch_cells(64, seed=0)
    assert all(np.array_equal(a["pos"], b["pos"]) for a, b in zip(cells, again))
    assert not np.array_equal(inputs.batch_cells(1, seed=1)[0]["pos"][:4], cells[0]["pos"][:4])
    small = inputs.small_cells(16, seed=1)
    assert 0 < len(small) <= 16 and all(c["natoms"] == 4 and c["Ns"] == 80 for c in small)


def test_c5_is_the_32_atom_qmd_run():
    c5 = inputs.C5
    assert c5.cell is inputs.C2 and c5.cell.natoms == 32 and c5.cell.n == 48
    assert c5.dt_fs == 0.5 and c5.nsteps == 300 and c5.train_steps == 100
    k_b_ev = 8.617333262e-5                                       # eV / K
    assert abs(c5.cell.kT_ev / k_b_ev - 116045) < 1.0
    assert abs(c5.mass_amu - 26.98) < 0.01
