"""CPU checks of the QMD driver's checkpoint and metrics files (no device:
a stand-in cell holds the state tensors on the host).

* save_checkpoint / load_checkpoint restore the block, the density kernel,
  the previous density and positions, the spectral bounds, the nuclei and
  the trajectory exactly, and refuse a checkpoint of another configuration;
* write_metrics writes one JSON line per SCF iteration and one per step."""
import json
import types

import numpy as np
import pytest
import torch


def _qmd():
    from paper_2112_08639_gb300 import build
    build.build()
    from paper_2112_08639_gb300 import qmd
    return qmd


def _cell(name="al4_test", prec=1, seed=0, Ns=6, N=40):
    g = torch.Generator().manual_seed(seed)
    c = types.SimpleNamespace()
    c.cfg = types.SimpleNamespace(name=name)
    c.prec = prec
    c.X = torch.randn((Ns, N), generator=g, dtype=torch.float32)
    c.D = torch.randn((Ns, Ns), generator=g, dtype=torch.float64)
    c.rho = torch.zeros(N, dtype=torch.float64)
    c.rho_prev = torch.rand(N, generator=g, dtype=torch.float64)
    c.pos_prev = np.random.default_rng(seed).normal(size=(4, 3))
    c.bounds = (0.25 + seed, 3.5)
    return c


def test_checkpoint_round_trip(tmp_path):
    qmd = _qmd()
    a = _cell(seed=1)
    rng = np.random.default_rng(2)
    R, V, F = rng.normal(size=(4, 3)), rng.normal(size=(4, 3)), rng.normal(size=(4, 3))
    traj = {"R": [R, R + 1], "iterations": [30, 7], "F": [-1.5, -1.6], "E_kin": [0.1, 0.1],
            "converged": [1, 1]}
    path = str(tmp_path / "qmd.ckpt")
    qmd.save_checkpoint(path, a, 1, R, V, F, 0.1, traj)
    b = _cell(seed=7)                          # different state, same shapes
    st = qmd.load_checkpoint(path, b)
    assert torch.equal(b.X, a.X) and torch.equal(b.D, a.D)
    assert torch.equal(b.rho_prev, a.rho_prev)
    assert np.array_equal(b.pos_prev, a.pos_prev) and b.bounds == a.bounds
    assert st["step"] == 1 and st["ke0"] == 0.1
    assert np.array_equal(st["R"], R) and np.array_equal(st["V"], V)
    assert np.array_equal(st["F"], F)
    assert st["traj"]["iterations"] == [30, 7]
    with pytest.raises(ValueError):
        qmd.load_checkpoint(path, _cell(name="al32_other"))
    with pytest.raises(ValueError):
        qmd.load_checkpoint(path, _cell(prec=0))


def test_metrics_lines(tmp_path):
    qmd = _qmd()
    path = tmp_path / "m.jsonl"
    hist = [{"err": 1e-2, "mu": 0.1, "F": -3.0}, {"err": 1e-6, "mu": 0.11, "F": -3.1}]
    res = {"iterations": 2, "converged": 1, "F": -3.1, "mu": 0.11, "err": 1e-6}
    with open(path, "w") as f:
        qmd.write_metrics(f, 4, res, hist, 0.25)
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert [l["kind"] for l in lines] == ["scf", "scf", "step"]
    assert [l["iteration"] for l in lines[:2]] == [1, 2]
    assert lines[1]["err"] == 1e-6 and lines[2]["iterations"] == 2
    assert all(l["step"] == 4 for l in lines) and lines[2]["E_kin"] == 0.25
