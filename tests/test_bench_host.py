"""CPU checks of the bench's roofline arithmetic: the algorithmic work per
launch of each dominant kernel class equals its closed form (three words
per point and vector for the FP32 stencil, a read and a write of the
covered points for the nonlocal pass, the useful flops of each GEMM with
six BF16 piece products issued per useful product, about 80 flop per point
and vector for the FP64 stencil), and the fraction is achieved / peak."""
import pytest

import bench
from paper_2112_08639_gb300 import inputs

PK = {"hbm_gbs": 6679.8, "bf16_tflops": 1899.4, "bf16_tflops_sustained": 1722.8}


def _entry(kind, ms=2.0, n=2, fp64=False, n_covered=None):
    cfg = inputs.C3
    prof = {kind: (ms, n)}
    esize = 8 if fp64 else 4
    return bench.roofline(kind, prof, cfg, esize, fp64, PK, "test",
                          cfg.N if n_covered is None else n_covered), cfg


def test_stencil_fp32_is_three_words_per_point_and_vector():
    r, cfg = _entry("stencil")                         # 1 ms per launch
    algo = 3 * cfg.N * cfg.Ns * 4
    assert r["bound"] == "hbm" and r["algorithmic"] == pytest.approx(algo / 1e9, abs=1e-3)
    assert abs(algo / 1e9 - 9.853) < 1e-3                 # 72^3 points x 2200 vectors
    assert r["achieved"] == pytest.approx(algo / 1e-3 / 1e9, abs=0.1)
    assert r["frac"] == pytest.approx(r["achieved"] / PK["hbm_gbs"], abs=1e-4)
    traffic = bench.MEASURED_TRAFFIC["stencil"][0] * cfg.N * cfg.Ns / 1e9
    assert r["traffic"] == pytest.approx(traffic, abs=1e-3)


def test_nonlocal_pass_reads_and_writes_the_covered_points():
    r, cfg = _entry("nl_pass", n_covered=300_000)
    algo = 2 * 300_000 * cfg.Ns * 4
    assert r["algorithmic"] == pytest.approx(algo / 1e9, abs=1e-3)
    assert r["achieved"] == pytest.approx(algo / 1e-3 / 1e9, abs=0.1)


@pytest.mark.parametrize("kind,flops", [("gram", "NNs2"), ("hs_gemm", "NNs2"),
                                        ("x_rinv", "NNs2"), ("rho", "NNs2"),
                                        ("cheb_gemm", "Ns3")])
def test_gemm_useful_flops_and_piece_products(kind, flops):
    r, cfg = _entry(kind)
    useful = cfg.N * cfg.Ns ** 2 if flops == "NNs2" else cfg.Ns ** 3
    assert r["bound"] == "tensor"
    assert r["useful"] == pytest.approx(useful / 1e-3 / 1e12, abs=0.01)
    assert r["achieved"] == pytest.approx(6 * r["useful"], abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / PK["bf16_tflops_sustained"], abs=1e-4)


def test_fp64_paths_report_against_the_derived_fp64_peak():
    r, cfg = _entry("stencil", fp64=True)
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(80 * cfg.N * cfg.Ns / 1e-3 / 1e12, abs=1e-3)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12, abs=1e-4)


@pytest.mark.parametrize("Ns", [640, 2200])
def test_symmetric_gemm_flops_against_the_tile_schedule(Ns):
    """The Gram product computes only the 128 x 128 output tiles on or above
    the diagonal (nt (nt + 1) / 2 of nt^2): the multiply-adds those tiles
    issue, 128^2 N per tile, bound the bench's useful count N Ns^2 (the
    product's upper triangle with the diagonal, 2 N Ns (Ns + 1) / 2 flops)
    from above, and exceed it only by the diagonal tiles' lower halves and
    the padding of the last tile row."""
    N = inputs.C3.N
    nt = (Ns + 127) // 128
    tiles = nt * (nt + 1) // 2
    issued = 2 * 128 * 128 * N * tiles
    useful = N * Ns * Ns
    exact_upper = N * Ns * (Ns + 1)
    assert exact_upper >= useful
    assert issued >= exact_upper
    pad = nt * 128
    assert issued <= 2 * N * pad * (pad + 128) / 2 + 1


def test_one_thread_oracle_sample_runs_in_a_child_process():
    """The 1-thread CPU figure: the same oracle sample in a fresh process
    with the BLAS pools at one thread (32-atom cell, one pass)."""
    v = bench.run_oracle_sample_one_thread("al32_48", 1)
    assert v is not None and v > 0.0


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host cores, no
    device) prints one JSON line with the reference arm's keys."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--config", "al32_48", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "s" and line["value"] > 0
    assert line["higher_is_better"] is False and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "sample" in cb
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
