"""The bench's accounting on CPU: HPCG's flop-counting rule per CG iteration,
the per-row algorithmic byte model the whole-solve rooflines use, and the
whole-job value of N replicas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_level_sizes_closed_form():
    for m in (16, 192):
        for l, (n, nnz) in enumerate(bench.level_sizes(m, m, m, 4)):
            e = m >> l
            assert n == e ** 3 and nnz == (3 * e - 2) ** 3


def test_hpcg_flop_rule_192cubed():
    # 2 nnz_0 + 12 n_0 + sum over levels 0..2 of (10 nnz_l + 2 n_{l+1}) + 4 nnz_3
    sz = bench.level_sizes(192, 192, 192, 4)
    expect = 2 * sz[0][1] + 12 * sz[0][0] + sum(10 * sz[l][1] + 2 * sz[l + 1][0] for l in range(3)) + 4 * sz[3][1]
    f = bench.hpcg_flops_per_iter(192, 192, 192, 4)
    assert f == expect
    assert f / 1e9 == pytest.approx(2.6203, abs=5e-4)


def test_byte_model_per_row():
    # FP64: 16 + 88 on the finest level, 2 x 48 + 9 + 2 per level but the
    # coarsest, 48 on the coarsest: 226.14 B/row at 192^3 (1.60 GB)
    n0 = 192 ** 3
    b = bench.algorithmic_bytes_per_iter(192, 192, 192, 4)
    sz = [n for n, _ in bench.level_sizes(192, 192, 192, 4)]
    assert b == 104 * n0 + sum(107 * sz[l] for l in range(3)) + 48 * sz[3]
    assert b / n0 == pytest.approx(226.14, abs=0.01)
    # one level: only the coarsest-level smoother application
    assert bench.algorithmic_bytes_per_iter(8, 8, 8, 1) == (104 + 48) * 512
    # FP32 preconditioner halves its terms; the CG passes read the FP32 z
    bm = bench.algorithmic_bytes_per_iter(192, 192, 192, 4, "mixed")
    assert bm == 100 * n0 + sum(53.5 * sz[l] for l in range(3)) + 24 * sz[3]
    # kappa: the FP64 SpMV reads it (+8), the FP32 smoother its inverse diagonal (+4 per application)
    bk = bench.algorithmic_bytes_per_iter(96, 96, 96, 4, "mixed", kappa=True)
    bm96 = bench.algorithmic_bytes_per_iter(96, 96, 96, 4, "mixed")
    sz96 = [n for n, _ in bench.level_sizes(96, 96, 96, 4)]
    assert bk - bm96 == 8 * sz96[0] + sum(2 * 4 * sz96[l] for l in range(3)) + 4 * sz96[3]


def test_whole_solve_roofline_and_job_value():
    r = bench.whole_solve_roofline(6.0e9, 1.0, 6000.0)
    assert r["gbs"] == pytest.approx(6000.0) and r["frac"] == pytest.approx(1.0)
    assert bench.whole_job_gflops(4, 2.0e9, 10.0) == pytest.approx(800.0)


def test_both_arms_report_the_same_metric_and_config(capsys, monkeypatch):
    """The reference arm (the CPU oracle) prints the GPU arm's metric, unit,
    direction and config, so that their values can be divided; here on a
    small grid so that it runs in a second."""
    import json

    class A:
        steps, warmup, gpus = 1, 0, 1
    monkeypatch.setattr(bench, "NX", 16)
    monkeypatch.setattr(bench, "NY", 16)
    monkeypatch.setattr(bench, "NZ", 16)
    assert bench.run_reference(A()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["config"] == bench.bench_config(1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
