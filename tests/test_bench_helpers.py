"""The bench's measurement helpers (CPU): the algorithmic bytes of a level-0 launch, the
recall rule, the order-statistic interval of a quantile, and the lookup of a profile's DRAM
traffic (valid only for the current kernel source, scaled by the query count)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_level0_bytes_counts_rows_codes_and_per_query_terms():
    # two queries: (n_dist, n_expand, n_dist_upper)
    st = np.array([[100, 10, 7], [50, 4, 3]])
    row, d, k = 32, 96, 10
    # ordered search: level-0 code rows only, plus y' (4d), the shortlist (4R) and the entry (12)
    want = (14 * 128 + 150 * row) + 2 * (4 * d + 4 * 10 + 12)
    assert bench.level0_bytes(st, row, d, k, True) == want
    # one launch for all levels: the upper evaluations' code rows too, no entry record
    want = (14 * 128 + 160 * row) + 2 * (4 * d + 4 * 10)
    assert bench.level0_bytes(st, row, d, k, False) == want
    # k > 10 widens the shortlist
    assert bench.level0_bytes(st, row, d, 100, True) - bench.level0_bytes(st, row, d, 10, True) == 2 * 4 * 90


def test_recall_counts_ties_and_empty_results():
    xb = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    xq = np.array([[0.0, 0.0], [0.5, 0.5], [1.0, 0.0]])
    gt_d = np.array([0.0, 0.5, 0.0])
    top1 = np.array([0, 2, -1])          # exact; a tie at the exact distance; nothing returned
    assert bench.recall_at_1(top1, xb, xq, gt_d) == 2 / 3


def test_quantile_interval_brackets_the_quantile():
    rng = np.random.default_rng(3)
    x = rng.exponential(size=20000)
    lo, hi = bench.quantile_ci(x, 0.99)
    q = np.quantile(x, 0.99)
    assert lo <= q <= hi
    # the interval narrows with the sample
    lo2, hi2 = bench.quantile_ci(x[:2000], 0.99)
    assert hi - lo < hi2 - lo2


def test_profiled_traffic_needs_the_current_source_and_scales_by_queries(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_hash()
    (prof / "a.md").write_text(f"workload: w1\nkernel_source_sha256_16: {h}\nqueries_per_launch: 10000\n"
                               "dram_bytes_per_level0_launch_batched_fp16_ef64: 1000000\n")
    (prof / "b.md").write_text("workload: w2\nkernel_source_sha256_16: 0000000000000000\n"
                               "dram_bytes_per_level0_launch_batched_fp16_ef64: 5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: h)
    assert bench.profiled_traffic("w1", "batched_fp16_ef64", 10000) == 1000000
    assert bench.profiled_traffic("w1", "batched_fp16_ef64", 100000) == 10000000
    assert bench.profiled_traffic("w1", "batched_fp16_ef128", 10000) is None      # another form
    assert bench.profiled_traffic("w2", "batched_fp16_ef64", 10000) is None       # another source
    assert bench.profiled_traffic("w3", "batched_fp16_ef64", 10000) is None       # another workload
