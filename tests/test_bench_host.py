"""Host-side arithmetic of bench.py (no GPU): the step slicing, the
stratified CPU sample and the roofline figures of the JSON line."""
import numpy as np

import bench


def test_slice_attempts_rounds_up_to_whole_groups():
    assert bench.slice_attempts(1400, 20, 8) == 72     # ceil(1400 / 20) = 70 -> 72
    assert bench.slice_attempts(1400, 1, 8) == 1400
    assert bench.slice_attempts(1, 20, 8) == 8
    assert bench.slice_attempts(0, 5, 8) == 8          # at least one group


def test_stratified_cells_cover_the_step_quantiles():
    cells, steps = bench.stratified_cells(64)
    assert len(cells) == 64 and len(set(cells)) == 64
    assert all(c % 128 == 0 and 0 <= c < 16384 for c in cells)
    s = np.asarray(steps)
    assert np.all(np.diff(s) >= 0)                     # ordered by the oracle's step count
    assert s[0] < np.median(s) < s[-1]


def _fake(kind_n=10, ms=100.0):
    info = {"n_jac_terms": 39398, "nnz_J": 18080, "lu_flops": 22600000, "rhs_flops": 56204,
            "lu_packed": 130304, "n_s": 470}
    stats = {"jac_evals": np.full(1000, 20.0), "newton_iters": np.full(1000, 200.0)}
    peaks = {"fp32_tflops": 80.0, "fp64_tflops": 1.25, "hbm_gbs": 6800.0, "hbm_source": "test",
             "alu_source": "test"}
    return info, stats, peaks, kind_n, ms


def test_refresh_roofline_arithmetic(monkeypatch):
    info, s, peaks, n, ms = _fake()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "h0")
    monkeypatch.setattr(bench, "TRAFFIC", {("refresh", "mixed", "h0"): 5.0e6})
    r = bench.roofline(info, s, "refresh", "mixed", ms, n, peaks)
    unit = 2 * 39398 + 2 * 18080 + 22600000
    per_launch = 20.0 * 1000 / n
    achieved = unit * per_launch / (ms * 1e-3 / n) / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert np.isclose(r["achieved"], achieved) and np.isclose(r["frac"], achieved / 80.0)
    assert np.isclose(r["traffic"], 5.0e6 * per_launch)
    # a kernel source the counters were not taken on reports no traffic
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "h1")
    assert bench.roofline(info, s, "refresh", "mixed", ms, n, peaks)["traffic"] is None


def test_solve_roofline_is_bandwidth():
    info, s, peaks, n, ms = _fake()
    r = bench.roofline(info, s, "solve", "mixed", ms, n, peaks)
    unit = 4 * 130304 + 8 * 6 * 470
    per_launch = 200.0 * 1000 / n
    achieved = unit * per_launch / (ms * 1e-3 / n) / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert np.isclose(r["achieved"], achieved) and np.isclose(r["frac"], achieved / 6800.0)
    assert bench.roofline(info, s, "refresh", "mixed", ms, 0, peaks) is None
