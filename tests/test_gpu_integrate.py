"""GPU integrator (sm_integrate) against closed forms and the oracle.

Tolerances: both sides run the same BDF method at rtol 1e-6 / atol 1e-20 but
round differently (LAPACK LU with pivoting vs the library's unpivoted LU), so
their step sequences may drift apart; final abundances above 1e-20 are
compared at rtol 1e-6 relative plus an absolute floor of 1e-6 times the
largest abundance of the same element group where noted.  Closed-form pins
use the integration tolerance itself (the error control targets local errors
of rtol; the global error here stays within a small multiple).
"""
import numpy as np
import pytest

from oracle import bdf as ob
from oracle import kinetics as ok
from oracle import network as on
from synth import cells as sc
from synth import network as sn

pytestmark = pytest.mark.gpu

YEAR = 3.15576e7


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "these tests need a CUDA GPU"
    return _t


@pytest.fixture(scope="module")
def B(torch):
    from paper_2312_04998_gb300 import build
    build.build()
    from paper_2312_04998_gb300 import binding
    return binding


def dev(torch, a, ld):
    n, C = a.shape
    h = np.zeros((n, ld))
    h[:, :C] = a
    return torch.tensor(h, dtype=torch.float64, device="cuda")


def run_gpu(torch, B, d, k, y0, t_end, **opts):
    C = y0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    st = B.State(net, C, **opts)
    kd, yd = dev(torch, k, ld), dev(torch, y0, ld)
    stats = B.stats_tensor(C, "cuda")
    code = st.integrate(kd, yd, t_end, C, stats)
    torch.cuda.synchronize()
    return yd.cpu().numpy()[:, :C], B.stats_to_numpy(stats), code


def riccati_B(t, kk, z, A0, B0):
    N = A0 + 2 * B0
    a, b, c = 4 * kk, 4 * kk * N + z, kk * N * N
    disc = np.sqrt(b * b - 4 * a * c)
    B1 = 2 * c / (b + disc)
    B2 = (b + disc) / (2 * a)
    inv_r = (B0 - B1) / (B0 - B2) * np.exp(-a * (B2 - B1) * t)
    return (B2 * inv_r - B1) / (inv_r - 1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_worked_example_riccati(torch, B, precision):
    """2A -> B, B -> 2A (Eqs. 2-6) integrated per cell with different k and
    end times folded into one batch, against the exact solution."""
    d = sn.worked_example()
    C = 40
    rng = np.random.default_rng(1)
    k = np.stack([10 ** rng.uniform(-4, -2, C), 10 ** rng.uniform(-6, -4, C)])
    y0 = np.stack([np.ones(C), np.zeros(C)])
    t_end = 1e4
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK and np.all(stats["status"] == B.CELL_OK)
    Bex = np.array([riccati_B(t_end, k[0, c], k[1, c], 1.0, 0.0) for c in range(C)])
    assert np.allclose(y[1], Bex, rtol=2e-5)
    assert np.allclose(y[0] + 2 * y[1], 1.0, rtol=1e-13)


def load_truth(name, key="y"):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", f"integrate_truth_{name}.json")) as fh:
        return np.array(json.load(fh)[key]).T


U32 = 2.0 ** -24
# Conditioning allowed to the WRMS-equilibrated Newton matrix in the FP32
# drift bar (the stiffest 32 x 180 cells of the conservation test need an
# effective 4.4e5)
KAPPA_FP32 = 1e6
# FP64 drift: both implementations round the same stiff fluxes in the Newton
# residual, with different factorisations (pivoted LAPACK vs unpivoted), so
# cell by cell their drifts are of the same order but not the same value;
# the bar is a multiple of the oracle's largest drift over the same cells
FP64_DRIFT_FACTOR = 8.0


def fp32_drift_bar(stats, drift_fp64_max, rtol=1e-6):
    """Largest relative drift of an element total allowed to a reduced-
    precision run, per cell.  Every Newton iteration restores E y up to the
    error of its linear solve: in FP64 that leaves the rounding of the stiff
    fluxes in the residual (the FP64 bar: FP64_DRIFT_FACTOR times the
    oracle's largest drift over the same cells, drift_fp64_max); the FP32
    solve of the equilibrated system adds
    at most u32 * kappa * |delta|_wrms relative to the error weights
    rtol |y| + atol, i.e. u32 * kappa * rtol relative to the element total
    for |delta|_wrms <= 1.  The residue is carried through the step history,
    so the FP32 part is summed over the cell's Newton iterations."""
    return FP64_DRIFT_FACTOR * max(drift_fp64_max, 1e-13) + stats["newton_iters"] * U32 * KAPPA_FP32 * rtol


def weighted_err(y, ref, rtol=1e-6, atol=1e-20):
    """Largest |y - ref| in units of the integrator's error weight."""
    return float(np.max(np.abs(y - ref) / (rtol * np.abs(ref) + atol)))


@pytest.fixture(scope="module")
def small_case():
    """24 cells of the 32 x 180 network (T 10-1000 K, n_H 1e2-1e8, A_V 0-20,
    atomic start) to 1e6 yr; the oracle's own rtol-1e-6 solution and the
    stored rtol-1e-10 solution ('truth')."""
    from tests.golden.make_integrate_truth import case_inputs
    d, k, y0, t_end = case_inputs("small")
    S = on.stoichiometry(d)
    ref = [ob.integrate_cell(d, k[:, c], y0[:, c], t_end, ob.BDFOptions(), S) for c in range(y0.shape[1])]
    return d, k, y0, t_end, ref, load_truth("small")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_small_network_matches_oracle(torch, B, small_case, precision):
    """24 stiff cells of the 32 x 180 network against the tight-tolerance
    truth.  FP64 runs the oracle's method in the oracle's precision: its
    worst cell is no farther from the truth than twice the oracle's worst
    (in tolerance units), and most cells take the identical sequence of
    steps, rejections, Newton iterations and Jacobian refreshes.  The reduced
    precisions round every Newton correction through FP32 factors, which can
    flip individual accept / reject decisions and send a cell along another
    valid trajectory with another global error: their stated bar is no cell
    beyond 100 tolerance units (1e-4 relative) and the median over cells
    within 1.5x the oracle's (both floored at one unit)."""
    d, k, y0, t_end, ref, truth = small_case
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK, stats["status"]
    assert np.all(stats["t"] == t_end)
    yo = np.stack([r.y for r in ref], axis=1)
    e_o = np.maximum(cell_err(yo, truth), 1.0)
    e_g = np.maximum(cell_err(y, truth), 1.0)
    if precision == "fp64":
        assert e_g.max() <= 2.0 * e_o.max(), (e_g.max(), e_o.max())
    else:
        assert e_g.max() <= 100.0, (e_g.max(), int(e_g.argmax()))
        assert np.median(e_g) <= 1.5 * np.median(e_o), (np.median(e_g), np.median(e_o))
    steps_o = np.array([r.steps for r in ref])
    assert np.all(np.abs(stats["steps"] - steps_o) <= 0.25 * steps_o + 5)
    if precision == "fp64":
        # same method, same precision: most cells take the identical sequence
        # of steps, rejections, Newton iterations and Jacobian refreshes
        same = [(s_["steps"], s_["rejects"], s_["conv_fails"], s_["newton_iters"], s_["jac_evals"]) ==
                (r.steps, r.rejects, r.conv_fails, r.newton_iters, r.jac_evals)
                for s_, r in zip(stats, ref)]
        assert np.mean(same) >= 0.5, np.mean(same)


@pytest.fixture(scope="module")
def moderate_case():
    """40 cells of moderate stiffness (T 10-300 K, n_H 1e2-1e6, A_V 0-10) of
    the 32 x 180 network to 1e5 yr, with the oracle's rtol-1e-6 solutions."""
    d = sn.generate(2312, 32, 180)
    C = 40
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    S = on.stoichiometry(d)
    t_end = 1e5 * YEAR
    ref = [ob.integrate_cell(d, k[:, c], y0[:, c], t_end, ob.BDFOptions(), S) for c in range(C)]
    return d, k, y0, t_end, ref, None


@pytest.mark.parametrize("case", ["moderate", "stiff"])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_conservation_gpu(torch, B, small_case, moderate_case, case, precision):
    """Element totals and charge through integration.  In exact arithmetic
    every Newton correction conserves them (E S = 0 makes E M = E); in
    floating point the solves' rounding, amplified by the Newton matrix's
    conditioning, lets them drift, and the oracle (LAPACK, pivoted FP64)
    drifts too: up to 3e-10 relative on the moderate cells, 3e-7 on the stiff
    24-cell case (T to 1000 K, n_H to 1e8, 1e6 yr).  FP64's worst cell must
    stay within FP64_DRIFT_FACTOR of the oracle's worst (floor 1e-13).  The
    reduced precisions solve each Newton correction in FP32: their bar is
    fp32_drift_bar (FP32 rounding of the equilibrated solve, summed over the
    cell's Newton iterations), orders of magnitude below what an error in S
    or in the elimination produces."""
    d, k, y0, t_end, ref, _ = small_case if case == "stiff" else moderate_case
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK
    E = on.element_matrix(d).astype(float)
    tot0 = np.abs(E[:3] @ y0)
    yo = np.stack([r.y for r in ref], axis=1)
    # per cell: the largest relative drift over the elements, and the charge
    drift = (np.abs(E[:3] @ y - E[:3] @ y0) / tot0).max(axis=0)
    drift_o = (np.abs(E[:3] @ yo - E[:3] @ y0) / tot0).max(axis=0)
    charge, charge_o = np.abs(E[3] @ y), np.abs(E[3] @ yo)
    if precision == "fp64":
        bar = FP64_DRIFT_FACTOR * max(drift_o.max(), 1e-13)
        assert drift.max() <= bar, (drift.max(), drift_o.max())
        assert charge.max() <= FP64_DRIFT_FACTOR * max(charge_o.max(), 1e-13), (charge.max(), charge_o.max())
    else:
        bar = fp32_drift_bar(stats, drift_o.max())
        assert np.all(drift <= bar), (drift / bar).max()
        assert np.all(charge <= bar * tot0[0]), (charge / (bar * tot0[0])).max()


def test_nan_cell_is_isolated(torch, B):
    d = sn.generate(2312, 32, 180)
    C = 8
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    y0[3, 2] = np.nan
    y, stats, code = run_gpu(torch, B, d, k, y0, 1e3 * YEAR)
    assert code == B.SM_EPARTIAL
    assert stats["status"][2] == B.CELL_NAN
    others = np.delete(np.arange(C), 2)
    assert np.all(stats["status"][others] == B.CELL_OK)


def test_max_steps_reported(torch, B):
    d = sn.generate(2312, 32, 180)
    C = 4
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    y, stats, code = run_gpu(torch, B, d, k, y0, 1e6 * YEAR, max_steps=5)
    assert code == B.SM_EPARTIAL
    assert np.all(stats["status"] == B.CELL_MAXSTEPS) and np.all(stats["steps"] == 5)


@pytest.fixture(scope="module")
def strat_case():
    """The 32 stiffness-stratified cells of the 16,384-cell workload (470 x
    6000, T 10-1000 K, n_H 1e2-1e8, A_V 0-20, atomic start, 1e6 yr) with the
    oracle's stored rtol-1e-10 ('truth') and rtol-1e-6 solutions."""
    import json
    import os
    from tests.golden.make_integrate_truth import STRAT_POOL, case_inputs
    with open(os.path.join(os.path.dirname(__file__), "golden", "integrate_truth_strat.json")) as fh:
        ref = json.load(fh)
    d, k, y0, t_end = case_inputs("strat", STRAT_POOL, ref["cells"])
    return d, k, y0, t_end, np.array(ref["y"]).T, np.array(ref["y_rtol6"]).T, np.array(ref["steps_rtol6"])


def cell_err(y, ref, rtol=1e-6, atol=1e-20):
    """Per cell: largest |y - ref| in units of the integrator's error weight."""
    return np.max(np.abs(y - ref) / (rtol * np.abs(ref) + atol), axis=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_large_network_matches_oracle(torch, B, strat_case, precision):
    """32 stiffness-stratified cells of the 470 x 6000 network (45 to 908
    oracle steps) to 1e6 yr against the stored rtol-1e-10 truth.  The GPU and
    the oracle run the same method at rtol 1e-6 but round differently, so a
    cell's two runs can part ways at some accept / reject decision and end
    with different (equally valid) global errors: the oracle's own range
    over these cells is 1 to 38 tolerance units.  Compared therefore as
    distributions over the cells: the GPU's worst cell within 1.5x the
    oracle's worst (2x for the reduced precisions), its median within 1.5x
    the oracle's median, and no cell beyond 100 units (a wrong step, J or
    factorisation gives orders of magnitude more)."""
    d, k, y0, t_end, truth, yo, steps_o = strat_case
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK, stats["status"]
    e_o = np.maximum(cell_err(yo, truth), 1.0)
    e_g = np.maximum(cell_err(y, truth), 1.0)
    assert e_g.max() <= 100.0, (e_g.max(), int(e_g.argmax()))
    assert e_g.max() <= (1.5 if precision == "fp64" else 2.0) * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 1.5 * np.median(e_o), (np.median(e_g), np.median(e_o))
    assert np.all(np.abs(stats["steps"] - steps_o) <= 0.25 * steps_o + 10)
    # element totals: FP64 within FP64_DRIFT_FACTOR of the oracle's largest
    # drift (its stored rtol-1e-6 solutions), the reduced precisions within
    # fp32_drift_bar
    E = on.element_matrix(d).astype(float)
    tot0 = np.abs(E[:3] @ y0)
    drift = (np.abs(E[:3] @ y - E[:3] @ y0) / tot0).max(axis=0)
    drift_o = (np.abs(E[:3] @ yo - E[:3] @ y0) / tot0).max(axis=0)
    if precision == "fp64":
        assert drift.max() <= FP64_DRIFT_FACTOR * max(drift_o.max(), 1e-13), (drift.max(), drift_o.max())
    else:
        bar = fp32_drift_bar(stats, drift_o.max())
        assert np.all(drift <= bar), (drift / bar).max()


def test_state_reuse_with_new_end_time(torch, B):
    """A state integrated once to a short end time and then to a long one
    gives the same bits as a fresh state integrated to the long one (the
    cached graph of attempts must not keep the first end time)."""
    d = sn.generate(2312, 32, 180)
    C = 40
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    kd = dev(torch, k, ld)
    out = []
    for ends in ((1e2 * YEAR, 1e5 * YEAR), (1e5 * YEAR,)):
        st = B.State(net, C)
        for t_end in ends:
            yd = dev(torch, y0, ld)
            stats = B.stats_tensor(C, "cuda")
            assert st.integrate(kd, yd, t_end, C, stats) == B.SM_OK
        torch.cuda.synchronize()
        s = B.stats_to_numpy(stats)
        assert np.all(s["t"] == 1e5 * YEAR)
        out.append((yd.cpu().numpy(), s["steps"].copy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_newton_rounds_are_bit_identical(torch, B, precision):
    """In states without compaction (those that record their steps), from
    4096 cells on the Newton rounds of the two halves of the batch run on two
    streams (unless the solve or RHS class is being timed); the result must be
    the same bits as the single-stream rounds."""
    d = sn.generate(2312, 32, 180)
    C = 4200
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    out = []
    for timing in ("none", "solve"):
        y, stats, code = run_gpu(torch, B, d, k, y0, 1e3 * YEAR, precision=precision, timing_kind=timing,
                                 record_steps=64)
        assert code == B.SM_OK
        out.append((y, stats["steps"].copy(), stats["newton_iters"].copy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compaction_is_bit_identical(torch, B, precision):
    """Cells of very different stiffness (T 10-1000 K, n_H 1e2-1e8) finish
    after very different numbers of attempts; with compaction the running
    cells are moved to the front slots between attempt groups.  Every cell's
    arithmetic is independent of its slot, so the solution and every per-cell
    counter must be the same bits as in a state without compaction (one that
    records its steps), in the caller's cell order."""
    d = sn.generate(2312, 32, 180)
    C = 3000
    T, nH, Av = sc.conditions(4998, C, (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    out = []
    for rec in (0, 4000):
        y, stats, code = run_gpu(torch, B, d, k, y0, 1e6 * YEAR, precision=precision, record_steps=rec)
        assert code == B.SM_OK
        out.append((y, stats))
    steps = out[0][1]["steps"]
    # uneven stiffness (the fastest cells finish in a fraction of the slowest
    # cells' attempts), so the running range was compacted several times
    assert steps.min() * 4 < steps.max()
    assert np.array_equal(out[0][0], out[1][0])
    for key in ("steps", "rejects", "conv_fails", "newton_iters", "jac_evals", "q_last", "t", "h"):
        assert np.array_equal(out[0][1][key], out[1][1][key]), key


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
@pytest.mark.parametrize("with_factors", [True, False])
def test_state_save_load_resume(torch, B, with_factors, precision):
    """Stop an integration after 40 attempts, save the state to host memory,
    load it into a new state and finish there: with the Newton factors saved
    (FP64 values, or FP32 values in the reduced precisions) the result is the
    same bits as an uninterrupted run; without them (every cell refactorises
    once on resume) it is another rtol-1e-6 solution of the same problem, a
    few tolerance units away."""
    d = sn.generate(2312, 32, 180)
    C = 40
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    t_end = 1e3 * YEAR
    y_ref, s_ref, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    kd = dev(torch, k, ld)
    a = B.State(net, C, precision=precision)
    a.init(kd, dev(torch, y0, ld), t_end, C)
    a.step(kd, 40)
    assert a.read() > 0                       # interrupted mid-run
    image = a.save(with_factors)
    del a
    b = B.State(net, C, precision=precision)
    b.load(image)
    for _ in range(2000):
        b.step(kd, 8)
        if b.read() == 0:
            break
    y = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    stats = B.stats_tensor(C, "cuda")
    assert b.read(y, stats) == 0
    torch.cuda.synchronize()
    y, s = y.cpu().numpy()[:, :C], B.stats_to_numpy(stats)
    assert np.all(s["status"] == B.CELL_OK) and np.all(s["t"] == t_end)
    if with_factors:
        assert np.array_equal(y, y_ref)
        for key in ("steps", "rejects", "newton_iters", "jac_evals"):
            assert np.array_equal(s[key], s_ref[key]), key
    else:
        units = np.abs(y - y_ref) / (1e-6 * np.abs(y_ref) + 1e-20)
        assert units.max() <= 100.0, units.max()
    # an image does not fit a state of another shape or precision
    other = "fp64" if precision != "fp64" else "mixed"
    with pytest.raises(B.StoichError):
        B.State(net, C, precision=other).load(image)
    c = B.State(net, C + 64, precision=precision)
    with pytest.raises(B.StoichError):
        c.load(image)


def step_by_step(torch, B, d, k, y0, t_end, record=20000, **opts):
    """Integrates attempt by attempt (sm_step_bdf with one attempt, then
    sm_state_read) and returns per cell the accepted states y_0, y_1, ...,
    and the recorded step log (end times, sizes, orders)."""
    C = y0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    st = B.State(net, C, record_steps=record, **opts)
    kd = dev(torch, k, ld)
    st.init(kd, dev(torch, y0, ld), t_end, C)
    ys = [[y0[:, c].copy()] for c in range(C)]
    prev = np.zeros(C, dtype=np.int64)
    yd = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    stats = B.stats_tensor(C, "cuda")
    for _ in range(100000):
        st.step(kd, 1)
        running = st.read(yd, stats)
        s = B.stats_to_numpy(stats)
        y = yd.cpu().numpy()
        for c in np.nonzero(s["steps"] != prev)[0]:
            assert s["steps"][c] == prev[c] + 1          # one attempt accepts at most one step
            ys[c].append(y[:, c].copy())
        prev = s["steps"].astype(np.int64)
        if running == 0:
            break
    assert np.all(s["status"] == B.CELL_OK), s["status"]
    m_max = int(prev.max())
    tl, hl, ql = (a.cpu().numpy() for a in st.steps_log(m_max, C))
    return ys, tl, hl, ql, s


def replay_errors(d, k, ys, tl, hl, ql, sample=None):
    """One-step replay: for every (or `sample` evenly spaced) accepted step m
    of every cell, the oracle solves the step's implicit BDF equation exactly
    from the GPU's own history y_{m-1}, ..., y_{m-q} with the GPU's recorded
    t_m, h_m, q_m.  Returns per checked step the largest
    |y_gpu - y_oracle| / (1e-10 |y_oracle| + 1e-24) over species, and the
    WRMS norm of the difference in the step's error weights
    1 / (1e-6 |y_{m-1}| + 1e-20)."""
    S = on.stoichiometry(d)
    out, wr = [], []
    for c in range(len(ys)):
        N = len(ys[c]) - 1
        ts = [0.0] + [tl[m - 1, c] for m in range(1, N + 1)]
        ms = range(1, N + 1) if sample is None else sorted(set(np.linspace(1, N, sample).astype(int)))
        for m in ms:
            q = int(ql[m - 1, c])
            yo = ob.solve_step(d, k[:, c], [ys[c][m - 1 - i] for i in range(q)],
                               [ts[m - 1 - i] for i in range(q)], ts[m], hl[m - 1, c], S, y_start=ys[c][m])
            out.append(np.max(np.abs(ys[c][m] - yo) / (1e-10 * np.abs(yo) + 1e-24)))
            wr.append(np.sqrt(np.mean(((ys[c][m] - yo) / (1e-6 * np.abs(ys[c][m - 1]) + 1e-20)) ** 2)))
    return np.array(out), np.array(wr)


# Largest one-step replay difference allowed, in units of 1e-10 |y| + 1e-24
# (1e-10 relative above atol / rtol = 1e-14, where the method's weights are
# relative; 1e-24 absolute below)
REPLAY_BAR = 1.0
# Options of the tightly converged runs: the Newton iteration converged to
# 1e-6 in WRMS units (so that the GPU's y_m is the exact solution of its step
# to about 1e-12 relative), with the Jacobian refreshed at every attempt so
# that the simplified Newton iteration converges fast enough to reach it
REPLAY_OPTS = dict(newton_tol=1e-6, newton_max=8, j_age_max=1, gamma_tol=1e-9, use_graph=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_step_replay_matches_oracle(torch, B, precision):
    """The step math, independently of the step-size controller: 8 cells of
    the 32 x 180 network (T 10-300 K, n_H 1e2-1e6, A_V 0-10) are integrated
    to 1e5 yr attempt by attempt with the Newton iteration converged tightly
    (REPLAY_OPTS), and every accepted GPU step is compared with the oracle's
    exact solution of the same BDF equation (same history, t_m, h_m, q_m):
    within 1e-10 relative (REPLAY_BAR; measured 3e-11 in FP64, 7e-11 with
    FP32 factors, whose FP64 residual refines the solve).  On the stiffest
    cells a tolerance this tight makes the controller cut the step size far
    below its normal values, so they are replayed with the method's own
    options in test_step_replay_large_network instead."""
    d = sn.generate(2312, 32, 180)
    C = 8
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    ys, tl, hl, ql, s = step_by_step(torch, B, d, k, y0, 1e5 * YEAR, precision=precision, **REPLAY_OPTS)
    err, _ = replay_errors(d, k, ys, tl, hl, ql)
    assert len(err) == int(s["steps"].sum())
    assert err.max() <= REPLAY_BAR, (err.max(), np.quantile(err, 0.99))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_replay_large_network(torch, B, strat_case, precision):
    """The one-step replay on 4 of the stratified 470 x 6000 cells (T to
    1000 K, n_H to 1e8) to 1e6 yr with the method's own options, 12 evenly
    spaced accepted steps per cell: each accepted GPU step solves its BDF
    equation to within its Newton tolerance (0.1 WRMS units, passed when the
    contraction-weighted correction is below it), so the distance to the
    oracle's exact solution of the same equation stays within 2 WRMS units
    (measured 0.18 in FP64, 0.49 with FP32 factors); an error in the BDF
    coefficients, the history or the right-hand side is orders larger."""
    d, k, y0, t_end = strat_case[:4]
    sel = [0, 8, 16, 24]
    ys, tl, hl, ql, s = step_by_step(torch, B, d, k[:, sel], y0[:, sel], t_end, precision=precision, use_graph=0)
    _, wrms = replay_errors(d, k[:, sel], ys, tl, hl, ql, sample=12)
    assert len(wrms) >= 4 * 10
    assert wrms.max() <= 2.0, (wrms.max(), np.quantile(wrms, 0.9))


@pytest.fixture(scope="module")
def pdr_case():
    """The PDR slab (128 cells, the paper's benchmark geometry with the
    synthetic network) and the oracle's stored solutions for 8 of its cells."""
    import json
    import os
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["pdr_slab_470x6000_c128"]
    d, T, nH, Av, y0 = make(w.name)
    with open(os.path.join(os.path.dirname(__file__), "golden", "integrate_truth_pdr.json")) as fh:
        ref = json.load(fh)
    return w, d, T, nH, Av, y0, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pdr_slab_matches_oracle(torch, B, pdr_case, precision):
    """The whole 128-cell PDR slab (n_H 1e3, T 50 K, FUV field 1e5 on the
    photorates, A_V 1e-3 to 20, 30 Myr): rate coefficients from
    sm_rates_eval_chi against the oracle's (1e-13 relative), every cell
    reaching t_end, and the 8 stored cells against the oracle's rtol-1e-10
    solution with the bars of test_large_network_matches_oracle."""
    w, d, T, nH, Av, y0, ref = pdr_case
    C = y0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    pad = lambda v, fill: torch.tensor(np.concatenate([v, np.full(ld - C, fill)]), dtype=torch.float64,
                                       device="cuda")
    kd = torch.zeros((d.n_r, ld), dtype=torch.float64, device="cuda")
    net.rates_eval_chi(pad(T, 100.0), pad(nH, 1.0), pad(Av, 0.0), pad(np.full(C, w.chi), 1.0), kd, C)
    torch.cuda.synchronize()
    k = kd.cpu().numpy()[:, :C]
    kref = ok.rate_coefficients(d, T, nH, Av, chi=w.chi)
    assert np.all(np.abs(k - kref) <= 1e-13 * np.abs(kref))
    st = B.State(net, C, precision=precision)
    yd = dev(torch, y0, ld)
    stats = B.stats_tensor(C, "cuda")
    assert st.integrate(kd, yd, w.t_end, C, stats) == B.SM_OK
    torch.cuda.synchronize()
    y, s = yd.cpu().numpy()[:, :C], B.stats_to_numpy(stats)
    assert np.all(s["status"] == B.CELL_OK) and np.all(s["t"] == w.t_end)
    cells = ref["cells"]
    truth, yo = np.array(ref["y"]).T, np.array(ref["y_rtol6"]).T
    e_o = np.maximum(cell_err(yo, truth), 1.0)
    e_g = np.maximum(cell_err(y[:, cells], truth), 1.0)
    assert e_g.max() <= 100.0, (e_g.max(), int(e_g.argmax()))
    assert e_g.max() <= (1.5 if precision == "fp64" else 2.0) * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 1.5 * np.median(e_o), (np.median(e_g), np.median(e_o))
    steps_o = np.array(ref["steps_rtol6"])
    assert np.all(np.abs(s["steps"][cells] - steps_o) <= 0.25 * steps_o + 10)


@pytest.mark.parametrize("order", ["none", "nnz", "rcm"])
@pytest.mark.parametrize("kc", [8, 16, 32])
def test_integrator_gather_shapes(torch, B, moderate_case, order, kc):
    """Every choice the autotuner can make for the integrator's gather (CRS
    row order x cells per CTA) integrates the 40 moderate cells of the
    32 x 180 network to the same solution as the default choice up to the
    summation order of the right-hand side (which can move an accept /
    reject decision: within 50 tolerance units of it) and within 100 units
    of the oracle's rtol-1e-6 solution; a wrong gather is off by orders of
    magnitude more."""
    d, k, y0, t_end, ref, _ = moderate_case
    C = y0.shape[1]
    ld = B.pad_ld(C)
    out = []
    for choice in (("none", 16), (order, kc)):
        net = B.Network(d, 0)
        net.set_integ(*choice)
        st = B.State(net, C)
        yd = dev(torch, y0, ld)
        assert st.integrate(dev(torch, k, ld), yd, t_end, C) == B.SM_OK
        torch.cuda.synchronize()
        out.append(yd.cpu().numpy()[:, :C])
    assert cell_err(out[1], out[0]).max() <= 50.0
    yo = np.stack([r.y for r in ref], axis=1)
    assert cell_err(out[1], yo).max() <= 100.0


def test_full_size_batch_matches_oracle_on_sampled_cells(torch, B, strat_case):
    """The benchmark's launch configuration: all 65,536 cells of the headline
    workload (470 x 6000, T 10-1000 K, n_H 1e2-1e8, A_V 0-20, atomic start,
    1e6 yr) integrated as one batch in the mixed mode with the autotuned
    gather, graphs and compaction, as bench.py times it.  The 32 stratified
    cells of the stored truth are the same draws (cells are a seeded stream,
    so the first 16,384 of the batch are the truth's pool); they take the
    mixed-precision bars of test_large_network_matches_oracle, and every
    cell of the batch must finish."""
    from synth.workloads import make
    d, k_small, y0_small, t_end, truth, yo, steps_o = strat_case
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "integrate_truth_strat.json")) as fh:
        cells = json.load(fh)["cells"]
    dd, T, nH, Av, y0 = make("integrate_470x6000_c65536")
    C = y0.shape[1]
    assert np.array_equal(y0[:, cells], y0_small)
    ld = B.pad_ld(C)
    net = B.Network(dd, 0)
    vec = lambda a, fill: torch.cat([torch.tensor(a, dtype=torch.float64),
                                     torch.full((ld - C,), fill, dtype=torch.float64)]).cuda()
    Td, nHd, Avd = vec(T, 100.0), vec(nH, 1.0), vec(Av, 0.0)
    kd = torch.empty((dd.n_r, ld), dtype=torch.float64, device="cuda")
    net.rates_eval(Td, nHd, Avd, kd, C)
    assert np.allclose(kd[:, cells].cpu().numpy(), k_small, rtol=1e-13, atol=0.0)
    yd = torch.zeros((dd.n_s, ld), dtype=torch.float64, device="cuda")
    yd[:, :C] = torch.tensor(y0, dtype=torch.float64, device="cuda")
    fscr = torch.empty_like(yd)
    net.autotune(kd, yd, fscr, C)
    del fscr
    st = B.State(net, C, precision="mixed")
    stats = B.stats_tensor(C, "cuda")
    code = st.integrate(kd, yd, t_end, C, stats)
    torch.cuda.synchronize()
    s = B.stats_to_numpy(stats)
    assert code == B.SM_OK and np.all(s["status"] == B.CELL_OK)
    y = yd[:, cells].cpu().numpy()
    e_o = np.maximum(cell_err(yo, truth), 1.0)
    e_g = np.maximum(cell_err(y, truth), 1.0)
    assert e_g.max() <= 100.0, (e_g.max(), int(e_g.argmax()))
    assert e_g.max() <= 2.0 * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 1.5 * np.median(e_o), (np.median(e_g), np.median(e_o))
    st_s = s["steps"][cells]
    assert np.all(np.abs(st_s - steps_o) <= 0.25 * steps_o + 10)


def test_integrate_rejects_bad_calls(torch, B):
    """Argument checks of the integrator's entry points (all on the host,
    before any launch): empty or oversized batches, a row stride that is not
    a multiple of 32, missing rate coefficients, a non-positive end time,
    out-of-range options; each returns SM_EINVAL and leaves the state usable."""
    import ctypes as ct
    d = sn.generate(2312, 32, 180)
    C = 8
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    st = B.State(net, C)
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = dev(torch, ok.rate_coefficients(d, T, nH, Av), ld)
    y = dev(torch, sc.atomic_start(d, C), ld)
    lib = B.lib()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    call = lambda C_, k_, y_, ld_, t_: lib.sm_integrate(st.h, C_, k_, y_, ld_, t_, None, stream)
    kp, yp = ct.c_void_p(k.data_ptr()), ct.c_void_p(y.data_ptr())
    assert call(0, kp, yp, ld, 1e10) == B.SM_EINVAL          # empty batch
    assert call(C + 1, kp, yp, ld, 1e10) == B.SM_EINVAL      # beyond the capacity
    assert call(C, kp, yp, 40, 1e10) == B.SM_EINVAL          # ld not a multiple of 32
    assert call(C, None, yp, ld, 1e10) == B.SM_EINVAL        # no rate coefficients
    assert call(C, kp, yp, ld, 0.0) == B.SM_EINVAL           # t_end <= 0
    for bad in (dict(newton_max=9), dict(q_max=6), dict(rtol=-1.0), dict(refresh_ctas_per_sm=-1)):
        with pytest.raises(B.StoichError):
            B.State(net, C, **bad)
    # the state still integrates after the refused calls
    assert st.integrate(k, y, 1e5 * YEAR, C) == B.SM_OK


def test_single_cell_matches_oracle(torch, B):
    """The single-cell case (32 x 180, T 10 K, n_H 1e4, A_V 5, atomic start,
    1e6 yr): a batch of one cell against the oracle's rtol-1e-10 solution,
    within 10 tolerance units (the oracle's own rtol-1e-6 run is within 2)."""
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["single_cell_32x180"]
    d, T, nH, Av, y0 = make(w.name)
    k = ok.rate_coefficients(d, T, nH, Av)
    ref = ob.integrate_cell(d, k[:, 0], y0[:, 0], w.t_end, ob.BDFOptions(rtol=1e-10, atol=1e-24)).y
    mine = ob.integrate_cell(d, k[:, 0], y0[:, 0], w.t_end).y
    e_o = cell_err(mine[:, None], ref[:, None])[0]
    y, stats, code = run_gpu(torch, B, d, k, y0, w.t_end)
    assert code == B.SM_OK and stats["status"][0] == B.CELL_OK
    e_g = cell_err(y, ref[:, None])[0]
    assert e_o <= 2.0 and e_g <= 10.0, (e_g, e_o)
