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
    """The GPU solution is no farther from the tight-tolerance truth than twice
    the oracle's own rtol-1e-6 solution is (both run the same method at the
    same tolerance; their global errors, a few tolerance units, set the bar).
    The reduced precisions (FP32 factors, with TF32 trailing updates in the
    tf32 mode) take the mixed bar."""
    d, k, y0, t_end, ref, truth = small_case
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK, stats["status"]
    assert np.all(stats["t"] == t_end)
    yo = np.stack([r.y for r in ref], axis=1)
    e_o = weighted_err(yo, truth)
    e_g = weighted_err(y, truth)
    # FP64 runs the oracle's method in the oracle's precision: its distance to
    # the truth is bounded by twice the oracle's own.  The mixed path rounds
    # every Newton correction to FP32, which can flip individual accept /
    # reject decisions and so take a different (equally valid) trajectory;
    # its stated bar is four times the oracle's global error.
    factor = 2.0 if precision == "fp64" else 4.0
    assert e_g <= factor * max(e_o, 1.0), (e_g, e_o)
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
    drifts too: up to 3e-10 relative on the moderate cells, 7e-7 on the stiff
    24-cell case (T to 1000 K, n_H to 1e8, 1e6 yr).  FP64 must stay within 4x
    the oracle's drift on the same cells, per element (floor 1e-13).  Mixed
    precision rounds each Newton correction to FP32 (relative error ~1e-7,
    over hundreds of steps): bar 1e-4 relative, still orders of magnitude
    below what an error in S or in the elimination produces."""
    d, k, y0, t_end, ref, _ = small_case if case == "stiff" else moderate_case
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK
    E = on.element_matrix(d).astype(float)
    tot0 = np.abs(E[:3] @ y0)
    drift = (np.abs(E[:3] @ y - E[:3] @ y0) / tot0).max(axis=1)
    charge = np.abs(E[3] @ y).max()
    if precision == "fp64":
        yo = np.stack([r.y for r in ref], axis=1)
        drift_o = (np.abs(E[:3] @ yo - E[:3] @ y0) / tot0).max(axis=1)
        charge_o = np.abs(E[3] @ yo).max()
        assert np.all(drift <= 4.0 * np.maximum(drift_o, 1e-13)), (drift, drift_o)
        assert charge <= 4.0 * max(charge_o, 1e-13), (charge, charge_o)
    else:
        assert np.all(drift <= 1e-4), drift
        assert charge <= 1e-4 * tot0[0].max(), charge


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


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_large_network_matches_oracle(torch, B, precision):
    """4 cells of the 470 x 6000 network to 1e6 yr against the stored
    rtol-1e-10 truth; the bar is the oracle's own rtol-1e-6 distance to it
    (stored by the same script), doubled for FP64 and quadrupled for mixed."""
    from tests.golden.make_integrate_truth import case_inputs
    d, k, y0, t_end = case_inputs("large")
    truth = load_truth("large")
    yo = load_truth("large", "y_rtol6")
    y, stats, code = run_gpu(torch, B, d, k, y0, t_end, precision=precision)
    assert code == B.SM_OK, stats["status"]
    e_o = weighted_err(yo, truth)
    e_g = weighted_err(y, truth)
    factor = 2.0 if precision == "fp64" else 4.0
    assert e_g <= factor * max(e_o, 1.0), (e_g, e_o)
    # element totals: the same bars as the conservation test (the oracle's
    # own drift, from its stored rtol-1e-6 solution, for FP64)
    E = on.element_matrix(d).astype(float)
    tot0 = np.abs(E[:3] @ y0)
    drift = (np.abs(E[:3] @ y - E[:3] @ y0) / tot0).max(axis=1)
    if precision == "fp64":
        drift_o = (np.abs(E[:3] @ yo - E[:3] @ y0) / tot0).max(axis=1)
        assert np.all(drift <= 4.0 * np.maximum(drift_o, 1e-13)), (drift, drift_o)
    else:
        assert np.all(drift <= 1e-4), drift


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
    """From 4096 cells on, the Newton rounds of the two halves of the batch run
    on two streams (unless the solve or RHS class is being timed); the result must be
    the same bits as the single-stream rounds."""
    d = sn.generate(2312, 32, 180)
    C = 4200
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    out = []
    for timing in ("none", "solve"):
        y, stats, code = run_gpu(torch, B, d, k, y0, 1e3 * YEAR, precision=precision, timing_kind=timing)
        assert code == B.SM_OK
        out.append((y, stats["steps"].copy(), stats["newton_iters"].copy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("with_factors", [True, False])
def test_state_save_load_resume(torch, B, with_factors):
    """Stop an integration after 40 attempts, save the state to host memory,
    load it into a new state and finish there: with the Newton factors saved
    the result is the same bits as an uninterrupted run; without them (every
    cell refactorises once on resume) it is another rtol-1e-6 solution of the
    same problem, a few tolerance units away."""
    d = sn.generate(2312, 32, 180)
    C = 40
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    t_end = 1e3 * YEAR
    y_ref, s_ref, code = run_gpu(torch, B, d, k, y0, t_end)
    assert code == B.SM_OK
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    kd = dev(torch, k, ld)
    a = B.State(net, C)
    a.init(kd, dev(torch, y0, ld), t_end, C)
    a.step(kd, 40)
    assert a.read() > 0                       # interrupted mid-run
    image = a.save(with_factors)
    del a
    b = B.State(net, C)
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
    # an image does not fit a state of another shape
    c = B.State(net, C + 64)
    with pytest.raises(B.StoichError):
        c.load(image)
