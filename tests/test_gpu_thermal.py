"""GPU integration with coupled gas temperature (sm_net_set_thermal) against
closed forms and the coupled-temperature oracle (oracle/thermal.py).

The energy equation is the reading stated in oracle/thermal.py and
include/stoich.h (the paper holds T fixed inside a chemistry step and
updates the energy outside the solver, Section 5).  Bars follow the fixed-T
integrator tests: closed forms at the integration tolerance; the oracle at
rtol 1e-10 is the truth, and the GPU's error in tolerance units is compared
with the oracle's own rtol-1e-6 solution's, as a distribution over cells
(two correct rtol-1e-6 runs that take different steps differ by their
global errors).
"""
import dataclasses
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import thermal as oth
from synth import cells as sc
from synth import network as sn
from synth import thermal as sth

pytestmark = pytest.mark.gpu

YEAR = 3.15576e7
HERE = os.path.dirname(os.path.abspath(__file__))


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
    a = np.atleast_2d(a)
    n, C = a.shape
    h = np.zeros((n, ld))
    h[:, :C] = a
    return torch.tensor(h, dtype=torch.float64, device="cuda")


def run_thermal(torch, B, d, th, nH, Av, z0, t_end, chi=None, **opts):
    C = z0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    net.set_thermal(th)
    st = B.State(net, C, **opts)
    vec = lambda a: torch.tensor(np.asarray(a, dtype=float), dtype=torch.float64, device="cuda")
    st.set_cells(vec(nH), vec(Av), vec(chi) if chi is not None else None, C)
    zd = dev(torch, z0, ld)
    stats = B.stats_tensor(C, "cuda")
    code = st.integrate(None, zd, t_end, C, stats)
    torch.cuda.synchronize()
    return zd.cpu().numpy()[:, :C], B.stats_to_numpy(stats), code


def truth(name):
    with open(os.path.join(HERE, "golden", f"integrate_truth_{name}.json")) as fh:
        return json.load(fh)


def cell_err(y, ref, rtol=1e-6, atol=1e-20):
    return np.max(np.abs(y - ref) / (rtol * np.abs(ref) + atol), axis=0)


def check_element_drift(d, th, z0, z, z_o, stats, precision):
    """Element totals (H, C, O) of the chemical rows: the coupled Newton
    correction keeps E y fixed like the fixed-T one (E S = 0 gives E u = 0
    and E z = 0 for the temperature border), so the drift bars of the
    fixed-T tests apply: FP64 within FP64_DRIFT_FACTOR of the oracle's
    largest drift (its rtol-1e-6 run, z_o), reduced precisions within
    fp32_drift_bar."""
    from oracle.network import element_matrix
    from tests.test_gpu_integrate import FP64_DRIFT_FACTOR, fp32_drift_bar
    E = element_matrix(d).astype(float)[:3]
    tot0 = np.abs(E @ z0)
    drift = (np.abs(E @ z - E @ z0) / tot0).max(axis=0)
    drift_o = (np.abs(E @ z_o - E @ z0) / tot0).max(axis=0)
    if precision == "fp64":
        assert drift.max() <= FP64_DRIFT_FACTOR * max(drift_o.max(), 1e-13), (drift.max(), drift_o.max())
    else:
        bar = fp32_drift_bar(stats, drift_o.max())
        assert np.all(drift <= bar), (drift / bar).max()


def _frozen(d):
    """Rate coefficients so small that the chemistry is frozen (the library
    requires alpha > 0): every reaction rate below 1e-250."""
    return dataclasses.replace(d, alpha=np.full_like(d.alpha, 1e-280))


def test_set_thermal_rejects_bad_slots(torch, B):
    """The slot must be a species with no atoms, no charge and no reaction;
    a thermal state has no replay (adjoint), cannot be saved and cannot skip
    its cell conditions."""
    d0 = sn.generate(2312, 32, 180)
    d = sth.with_temperature(d0)
    th = sth.thermal_params(d)
    net = B.Network(d, 0)
    with pytest.raises(B.StoichError):
        net.set_thermal(dataclasses.replace(th, t_index=d.species_index("H")))
    net.set_thermal(th)
    st_r = B.State(net, 4, record_steps=16)
    kd = torch.zeros((d.n_r, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(B.StoichError):
        st_r.replay(kd, dev(torch, np.zeros((d.n_s, 4)), 32))
    st = B.State(net, 4)
    z = dev(torch, sth.thermal_start(d, sc.atomic_start(d, 4), 50.0), 32)
    with pytest.raises(B.StoichError):
        st.integrate(None, z, 1e3 * YEAR, 4)           # no cell conditions yet
    with pytest.raises(B.StoichError):
        st.save()
    plain = B.State(B.Network(d0, 0), 4)
    v = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.StoichError):
        plain.set_cells(v, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grain_coupling_closed_form(torch, B, precision):
    """Frozen chemistry, no line cooling: T relaxes exponentially to
    T_dust + heat / (lam n_H) at the rate lam n_H / (3/2 x_tot); cells of
    different density and initial T in one batch."""
    d = _frozen(sth.with_temperature(sn.generate(2312, 32, 180)))
    th = dataclasses.replace(sth.thermal_params(d), L=np.zeros(d.n_s))
    C = 24
    nH = np.logspace(2, 6, C)
    T0 = np.linspace(10.0, 900.0, C)
    z0 = sth.thermal_start(d, sc.atomic_start(d, C), T0)
    x_tot = z0[np.arange(d.n_s) != th.t_index, 0].sum()
    tau = 1.5 * x_tot / (th.lam * nH)
    t_end = 2.0 * tau.max() / 10.0        # 0.2 (densest) to 2e3 (thinnest) relaxation times
    z, stats, code = run_thermal(torch, B, d, th, nH, np.ones(C), z0, t_end, precision=precision, rtol=1e-8)
    assert code == B.SM_OK, stats["status"]
    T_eq = th.T_dust + th.heat / (th.lam * nH)
    exact = T_eq + (T0 - T_eq) * np.exp(-t_end / tau)
    err = np.abs(z[th.t_index] - exact) / exact
    assert err.max() < 2e-7, (err.max(), int(err.argmax()))


def test_line_cooling_against_quadrature(torch, B):
    """Frozen chemistry, C+ line cooling alone: T reaches T1 at the time the
    quadrature of 3/2 x_tot exp(E/T) / (n_H x_C+ L) dT gives."""
    d = _frozen(sth.with_temperature(sn.generate(2312, 32, 180)))
    th = sth.thermal_params(d)
    c = d.species_index("C+")
    L = np.zeros(d.n_s)
    L[c] = th.L[c]
    th1 = dataclasses.replace(th, heat=0.0, lam=0.0, L=L)
    T1 = np.array([150.0, 100.0, 60.0, 40.0])
    C = len(T1)
    z0 = sth.thermal_start(d, sc.atomic_start(d, C), 200.0)
    z0[c] = 1e-4
    m = np.arange(d.n_s) != th.t_index
    x_tot, nH, E = z0[m, 0].sum(), 1e4, th.E[c]
    rate = nH * 1e-4 * L[c] / (1.5 * x_tot)
    # one end time per batch: run each target separately
    for T_target in T1:
        t1, _ = quad(lambda T: np.exp(E / T) / rate, T_target, 200.0, epsabs=0.0, epsrel=1e-12)
        z, stats, code = run_thermal(torch, B, d, th1, [nH], [1.0], z0[:, :1], t1, rtol=1e-9)
        assert code == B.SM_OK
        assert abs(z[th.t_index, 0] - T_target) <= 2e-6 * T_target, (T_target, z[th.t_index, 0])


def test_energy_invariant_without_heating_or_cooling(torch, B):
    """heat = L = lam = 0: 3/2 T x_tot stays constant while the chemistry
    changes the particle number; the GPU's drift stays within a few times the
    oracle's at the same tolerance."""
    d = sth.with_temperature(sn.generate(2312, 32, 180))
    th = dataclasses.replace(sth.thermal_params(d), heat=0.0, lam=0.0, L=np.zeros(d.n_s))
    C = 8
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    z0 = sth.thermal_start(d, sc.atomic_start(d, C), T)
    t_end = 1e6 * YEAR
    z, stats, code = run_thermal(torch, B, d, th, nH, Av, z0, t_end, rtol=1e-8)
    assert code == B.SM_OK
    m = np.arange(d.n_s) != th.t_index
    e0 = z0[th.t_index] * z0[m].sum(axis=0)
    drift = np.abs(z[th.t_index] * z[m].sum(axis=0) / e0 - 1.0)
    from oracle import bdf as ob
    ref = oth.integrate(d, th, nH, Av, 1.0, z0, t_end, ob.BDFOptions(rtol=1e-8, atol=1e-20))
    drift_o = np.array([abs(r.y[th.t_index] * r.y[m].sum() / e0[i] - 1.0) for i, r in enumerate(ref)])
    moved = np.abs(z[m].sum(axis=0) / z0[m].sum(axis=0) - 1.0)
    assert moved.max() > 0.05
    assert drift.max() <= 10.0 * max(drift_o.max(), 1e-9), (drift.max(), drift_o.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
def test_small_network_matches_oracle(torch, B, precision):
    """16 cells of the 32 x 180 network with T coupled (T 10-1000 K, n_H
    1e2-1e8) to 1e6 yr against the oracle's rtol-1e-10 truth: worst cell
    within 2x (FP64) / 3x (reduced precision) of the oracle's own rtol-1e-6
    worst, median within 2x, no cell beyond 100 units; step counts within
    25 % + 10 of the oracle's."""
    from tests.golden.make_integrate_truth import thermal_inputs
    ref = truth("thermal_small")
    d, th, nH, Av, z0 = thermal_inputs(32, 180, ref["cells"])
    z, stats, code = run_thermal(torch, B, d, th, nH, Av, z0, ref["t_end"], precision=precision)
    assert code == B.SM_OK, stats["status"]
    y10, y6 = np.array(ref["y"]).T, np.array(ref["y_rtol6"]).T
    e_g, e_o = np.maximum(cell_err(z, y10), 1.0), np.maximum(cell_err(y6, y10), 1.0)
    f = 2.0 if precision == "fp64" else 3.0
    assert e_g.max() <= 100.0 and e_g.max() <= f * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 2.0 * np.median(e_o), (np.median(e_g), np.median(e_o))
    steps_o = np.array(ref["steps_rtol6"])
    assert np.all(np.abs(stats["steps"] - steps_o) <= 0.25 * steps_o + 10), (stats["steps"], steps_o)
    # the temperature itself: within 1e-4 relative of the truth everywhere
    t = th.t_index
    assert np.all(np.abs(z[t] - y10[t]) <= 1e-4 * y10[t]), np.abs(z[t] / y10[t] - 1).max()
    check_element_drift(d, th, z0, z, y6, stats, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_network_matches_oracle(torch, B, precision):
    """8 cells of the 470 x 6000 network (n_H quantiles of 256 cells) with T
    coupled, to 1e6 yr: the same bars as the small network."""
    from tests.golden.make_integrate_truth import thermal_inputs
    ref = truth("thermal_large")
    d, th, nH, Av, z0 = thermal_inputs(470, 6000, ref["cells"])
    z, stats, code = run_thermal(torch, B, d, th, nH, Av, z0, ref["t_end"], precision=precision)
    assert code == B.SM_OK, stats["status"]
    y10, y6 = np.array(ref["y"]).T, np.array(ref["y_rtol6"]).T
    e_g, e_o = np.maximum(cell_err(z, y10), 1.0), np.maximum(cell_err(y6, y10), 1.0)
    f = 2.0 if precision == "fp64" else 3.0
    assert e_g.max() <= 100.0 and e_g.max() <= f * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 2.0 * np.median(e_o), (np.median(e_g), np.median(e_o))
    steps_o = np.array(ref["steps_rtol6"])
    assert np.all(np.abs(stats["steps"] - steps_o) <= 0.25 * steps_o + 10), (stats["steps"], steps_o)
    t = th.t_index
    assert np.all(np.abs(z[t] - y10[t]) <= 1e-4 * y10[t]), np.abs(z[t] / y10[t] - 1).max()
    check_element_drift(d, th, z0, z, y6, stats, precision)


def test_fixed_temperature_limit_matches_plain_integrator(torch, B):
    """With beta = gamma = 0 the rate coefficients do not depend on T, and the
    coupled run's abundances follow the fixed-T library integrator (whatever
    T does) to within the integration tolerance."""
    from oracle import thermal as _oth
    d0 = sn.generate(2312, 32, 180)
    dep = np.isin(d0.rclass, _oth.T_DEPENDENT)
    d0 = dataclasses.replace(d0, beta=np.where(dep, 0.0, d0.beta), gamma=np.where(dep, 0.0, d0.gamma))
    d = sth.with_temperature(d0)
    th = sth.thermal_params(d)
    C = 16
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    z0 = sth.thermal_start(d, sc.atomic_start(d, C), T)
    t_end = 1e5 * YEAR
    z, stats, code = run_thermal(torch, B, d, th, nH, Av, z0, t_end, rtol=1e-9)
    assert code == B.SM_OK
    # the plain integrator on the chemical network with k' at any T
    ld = B.pad_ld(C)
    net0 = B.Network(d0, 0)
    vec = lambda a: torch.tensor(np.asarray(a, dtype=float), dtype=torch.float64, device="cuda")
    kd = torch.zeros((d0.n_r, ld), dtype=torch.float64, device="cuda")
    net0.rates_eval(vec(T), vec(nH), vec(Av), kd, C, zeta=th.zeta)
    st0 = B.State(net0, C, rtol=1e-9)
    yd = dev(torch, sc.atomic_start(d0, C), ld)
    assert st0.integrate(kd, yd, t_end, C) == B.SM_OK
    y = yd.cpu().numpy()[:, :C]
    m = np.arange(d.n_s) != th.t_index
    big = y > 1e-14
    err = np.abs(z[m][big] - y[big]) / y[big]
    assert err.max() < 1e-5, err.max()


def thermal_step_by_step(torch, B, d, th, nH, Av, z0, t_end, **opts):
    """Attempt by attempt (sm_step_bdf with one attempt, then
    sm_state_read): per cell the accepted states z_0, z_1, ... and the step
    log (end times, sizes, orders)."""
    C = z0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    net.set_thermal(th)
    st = B.State(net, C, record_steps=20000, **opts)
    vec = lambda a: torch.tensor(np.asarray(a, dtype=float), dtype=torch.float64, device="cuda")
    st.set_cells(vec(nH), vec(Av), None, C)
    st.init(None, dev(torch, z0, ld), t_end, C)
    zs = [[z0[:, c].copy()] for c in range(C)]
    prev = np.zeros(C, dtype=np.int64)
    zd = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    stats = B.stats_tensor(C, "cuda")
    for _ in range(100000):
        st.step(None, 1)
        running = st.read(zd, stats)
        s = B.stats_to_numpy(stats)
        z = zd.cpu().numpy()
        for c in np.nonzero(s["steps"] != prev)[0]:
            assert s["steps"][c] == prev[c] + 1
            zs[c].append(z[:, c].copy())
        prev = s["steps"].astype(np.int64)
        if running == 0:
            break
    assert np.all(s["status"] == B.CELL_OK), s["status"]
    tl, hl, ql = (a.cpu().numpy() for a in st.steps_log(int(prev.max()), C))
    return zs, tl, hl, ql


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_replay_matches_oracle(torch, B, precision):
    """The coupled step math, independently of the step-size controller: 6
    cells of the 32 x 180 network with T coupled are integrated to 1e5 yr
    attempt by attempt with the Newton iteration converged tightly (Jacobian
    refreshed every attempt, Newton tolerance 1e-6 WRMS units), and every
    accepted GPU step, temperature included, agrees with the oracle's exact
    solution of the same BDF equation (same history, t_m, h_m, q_m) to
    1e-10 relative (1e-24 absolute)."""
    d = sth.with_temperature(sn.generate(2312, 32, 180))
    th = sth.thermal_params(d)
    C = 6
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    z0 = sth.thermal_start(d, sc.atomic_start(d, C), T)
    zs, tl, hl, ql = thermal_step_by_step(torch, B, d, th, nH, Av, z0, 1e5 * YEAR, precision=precision,
                                          newton_tol=1e-6, newton_max=8, j_age_max=1, gamma_tol=1e-9,
                                          use_graph=0)
    from oracle.network import stoichiometry
    S = stoichiometry(d)
    errs = []
    for c in range(C):
        N = len(zs[c]) - 1
        ts = [0.0] + [tl[m - 1, c] for m in range(1, N + 1)]
        for m in sorted(set(np.linspace(1, N, 40).astype(int))):
            q = int(ql[m - 1, c])
            zo = oth.solve_step(d, th, (nH[c], Av[c], 1.0), [zs[c][m - 1 - i] for i in range(q)],
                                [ts[m - 1 - i] for i in range(q)], ts[m], hl[m - 1, c], S, y_start=zs[c][m])
            errs.append(np.max(np.abs(zs[c][m] - zo) / (1e-10 * np.abs(zo) + 1e-24)))
    errs = np.array(errs)
    assert len(errs) > 100
    assert errs.max() <= 1.0, (errs.max(), np.quantile(errs, 0.99))


def test_bench_batch_matches_oracle_on_sampled_cells(torch, B):
    """The thermal bench leg's launch configuration: the first 4096 cells of
    the coupled-temperature workload as one batch (mixed precision); the 8
    cells of the stored large-network truth are among them (cells are a
    seeded stream) and take the bars of test_large_network_matches_oracle."""
    from synth.workloads import make_thermal
    ref = truth("thermal_large")
    cells = ref["cells"]
    d, th, nH, Av, z0 = make_thermal("thermal_470x6000_c16384", cells=4096)
    from tests.golden.make_integrate_truth import thermal_inputs
    _, _, nH_s, Av_s, z0_s = thermal_inputs(470, 6000, cells)
    assert np.array_equal(nH[cells], nH_s) and np.array_equal(z0[:, cells], z0_s)
    z, stats, code = run_thermal(torch, B, d, th, nH, Av, z0, ref["t_end"], precision="mixed")
    assert code == B.SM_OK and np.all(stats["status"] == B.CELL_OK)
    y10, y6 = np.array(ref["y"]).T, np.array(ref["y_rtol6"]).T
    zs = z[:, cells]
    e_g, e_o = np.maximum(cell_err(zs, y10), 1.0), np.maximum(cell_err(y6, y10), 1.0)
    assert e_g.max() <= 100.0 and e_g.max() <= 3.0 * e_o.max(), (e_g.max(), e_o.max())
    assert np.median(e_g) <= 2.0 * np.median(e_o), (np.median(e_g), np.median(e_o))
    t = th.t_index
    assert np.all(np.abs(zs[t] - y10[t]) <= 1e-4 * y10[t]), np.abs(zs[t] / y10[t] - 1).max()
