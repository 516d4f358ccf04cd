"""Pins of the coupled-temperature oracle (oracle/thermal.py) against closed
forms, an invariant, a quadrature, central differences and the fixed-T
integrator.  The energy equation is the reading stated in oracle/thermal.py
(the paper holds T fixed inside a chemistry step, Section 5)."""
import dataclasses

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import bdf as ob
from oracle import kinetics as ok
from oracle import thermal as oth
from synth import cells as sc
from synth import network as sn
from synth import thermal as sth

YEAR = ok.YEAR


@pytest.fixture(scope="module")
def net():
    d = sth.with_temperature(sn.generate(2312, 32, 180))
    return d, sth.thermal_params(d)


def _cells(d, C=4):
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    return T, nH, Av, sth.thermal_start(d, sc.atomic_start(d, C), T)


def test_rates_match_kinetics(net):
    """The per-cell rate laws equal kinetics.rate_coefficients (the pinned
    fixed-T rates) at every temperature."""
    d, th = net
    for T, nH, Av, chi in ((12.0, 1e3, 0.5, 1.0), (250.0, 1e6, 7.0, 3.0)):
        k = oth.rates_at(d, th, T, nH, Av, chi)
        ref = ok.rate_coefficients(d, [T], [nH], [Av], zeta=th.zeta, chi=[chi])[:, 0]
        assert np.allclose(k, ref, rtol=1e-14, atol=0.0)


def test_dlnk_dT_is_the_log_derivative(net):
    """d ln k'/dT against a central difference of ln k'(T)."""
    d, th = net
    T, eps = 40.0, 1e-5
    kp, km = oth.rates_at(d, th, T * (1 + eps), 1e4, 1.0), oth.rates_at(d, th, T * (1 - eps), 1e4, 1.0)
    fd = (np.log(kp) - np.log(km)) / (2 * eps * T)
    assert np.allclose(oth.dlnk_dT(d, T), fd, rtol=1e-7, atol=1e-12)


def test_temperature_slot_has_no_chemistry(net):
    """The slot has no atoms, no charge and no reactions: its S row is zero,
    and the chemical rows do not see it except through k'(T)."""
    d, th = net
    t = th.t_index
    assert d.names[t] == "T" and not np.any(d.comp[t])
    assert not np.any(d.reactants == t) and not np.any(d.products == t)


def test_jacobian_matches_central_differences(net):
    """Every entry of the temperature row and column (and the species block)
    against central differences of the right-hand side.  The right-hand side
    is a polynomial of degree <= 2 in the abundances (times 1 / x_tot in the
    temperature row), so a central difference with an absolute step of 1e-7
    in an abundance is exact up to rounding; in T the step is 1e-6 T."""
    d, th = net
    T, nH, Av, z0 = _cells(d, 2)
    t = th.t_index
    for c in range(2):
        cell = (nH[c], Av[c], 1.0)
        # a state away from the atomic start, so that every term is alive
        z = oth.integrate_cell(d, th, cell, z0[:, c], 1e3 * YEAR).y
        J = oth.jacobian(d, th, cell, z)
        k = oth.rates_at(d, th, z[t], *cell)
        # magnitude of the terms each row sums (what its rounding is relative to)
        size = ok.rhs_scale(d, k, z)
        m = np.arange(d.n_s) != t
        size[t] = (th.heat + 1.5 * z[t] * size[m].sum() + th.lam * cell[0] * z[t]
                   + cell[0] * np.sum(z * th.L)) / (1.5 * z[m].sum())
        for l in range(d.n_s):
            h = 1e-6 * z[t] if l == t else 1e-7
            zp, zm = z.copy(), z.copy()
            zp[l] += h
            zm[l] -= h
            fd = (oth.rhs(d, th, cell, zp) - oth.rhs(d, th, cell, zm)) / (2 * h)
            noise = 1e-14 * size / h
            bad = np.abs(J[:, l] - fd) > 1e-6 * np.abs(J[:, l]) + noise
            assert not np.any(bad), (c, l, np.flatnonzero(bad), J[bad, l], fd[bad], noise[bad])


def test_no_heating_no_cooling_conserves_T_times_xtot(net):
    """With heat = L = lam = 0 the energy 3/2 T x_tot is constant while the
    chemistry changes the particle number (H -> H2 halves x_tot)."""
    d, th = net
    th0 = dataclasses.replace(th, heat=0.0, lam=0.0, L=np.zeros_like(th.L))
    opts = ob.BDFOptions(rtol=1e-9, atol=1e-24)
    T, nH, Av, z0 = _cells(d, 4)
    m = np.arange(d.n_s) != th.t_index
    moved = 0.0
    for c in range(4):
        r = oth.integrate_cell(d, th0, (nH[c], Av[c], 1.0), z0[:, c], 1e6 * YEAR, opts)
        assert r.status == 0
        e0 = z0[th.t_index, c] * z0[m, c].sum()
        e1 = r.y[th.t_index] * r.y[m].sum()
        assert abs(e1 / e0 - 1.0) < 1e-6, (c, e1 / e0)
        moved = max(moved, abs(r.y[m].sum() / z0[m, c].sum() - 1.0))
    assert moved > 0.05      # the invariant was exercised


def _frozen(d):
    """The same network with every rate coefficient zero."""
    return dataclasses.replace(d, alpha=np.zeros_like(d.alpha))


def test_grain_coupling_relaxes_exponentially(net):
    """Frozen chemistry, no line cooling: 3/2 x_tot dT/dt = heat - lam n_H (T - T_d),
    so T = T_eq + (T0 - T_eq) exp(-lam n_H t / (3/2 x_tot))."""
    d, th = net
    df = _frozen(d)
    th1 = dataclasses.replace(th, L=np.zeros_like(th.L))
    opts = ob.BDFOptions(rtol=1e-10, atol=1e-24)
    z0 = sth.thermal_start(d, sc.atomic_start(d, 1), 150.0)[:, 0]
    m = np.arange(d.n_s) != th.t_index
    x_tot = z0[m].sum()
    for nH in (1e3, 1e5):
        tau = 1.5 * x_tot / (th.lam * nH)
        for t_end in (0.3 * tau, 3.0 * tau):
            r = oth.integrate_cell(df, th1, (nH, 1.0, 1.0), z0, t_end, opts)
            T_eq = th.T_dust + th.heat / (th.lam * nH)
            exact = T_eq + (150.0 - T_eq) * np.exp(-t_end / tau)
            assert abs(r.y[th.t_index] - exact) <= 1e-7 * exact, (nH, t_end, r.y[th.t_index], exact)


def test_line_cooling_against_quadrature(net):
    """Frozen chemistry, one coolant, no heating: the time to cool from T0 to
    T1 is the integral of 3/2 x_tot exp(E/T) / (n_H x_c L_c) dT (quadrature)."""
    d, th = net
    df = _frozen(d)
    c = d.species_index("C+")
    L = np.zeros_like(th.L)
    L[c] = th.L[c]
    th1 = dataclasses.replace(th, heat=0.0, lam=0.0, L=L)
    z0 = sth.thermal_start(d, sc.atomic_start(d, 1), 200.0)[:, 0]
    z0[c] = 1e-4
    m = np.arange(d.n_s) != th.t_index
    x_tot, nH, E = z0[m].sum(), 1e4, th.E[c]
    rate = nH * z0[c] * L[c] / (1.5 * x_tot)
    opts = ob.BDFOptions(rtol=1e-10, atol=1e-24)
    for T1 in (120.0, 40.0):
        t1, _ = quad(lambda T: np.exp(E / T) / rate, T1, 200.0, epsabs=0.0, epsrel=1e-12)
        r = oth.integrate_cell(df, th1, (nH, 1.0, 1.0), z0, t1, opts)
        assert abs(r.y[th.t_index] - T1) <= 1e-6 * T1, (T1, r.y[th.t_index])


def test_temperature_free_rates_reduce_to_fixed_T_chemistry(net):
    """With beta = gamma = 0 for the T-dependent classes the rate coefficients
    do not depend on T, so the abundances follow the fixed-T integrator
    (oracle/bdf.py) whatever T does."""
    d, th = net
    dep = np.isin(d.rclass, oth.T_DEPENDENT)
    dn = dataclasses.replace(d, beta=np.where(dep, 0.0, d.beta), gamma=np.where(dep, 0.0, d.gamma))
    opts = ob.BDFOptions(rtol=1e-10, atol=1e-26)
    T, nH, Av, z0 = _cells(dn, 3)
    m = np.arange(d.n_s) != th.t_index
    for c in range(3):
        r = oth.integrate_cell(dn, th, (nH[c], Av[c], 1.0), z0[:, c], 1e5 * YEAR, opts)
        k = oth.rates_at(dn, th, 100.0, nH[c], Av[c])      # any T: the same k'
        ref = ob.integrate_cell(dn, k, z0[:, c], 1e5 * YEAR, opts)
        big = ref.y[m] > 1e-16
        err = np.abs(r.y[m][big] - ref.y[m][big]) / ref.y[m][big]
        assert err.max() < 1e-6, (c, err.max())
        assert r.y[th.t_index] != z0[th.t_index, c]   # T itself did evolve


def test_solve_step_reproduces_integrator_steps(net):
    """With a tight Newton tolerance the coupled integrator's accepted steps
    solve the same equation: solve_step from the recorded history gives every
    accepted state (T included) to within that tolerance; a history in the
    wrong order is caught."""
    d, th = net
    T, nH, Av, z0 = _cells(d, 1)
    cell = (nH[0], Av[0], 1.0)
    t_end = 1e3 * YEAR
    r = oth.integrate_cell(d, th, cell, z0[:, 0], t_end, ob.BDFOptions(newton_tol=1e-9, newton_max=8),
                           record=True)
    assert r.status == ob.STATUS_OK and r.steps > 30
    acc = [e for e in r.log if e["outcome"] == "accept"]
    ys, ts = [z0[:, 0]], [0.0]
    for e in acc:
        ys.append(e["y"])
        ts.append(t_end if e["t"] + e["h"] >= t_end else e["t"] + e["h"])
    for m, e in enumerate(acc):
        q = e["q"]
        zm = oth.solve_step(d, th, cell, [ys[m - i] for i in range(q)], [ts[m - i] for i in range(q)],
                            ts[m + 1], e["h"])
        w = 1.0 / (1e-6 * np.abs(ys[m]) + 1e-20)
        assert ob.wrms(zm - ys[m + 1], w) <= 1e-8, m
    m = next(i for i, e in enumerate(acc) if e["q"] >= 3)
    q = acc[m]["q"]
    bad = oth.solve_step(d, th, cell, [ys[m - q + 1 + i] for i in range(q)], [ts[m - i] for i in range(q)],
                         ts[m + 1], acc[m]["h"])
    w = 1.0 / (1e-6 * np.abs(ys[m]) + 1e-20)
    assert ob.wrms(bad - ys[m + 1], w) > 1e-3
