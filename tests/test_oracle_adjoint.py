"""Pins for the oracle's discrete adjoint: it must equal the transpose of the
independent forward (tangent) sensitivity through the same frozen-step map,
and central finite differences of that map."""
import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import bdf as ob
from oracle import kinetics as ok
from synth import cells as sc
from synth import network as sn

YEAR = 3.15576e7


@pytest.fixture(scope="module")
def case():
    d = sn.generate(2312, 32, 180)
    T, nH, Av = sc.conditions(4998, 1, (10.0, 300.0), (1e3, 1e5), (0.0, 5.0))
    k = ok.rate_coefficients(d, T, nH, Av)[:, 0]
    y0 = sc.atomic_start(d, 1)[:, 0]
    t_end = 1e3 * YEAR
    steps, res = oa.record_steps(d, k, y0, t_end)
    ys = oa.frozen_forward(d, k, y0, steps)
    return d, k, y0, steps, ys, res


def test_frozen_map_reproduces_adaptive_run(case):
    """Re-solving the recorded steps exactly lands within the Newton tolerance
    of the adaptive run (same method, tighter implicit solves)."""
    d, k, y0, steps, ys, res = case
    assert len(steps) == res.steps and steps[-1][0] == 1e3 * YEAR
    w = 1e-6 * np.abs(ys[-1]) + 1e-20
    assert np.max(np.abs(ys[-1] - res.y) / w) < 5.0


def test_adjoint_equals_forward_sensitivity(case):
    d, k, y0, steps, ys, _ = case
    targets = [d.species_index(s) for s in ("CO", "H2O", "E-")]
    cot = np.zeros((len(targets), d.n_s))
    for r, t in enumerate(targets):
        cot[r, t] = 1.0 / ys[-1][t]
    g = oa.adjoint(d, k, ys, steps, cot)
    sens = oa.forward_sensitivity(d, k, ys, steps)
    ref = cot @ sens
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - ref) <= 1e-9 * scale)


def test_adjoint_against_central_differences(case):
    """Central differences of log y_N[target] in log k_j (h = 1e-6) through the
    frozen map with implicit steps solved to 1e-14."""
    d, k, y0, steps, ys, _ = case
    t = d.species_index("CO")
    cot = np.zeros(d.n_s)
    cot[t] = 1.0 / ys[-1][t]
    g = oa.adjoint(d, k, ys, steps, cot)[0]
    rng = np.random.default_rng(0)
    js = list(np.argsort(-np.abs(g))[:4]) + list(rng.choice(d.n_r, 4, replace=False))
    hh = 1e-6
    for j in js:
        kp, km = k.copy(), k.copy()
        kp[j] *= np.exp(hh)
        km[j] *= np.exp(-hh)
        fp = np.log(oa.frozen_forward(d, kp, y0, steps)[-1][t])
        fm = np.log(oa.frozen_forward(d, km, y0, steps)[-1][t])
        fd = (fp - fm) / (2 * hh)
        assert abs(fd - g[j]) <= 1e-6 * max(abs(g).max(), 1e-30) + 1e-7 * abs(g[j]), (j, fd, g[j])


def test_linear_network_adjoint_is_exact():
    """One-body network: the frozen map is linear in y, and a rate constant
    scaled by exp(s) enters linearly; adjoint and forward sensitivity agree."""
    d = sn.generate(2312, 32, 180)
    keep = np.nonzero(d.reactants[:, 1] < 0)[0]
    lin = sn.NetDesc(d.names, d.comp, d.reactants[keep], d.products[keep], d.rclass[keep],
                     d.alpha[keep], d.beta[keep], d.gamma[keep])
    rng = np.random.default_rng(3)
    k = 10 ** rng.uniform(-3, -1, lin.n_r)
    y0 = 10 ** rng.uniform(-3, 0, lin.n_s)
    steps, _ = oa.record_steps(lin, k, y0, 50.0, ob.BDFOptions(rtol=1e-6, atol=1e-14))
    ys = oa.frozen_forward(lin, k, y0, steps)
    c = np.zeros(lin.n_s)
    c[0] = 1.0
    g = oa.adjoint(lin, k, ys, steps, c)[0]
    ref = c @ oa.forward_sensitivity(lin, k, ys, steps)
    assert np.allclose(g, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_initial_state_gradient_equals_tangent(case):
    """dPhi/dy_0 from the backward recursion against the independent tangent
    recursion dy_N/dy_0."""
    d, k, y0, steps, ys, _ = case
    t = d.species_index("CO")
    cot = np.zeros(d.n_s)
    cot[t] = 1.0 / ys[-1][t]
    _, g0 = oa.adjoint(d, k, ys, steps, cot, with_y0=True)
    ref = cot @ oa.forward_sensitivity_y0(d, k, ys, steps)
    assert np.all(np.abs(g0[0] - ref) <= 1e-9 * np.abs(ref).max())


def test_initial_state_gradient_against_central_differences(case):
    """Central differences in the abundant initial species (relative step
    1e-6), through the frozen map."""
    d, k, y0, steps, ys, _ = case
    t = d.species_index("CO")
    cot = np.zeros(d.n_s)
    cot[t] = 1.0 / ys[-1][t]
    _, g0 = oa.adjoint(d, k, ys, steps, cot, with_y0=True)
    for i in np.nonzero(y0 > 0)[0]:
        dy = 1e-6 * y0[i]
        yp, ym = y0.copy(), y0.copy()
        yp[i] += dy
        ym[i] -= dy
        fp = np.log(oa.frozen_forward(d, k, yp, steps)[-1][t])
        fm = np.log(oa.frozen_forward(d, k, ym, steps)[-1][t])
        fd = (fp - fm) / (2 * dy)
        assert abs(fd - g0[0][i]) <= 1e-6 * np.abs(g0[0]).max() + 1e-6 * abs(g0[0][i]), (i, fd, g0[0][i])
