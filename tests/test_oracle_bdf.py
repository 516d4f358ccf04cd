"""Pins for the oracle's BDF integrator."""
from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bdf
from oracle import kinetics as ok
from oracle import network as on
from synth import network as sn

# Textbook fixed-step BDF coefficients (sum_i a_i y_{n+1-i} = h f_{n+1}).
BDF_TEXTBOOK = {
    1: [Fr(1), Fr(-1)],
    2: [Fr(3, 2), Fr(-2), Fr(1, 2)],
    3: [Fr(11, 6), Fr(-3), Fr(3, 2), Fr(-1, 3)],
    4: [Fr(25, 12), Fr(-4), Fr(3), Fr(-4, 3), Fr(1, 4)],
    5: [Fr(137, 60), Fr(-5), Fr(5), Fr(-10, 3), Fr(5, 4), Fr(-1, 5)],
}


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_bdf_coefficients_constant_step(q):
    h = 0.37
    t0 = 12.5
    tau = [t0 + h] + [t0 - i * h for i in range(q)]
    a = bdf.bdf_alphas(tau, h)
    assert np.allclose(a, [float(x) for x in BDF_TEXTBOOK[q]], rtol=1e-12, atol=1e-12)


def test_bdf_coefficients_exact_on_polynomials_variable_step():
    """Variable nodes: sum_i alpha_i p(tau_i) = h p'(tau_0) for deg p <= q."""
    rng = np.random.default_rng(1)
    for q in range(1, 6):
        tau = np.cumsum(rng.uniform(0.2, 1.5, q + 1))[::-1].tolist()
        h = tau[0] - tau[1]
        a = bdf.bdf_alphas(tau, h)
        for deg in range(q + 1):
            lhs = sum(ai * ti ** deg for ai, ti in zip(a, tau))
            rhs = h * deg * tau[0] ** (deg - 1) if deg else 0.0
            assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9)


def test_lagrange_extrapolation_exact_for_polynomials():
    rng = np.random.default_rng(2)
    nodes = sorted(rng.uniform(0, 3, 5).tolist(), reverse=True)
    c = rng.standard_normal(5)
    p = lambda t: sum(c[i] * t ** i for i in range(5))
    w = bdf.lagrange_weights(nodes, 3.7)
    assert sum(wi * p(ti) for wi, ti in zip(w, nodes)) == pytest.approx(p(3.7), rel=1e-11)


def riccati_B(t, kk, z, A0, B0):
    """Exact solution of dB/dt = k (N - 2B)^2 - zeta B (the worked example with
    A = N - 2B, N = A0 + 2 B0), by separation with the roots B1 < B2 of
    4k B^2 - (4kN + zeta) B + k N^2."""
    N = A0 + 2 * B0
    a, b, c = 4 * kk, 4 * kk * N + z, kk * N * N
    disc = np.sqrt(b * b - 4 * a * c)
    B1 = 2 * c / (b + disc)
    B2 = (b + disc) / (2 * a)
    lam = a * (B2 - B1)
    inv_r = (B0 - B1) / (B0 - B2) * np.exp(-lam * t)   # 1/R(t)
    return (B2 * inv_r - B1) / (inv_r - 1.0)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_fixed_step_convergence_order(q):
    """Global error of fixed-step BDF-q on the worked example falls as h^q.
    The step history is seeded with the exact solution at t = -h, -2h, ... so
    that no lower-order start-up step pollutes the rate."""
    d = sn.worked_example()
    k = np.array([1.0, 0.5])
    A0, B0 = 0.6, 0.2
    N = A0 + 2 * B0
    t_end = 2.0
    errs = []
    for n in (40, 80, 160):
        h = t_end / n
        ts = [-i * h for i in range(1, q + 1)]
        Bs = [riccati_B(t, k[0], k[1], A0, B0) for t in ts]
        ys = [np.array([N - 2 * B, B]) for B in Bs]
        opts = bdf.BDFOptions(q_max=q, fixed_h=h, newton_max=12, newton_tol=1e-13,
                              j_age_max=1, rtol=1e-12, atol=1e-14)
        r = bdf.integrate_cell(d, k, np.array([A0, B0]), t_end, opts, history=(ts, ys))
        errs.append(abs(r.y[1] - riccati_B(t_end, k[0], k[1], A0, B0)))
    rate = np.log2(errs[1] / errs[2])
    assert rate == pytest.approx(q, abs=0.35)


def test_backward_euler_step_on_linear_network():
    """One BDF1 step on a linear (one-body) network is (I - hA)^-1 y0."""
    d = sn.generate(2312, 32, 180)
    keep = np.nonzero(d.rclass != 0)[0]
    keep = keep[(d.reactants[keep, 1] < 0)]         # one reactant only
    lin = sn.NetDesc(d.names, d.comp, d.reactants[keep], d.products[keep], d.rclass[keep],
                     d.alpha[keep], d.beta[keep], d.gamma[keep])
    rng = np.random.default_rng(3)
    k = 10 ** rng.uniform(-3, 0, lin.n_r)
    y0 = 10 ** rng.uniform(-4, 0, lin.n_s)
    A = ok.jacobian(lin, k, y0)
    h = 0.7
    opts = bdf.BDFOptions(q_max=1, fixed_h=h, newton_max=1, j_age_max=1)
    r = bdf.integrate_cell(lin, k, y0, h, opts)
    ref = np.linalg.solve(np.eye(lin.n_s) - h * A, y0)
    assert np.allclose(r.y, ref, rtol=1e-12, atol=1e-15)


def test_adaptive_worked_example_against_riccati():
    d = sn.worked_example()
    k = np.array([1.0e-3, 2.0e-5])
    A0, B0 = 1.0, 0.0
    for t_end in (1e2, 1e4, 1e7):
        r = bdf.integrate_cell(d, k, np.array([A0, B0]), t_end, bdf.BDFOptions(rtol=1e-6, atol=1e-20))
        assert r.status == bdf.STATUS_OK
        B = riccati_B(t_end, k[0], k[1], A0, B0)
        assert r.y[1] == pytest.approx(B, rel=2e-5)
        assert r.y[0] + 2 * r.y[1] == pytest.approx(1.0, rel=1e-13)


def test_adaptive_linear_network_against_expm():
    """One-body networks are linear: x(t) = expm(t A) x0."""
    d = sn.generate(2312, 32, 180)
    keep = np.nonzero((d.reactants[:, 1] < 0))[0]
    lin = sn.NetDesc(d.names, d.comp, d.reactants[keep], d.products[keep], d.rclass[keep],
                     d.alpha[keep], d.beta[keep], d.gamma[keep])
    rng = np.random.default_rng(8)
    k = 10 ** rng.uniform(-4, 0, lin.n_r)
    y0 = 10 ** rng.uniform(-3, 0, lin.n_s)
    A = ok.jacobian(lin, k, y0)
    for t_end in (1.0, 30.0, 1e4):
        r = bdf.integrate_cell(lin, k, y0, t_end, bdf.BDFOptions(rtol=1e-8, atol=1e-14))
        ref = sla.expm(t_end * A) @ y0
        big = ref > 1e-6 * ref.max()
        assert np.allclose(r.y[big], ref[big], rtol=2e-5)


def test_conservation_through_integration():
    d = sn.generate(2312, 32, 180)
    from synth import cells
    T, nH, Av = cells.conditions(4998, 2, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = cells.atomic_start(d, 2)
    E = on.element_matrix(d).astype(float)
    for c in range(2):
        r = bdf.integrate_cell(d, k[:, c], y0[:, c], 1e5 * ok.YEAR)
        assert r.status == bdf.STATUS_OK and r.steps > 20
        tot0 = E[:3] @ y0[:, c]
        assert np.allclose(E[:3] @ r.y, tot0, rtol=1e-12, atol=0.0)
        assert abs(E[3] @ r.y) <= 1e-12 * np.abs(y0[:, c]).sum()


def _quadratic_root(a2, a1, a0, lo, hi):
    """The root of a2 B^2 + a1 B + a0 = 0 in [lo, hi] (closed form)."""
    disc = np.sqrt(a1 * a1 - 4 * a2 * a0)
    roots = [(-a1 - disc) / (2 * a2), (-a1 + disc) / (2 * a2)]
    inside = [r for r in roots if lo - 1e-12 <= r <= hi + 1e-12]
    assert len(inside) == 1
    return inside[0]


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_solve_step_worked_example_closed_form(q):
    """One constant-step BDF-q step of the worked example (2A -> B at k, B ->
    2A at zeta; A = N - 2B conserved) from an arbitrary history: with the
    textbook coefficients the implicit equation for B is the quadratic
    a_0 B + sum_i a_i B_{n+1-i} = h (k (N - 2B)^2 - zeta B), solved in closed
    form; solve_step must return that root and A = N - 2B."""
    d = sn.worked_example()
    kk, z = 0.8, 0.3
    N = 1.0
    h = 0.45
    t0 = 3.0
    Bh = [0.11 + 0.03 * i for i in range(q)]               # B_n, B_{n-1}, ...
    hist_y = [np.array([N - 2 * B, B]) for B in Bh]
    hist_t = [t0 - i * h for i in range(q)]
    a = [float(x) for x in BDF_TEXTBOOK[q]]
    c = sum(a[i] * Bh[i - 1] for i in range(1, q + 1))
    # a0 B + c - h k (N^2 - 4 N B + 4 B^2) + h z B = 0
    B = _quadratic_root(-4 * h * kk, a[0] + 4 * h * kk * N + h * z, c - h * kk * N * N, 0.0, N / 2)
    y = bdf.solve_step(d, np.array([kk, z]), hist_y, hist_t, t0 + h, h)
    assert y[1] == pytest.approx(B, rel=1e-13)
    assert y[0] == pytest.approx(N - 2 * B, rel=1e-13)


def test_solve_step_reproduces_integrator_steps():
    """With a tight Newton tolerance the integrator's accepted steps solve the
    same equation: solve_step from the recorded history (newest first) gives
    every accepted y_m to within that tolerance."""
    from synth import cells
    d = sn.generate(2312, 32, 180)
    T, nH, Av = cells.conditions(4998, 1, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)[:, 0]
    y0 = cells.atomic_start(d, 1)[:, 0]
    S = on.stoichiometry(d)
    t_end = 1e3 * ok.YEAR
    r = bdf.integrate_cell(d, k, y0, t_end, bdf.BDFOptions(newton_tol=1e-9, newton_max=8), S, record=True)
    assert r.status == bdf.STATUS_OK and r.steps > 30
    acc = [e for e in r.log if e["outcome"] == "accept"]
    ys, ts = [y0], [0.0]
    for e in acc:
        ys.append(e["y"])
        ts.append(t_end if e["t"] + e["h"] >= t_end else e["t"] + e["h"])
    for m, e in enumerate(acc):
        q = e["q"]
        hy = [ys[m - i] for i in range(q)]
        ht = [ts[m - i] for i in range(q)]
        ym = bdf.solve_step(d, k, hy, ht, ts[m + 1], e["h"], S)
        w = 1.0 / (1e-6 * np.abs(ys[m]) + 1e-20)
        assert bdf.wrms(ym - ys[m + 1], w) <= 1e-8, m
    # a wrong history order (oldest first) is caught
    m = next(i for i, e in enumerate(acc) if e["q"] >= 3)
    q = acc[m]["q"]
    bad = bdf.solve_step(d, k, [ys[m - q + 1 + i] for i in range(q)], [ts[m - i] for i in range(q)],
                         ts[m + 1], acc[m]["h"], S)
    w = 1.0 / (1e-6 * np.abs(ys[m]) + 1e-20)
    assert bdf.wrms(bad - ys[m + 1], w) > 1e-3
