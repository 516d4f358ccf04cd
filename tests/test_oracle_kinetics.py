"""Pins for the oracle's rate coefficients, right-hand side and Jacobian."""
import numpy as np
import pytest

from oracle import kinetics as ok
from oracle import network as on
from synth import network as sn


def test_worked_example_rhs_closed_form():
    """Eqs. 4-5: dA/dt = -2 k A^2 + 2 zeta B, dB/dt = k A^2 - zeta B."""
    d = sn.worked_example()
    k = np.array([3.0e-2, 7.0e-3])     # (k, zeta)
    for A, B in ((0.25, 0.5), (1.0, 0.0), (1e-10, 2.0)):
        f = ok.rhs(d, k, np.array([A, B]))
        assert f[0] == pytest.approx(-2 * k[0] * A * A + 2 * k[1] * B, rel=1e-15, abs=1e-300)
        assert f[1] == pytest.approx(k[0] * A * A - k[1] * B, rel=1e-15, abs=1e-300)


def test_matrix_form_equals_gain_loss_form():
    """Eq. 7 (S.R) against Eq. 1's gains-minus-losses sum, accumulated reaction by
    reaction: the identity the paper's algorithm rests on."""
    d = sn.generate(11, 32, 180)
    rng = np.random.default_rng(3)
    k = 10 ** rng.uniform(-6, 0, d.n_r)
    y = 10 ** rng.uniform(-8, 0, d.n_s)
    f = ok.rhs(d, k, y)
    g = np.zeros(d.n_s)
    for j in range(d.n_r):
        R = k[j]
        for a in d.reactants[j]:
            if a >= 0:
                R *= y[a]
        for a in d.reactants[j]:
            if a >= 0:
                g[a] -= R
        for p in d.products[j]:
            if p >= 0:
                g[p] += R
    scale = ok.rhs_scale(d, k, y)
    assert np.all(np.abs(f - g) <= 1e-14 * scale + 1e-300)


def test_rhs_conserves_elements():
    """E.S = 0 makes E.f = 0 for any state."""
    d = sn.generate(2312, 120, 1200)
    rng = np.random.default_rng(4)
    k = 10 ** rng.uniform(-6, 0, d.n_r)
    y = 10 ** rng.uniform(-10, 0, (d.n_s, 3))
    f = ok.rhs(d, k[:, None] * np.ones((1, 3)), y)
    E = on.element_matrix(d).astype(float)
    scale = np.abs(E) @ ok.rhs_scale(d, k[:, None] * np.ones((1, 3)), y)
    assert np.all(np.abs(E @ f) <= 1e-13 * scale)


def test_rate_coefficient_special_cases():
    """T = 300 K removes the (T/300)^beta factor; gamma = 0 removes the
    exponential; A_V = 0 leaves the bare photorate; two-body k' carries one
    factor of n_H and one-body k' none."""
    d = sn.generate(2312, 32, 180)
    two = np.nonzero(d.rclass == 0)[0]
    cr = np.nonzero(d.rclass == 1)[0]
    ph = np.nonzero(d.rclass == 2)[0]
    k300 = ok.rate_coefficients(d, [300.0], [1.0], [0.0])[:, 0]
    assert np.allclose(k300[two], d.alpha[two] * np.exp(-d.gamma[two] / 300.0), rtol=1e-15)
    assert np.allclose(k300[cr], d.alpha[cr] * ok.ZETA_CR, rtol=1e-15)
    assert np.allclose(k300[ph], d.alpha[ph], rtol=1e-15)
    k_n = ok.rate_coefficients(d, [50.0, 50.0], [1.0, 1e3], [2.0, 2.0])
    assert np.allclose(k_n[two, 1] / k_n[two, 0], 1e3, rtol=1e-14)
    assert np.allclose(k_n[cr, 1], k_n[cr, 0], rtol=0) and np.allclose(k_n[ph, 1], k_n[ph, 0], rtol=0)


def test_dissociative_recombination_rate_law():
    """Dissociative recombination (class 3) follows the two-body law on its
    own parameters: at T = 300 K and gamma read off k(T), alpha and beta are
    recovered from two temperatures, k' carries one factor of n_H (two
    reactants: ion and electron), and a cell's A_V and zeta leave it alone."""
    d = sn.generate(2312, 470, 6000)
    dr = np.nonzero(d.rclass == 3)[0]
    assert len(dr) > 100
    assert np.all((d.reactants[dr] >= 0).sum(axis=1) == 2)
    T = np.array([300.0, 30.0, 300.0, 300.0])
    nH = np.array([1.0, 1.0, 1e4, 1.0])
    Av = np.array([0.0, 0.0, 0.0, 7.0])
    k = ok.rate_coefficients(d, T, nH, Av)[dr]
    kz = ok.rate_coefficients(d, T, nH, Av, zeta=1e-15)[dr]
    # T = 300 K: k = alpha exp(-gamma / 300)
    assert np.allclose(k[:, 0], d.alpha[dr] * np.exp(-d.gamma[dr] / 300.0), rtol=1e-15)
    # T = 30 K: k = alpha 0.1^beta exp(-gamma / 30)
    assert np.allclose(k[:, 1], d.alpha[dr] * 0.1 ** d.beta[dr] * np.exp(-d.gamma[dr] / 30.0), rtol=1e-13)
    # one factor of n_H; no dependence on A_V or zeta
    assert np.allclose(k[:, 2], 1e4 * k[:, 0], rtol=1e-15)
    assert np.array_equal(k[:, 3], k[:, 0])
    assert np.array_equal(kz, k)


def test_fuv_field_scales_photorates_only():
    """chi (the FUV field, Section 3) multiplies every photorate and nothing
    else; chi = 1 is the default."""
    d = sn.generate(2312, 470, 6000)
    ph = d.rclass == 2
    T, nH, Av = np.array([50.0, 50.0]), np.array([1e3, 1e3]), np.array([0.3, 7.0])
    k1 = ok.rate_coefficients(d, T, nH, Av)
    kc = ok.rate_coefficients(d, T, nH, Av, chi=np.array([1e5, 2.0]))
    assert np.array_equal(ok.rate_coefficients(d, T, nH, Av, chi=1.0), k1)
    assert np.allclose(kc[ph, 0], 1e5 * k1[ph, 0], rtol=1e-15)
    assert np.allclose(kc[ph, 1], 2.0 * k1[ph, 1], rtol=1e-15)
    assert np.array_equal(kc[~ph], k1[~ph])


def test_rate_coefficient_log_linearity():
    """log k is linear in log(T/300) with slope beta, in 1/T with slope -gamma,
    and photorates fall as exp(-gamma A_V)."""
    d = sn.generate(2312, 32, 180)
    two = np.nonzero(d.rclass == 0)[0]
    ph = np.nonzero(d.rclass == 2)[0]
    T = np.array([20.0, 80.0, 320.0])
    k = ok.rate_coefficients(d, T, np.ones(3), np.array([0.0, 1.0, 3.0]))
    lk = np.log(k)
    for j in two[:20]:
        # log k(T) = log alpha + beta log(T/300) - gamma / T: solve the 3 points
        M = np.stack([np.ones(3), np.log(T / 300.0), -1.0 / T], axis=1)
        coef = np.linalg.solve(M, lk[j])
        assert coef[1] == pytest.approx(d.beta[j], abs=1e-9)
        assert coef[2] == pytest.approx(d.gamma[j], rel=1e-9, abs=1e-9)
    slope = (lk[ph, 2] - lk[ph, 1]) / 2.0
    assert np.allclose(slope, -d.gamma[ph], rtol=1e-10)


def test_jacobian_equals_central_difference():
    """f is a quadratic polynomial in x, so the central difference of f along v
    equals J v with no truncation error: only rounding remains."""
    d = sn.generate(2312, 120, 1200)
    rng = np.random.default_rng(5)
    k = 10 ** rng.uniform(-4, 0, d.n_r)
    y = 10 ** rng.uniform(-6, 0, d.n_s)
    v = rng.standard_normal(d.n_s) * y
    J = ok.jacobian(d, k, y)
    for eps in (1e-1, 1e-3):
        fd = (ok.rhs(d, k, y + eps * v) - ok.rhs(d, k, y - eps * v)) / (2 * eps)
        scale = ok.jacobian_scale(d, k, y) @ np.abs(v) + ok.rhs_scale(d, k, y) / eps
        assert np.all(np.abs(J @ v - fd) <= 1e-13 * scale + 1e-300)


def test_jacobian_conserves_elements():
    d = sn.generate(2312, 120, 1200)
    rng = np.random.default_rng(6)
    k = 10 ** rng.uniform(-4, 0, d.n_r)
    y = 10 ** rng.uniform(-6, 0, d.n_s)
    J = ok.jacobian(d, k, y)
    E = on.element_matrix(d).astype(float)
    assert np.all(np.abs(E @ J) <= 1e-13 * (np.abs(E) @ ok.jacobian_scale(d, k, y)) + 1e-300)


def test_worked_example_jacobian_closed_form():
    d = sn.worked_example()
    k = np.array([0.3, 0.05])
    A, B = 0.7, 0.2
    J = ok.jacobian(d, k, np.array([A, B]))
    assert np.allclose(J, [[-4 * k[0] * A, 2 * k[1]], [2 * k[0] * A, -k[1]]], rtol=1e-15)
