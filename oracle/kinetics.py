"""Rate coefficients, reaction rates, right-hand side and analytic Jacobian.

Test infrastructure (oracle): see the package docstring.

State variable: fractional abundance x_i = n_i / n_H (the paper's n_i are
number densities, Eq. 1; dividing Eq. 7 by n_H gives the same form with
k'_j = k_j n_H^(order_j - 1)).  Rate coefficients are evaluated once per cell
outside the ODE solver, as the paper's KM2 does (Section 3):

* two-body and dissociative recombination:  k = alpha (T/300)^beta exp(-gamma/T)
* cosmic ray:                               k = alpha zeta
* photoreaction:                            k = chi alpha exp(-gamma A_V)
  (chi: the FUV field in units of the Draine field, Section 3; 1 by default)

R_j = k'_j prod_{a in reactants(j)} x_a  (a species listed twice is squared,
Eqs. 2-6), and dx/dt = S R (Eq. 7).
"""
from __future__ import annotations

import numpy as np

from .network import stoichiometry

ZETA_CR = 1.3e-17   # s^-1, cosmic-ray ionisation rate of the workload definition
YEAR = 3.15576e7    # s, Julian year


def order_of(desc) -> np.ndarray:
    return (desc.reactants >= 0).sum(axis=1)


def rate_coefficients(desc, T, nH, Av, zeta=ZETA_CR, chi=None) -> np.ndarray:
    """k'[n_r, C] for cells with temperature T, density n_H and extinction A_V;
    chi (per cell, default 1) scales the photorates."""
    T = np.atleast_1d(np.asarray(T, dtype=float))
    nH = np.atleast_1d(np.asarray(nH, dtype=float))
    Av = np.atleast_1d(np.asarray(Av, dtype=float))
    C = T.shape[0]
    chi = np.ones(C) if chi is None else np.broadcast_to(np.asarray(chi, dtype=float), (C,))
    k = np.empty((desc.n_r, C))
    order = order_of(desc)
    for j in range(desc.n_r):
        a, b, g = desc.alpha[j], desc.beta[j], desc.gamma[j]
        cls = int(desc.rclass[j])
        if cls in (0, 3):
            kj = a * (T / 300.0) ** b * np.exp(-g / T)
        elif cls == 1:
            kj = np.full(C, a * zeta)
        elif cls == 2:
            kj = chi * a * np.exp(-g * Av)
        else:
            raise ValueError(f"unknown reaction class {cls}")
        k[j] = kj * nH ** (order[j] - 1)
    return k


def reaction_rates(desc, k, y) -> np.ndarray:
    """R[n_r, C] = k' times the product of reactant abundances."""
    y = np.asarray(y, dtype=float)
    single = y.ndim == 1
    if single:
        y = y[:, None]
        k = np.asarray(k)[:, None] if np.ndim(k) == 1 else k
    R = np.array(k, dtype=float, copy=True)
    for slot in range(desc.reactants.shape[1]):
        a = desc.reactants[:, slot]
        has = a >= 0
        R[has] *= y[a[has]]
    return R[:, 0] if single else R


def rhs(desc, k, y, S=None) -> np.ndarray:
    """dx/dt = S R (Eq. 7), dense matrix product."""
    if S is None:
        S = stoichiometry(desc)
    return S @ reaction_rates(desc, k, y)


def rhs_scale(desc, k, y, S=None) -> np.ndarray:
    """sum_j |S_ij R_j|: the magnitude against which a sum of S_ij R_j can be
    resolved in floating point (the condition of the sum)."""
    if S is None:
        S = stoichiometry(desc)
    return np.abs(S) @ np.abs(reaction_rates(desc, k, y))


def rate_derivatives(desc, k, y):
    """dR_j/dx_l for the (at most two) reactants l of each reaction.

    Returns a list of (j, l, value) with value an array over cells: for a
    one-body reaction dR/dx_a = k'; for a + b (a != b) dR/dx_a = k' x_b and
    dR/dx_b = k' x_a; for 2a dR/dx_a = 2 k' x_a."""
    y = np.asarray(y, dtype=float)
    out = []
    for j in range(desc.n_r):
        a, b = int(desc.reactants[j, 0]), int(desc.reactants[j, 1])
        if b < 0:
            out.append((j, a, k[j]))
        elif a == b:
            out.append((j, a, 2.0 * k[j] * y[a]))
        else:
            out.append((j, a, k[j] * y[b]))
            out.append((j, b, k[j] * y[a]))
    return out


def jacobian(desc, k, y, S=None) -> np.ndarray:
    """Dense analytic J = S dR/dx for ONE cell (k[n_r], y[n_s])."""
    if S is None:
        S = stoichiometry(desc)
    D = np.zeros((desc.n_r, desc.n_s))
    for j, l, v in rate_derivatives(desc, k, y):
        D[j, l] += v
    return S @ D


def jacobian_scale(desc, k, y, S=None) -> np.ndarray:
    """sum_j |S_ij| |dR_j/dx_l|: the condition of each Jacobian entry's sum."""
    if S is None:
        S = stoichiometry(desc)
    D = np.zeros((desc.n_r, desc.n_s))
    for j, l, v in rate_derivatives(desc, k, y):
        D[j, l] += abs(v)
    return np.abs(S) @ D
