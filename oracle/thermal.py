"""Coupled gas temperature: the energy equation as one more state component.

Test infrastructure (oracle): see the package docstring.

The paper keeps T fixed during a chemistry step and updates the energy
outside the chemical solver (Section 5); it gives no energy equation.  The
coupled variant integrates T in the same BDF system as the abundances, with
the rate coefficients re-evaluated from the current T inside every step.
The energy equation is our reading, stated here in full:

* state z = (x_0 .. x_{n-1}, T): the network carries a temperature slot
  t (a species with no atoms, no charge and no reactions; its S row is 0);
* thermal energy per H nucleus of an ideal monatomic gas, in kelvin units:
  u = 3/2 T x_tot, x_tot = sum_{i != t} x_i (electrons included);
* du/dt = heat - L_line - L_gg with
    heat    constant heating per H nucleus (cosmic rays),
    L_line  = n_H sum_i x_i L_i exp(-E_i / T)   (two-level coolants, low density),
    L_gg    = lam n_H (T - T_dust)              (gas-grain energy exchange);
* hence dT/dt = (heat - L_line - L_gg - 3/2 T sum_{i != t} f_i) / (3/2 x_tot),
  f = S R(k'(T), x) the chemical right-hand side of Eq. 7.

Only the two-body and dissociative-recombination coefficients depend on T
(k' = alpha (T/300)^beta exp(-gamma/T) n_H, d ln k'/dT = beta/T + gamma/T^2);
cosmic-ray and photo coefficients do not.

Closed forms that pin this file (tests/test_oracle_thermal.py): with no
heating and no cooling, T x_tot is invariant; with the chemistry frozen,
T relaxes exponentially to T_dust + heat / (lam n_H) when only the grains
couple; the Jacobian agrees with central differences of the right-hand side.
"""
from __future__ import annotations

import numpy as np

from .bdf import BDFOptions, CellResult, STATUS_NAN, integrate_system, solve_step_system
from .kinetics import jacobian as chem_jacobian
from .kinetics import reaction_rates
from .network import stoichiometry

T_DEPENDENT = (0, 3)   # two-body, dissociative recombination


def rates_at(desc, th, T, nH, Av, chi=1.0):
    """k'[n_r] of one cell at temperature T: the rate laws of
    kinetics.rate_coefficients, vectorised over the reactions of one cell."""
    cls = desc.rclass
    order = (desc.reactants >= 0).sum(axis=1)
    coll = desc.alpha * (T / 300.0) ** desc.beta * np.exp(-desc.gamma / T)
    k = np.where(cls == 1, desc.alpha * th.zeta, 0.0)
    k = np.where(cls == 2, chi * desc.alpha * np.exp(-desc.gamma * Av), k)
    k = np.where(np.isin(cls, T_DEPENDENT), coll, k)
    return k * nH ** (order - 1)


def dlnk_dT(desc, T):
    """d ln k'_j / dT [n_r]: beta/T + gamma/T^2 for the T-dependent classes, else 0."""
    g = desc.beta / T + desc.gamma / T ** 2
    dep = np.isin(desc.rclass, T_DEPENDENT)
    return np.where(dep, g, 0.0)


def _chem_mask(desc, th):
    m = np.ones(desc.n_s, dtype=bool)
    m[th.t_index] = False
    return m


def energy_rhs(desc, th, nH, z, f):
    """dT/dt for state z, given the chemical right-hand side f (its T entry unused)."""
    m = _chem_mask(desc, th)
    T = z[th.t_index]
    x_tot = z[m].sum()
    line = nH * np.sum(z[m] * th.L[m] * np.exp(-th.E[m] / T))
    gg = th.lam * nH * (T - th.T_dust)
    return (th.heat - line - gg - 1.5 * T * f[m].sum()) / (1.5 * x_tot)


def rhs(desc, th, cell, z, S=None):
    """dz/dt [n_s] for one cell; cell = (n_H, A_V, chi)."""
    if S is None:
        S = stoichiometry(desc)
    nH, Av, chi = cell
    z = np.asarray(z, dtype=float)
    k = rates_at(desc, th, z[th.t_index], nH, Av, chi)
    f = S @ reaction_rates(desc, k, z)
    f[th.t_index] = energy_rhs(desc, th, nH, z, f)
    return f


def jacobian(desc, th, cell, z, S=None):
    """Dense d(dz/dt)/dz [n_s, n_s] for one cell."""
    if S is None:
        S = stoichiometry(desc)
    nH, Av, chi = cell
    z = np.asarray(z, dtype=float)
    t = th.t_index
    T = z[t]
    m = _chem_mask(desc, th)
    k = rates_at(desc, th, T, nH, Av, chi)
    R = reaction_rates(desc, k, z)
    f = S @ R
    J = chem_jacobian(desc, k, z, S)          # species block; column t is 0 (T is no reactant)
    u = S @ (R * dlnk_dT(desc, T))            # d f / dT
    J[:, t] = u
    # the temperature row: dT/dt = N / (3/2 x_tot)
    x_tot = z[m].sum()
    fT = energy_rhs(desc, th, nH, z, f)
    cool = th.L * np.exp(-th.E / T)
    dN_dx = -nH * cool - 1.5 * T * J[m].sum(axis=0)
    row = dN_dx / (1.5 * x_tot) - fT / x_tot
    dN_dT = (-nH * np.sum(z[m] * cool[m] * th.E[m] / T ** 2) - th.lam * nH
             - 1.5 * f[m].sum() - 1.5 * T * u[m].sum())
    row[t] = dN_dT / (1.5 * x_tot)
    J[t] = row
    return J


def integrate_cell(desc, th, cell, z0, t_end, opts: BDFOptions = BDFOptions(), S=None,
                   record=False) -> CellResult:
    """The BDF method of oracle/bdf.py on the coupled system of one cell."""
    if S is None:
        S = stoichiometry(desc)
    z0 = np.array(z0, dtype=float)
    if not np.all(np.isfinite(np.asarray(cell, dtype=float))) or not z0[th.t_index] > 0.0:
        return CellResult(y=z0.copy(), t=0.0, status=STATUS_NAN)
    return integrate_system(lambda z: rhs(desc, th, cell, z, S),
                            lambda z: jacobian(desc, th, cell, z, S), z0, t_end, opts, record)


def integrate(desc, th, nH, Av, chi, z0, t_end, opts: BDFOptions = BDFOptions(), cells=None):
    """Integrate every cell (columns of z0[n_s, C]; n_H, A_V, chi per cell) in turn."""
    S = stoichiometry(desc)
    C = z0.shape[1]
    chi = np.broadcast_to(np.asarray(chi, dtype=float), (C,))
    cells = range(C) if cells is None else cells
    return [integrate_cell(desc, th, (float(nH[c]), float(Av[c]), float(chi[c])), z0[:, c], t_end, opts, S)
            for c in cells]


def solve_step(desc, th, cell, hist_y, hist_t, t_new, h, S=None, tol=1e-14, max_iter=30, y_start=None):
    """Exact solution of one implicit BDF step of the coupled system (see
    oracle/bdf.py solve_step), given its history newest first."""
    if S is None:
        S = stoichiometry(desc)
    return solve_step_system(lambda z: rhs(desc, th, cell, z, S), lambda z: jacobian(desc, th, cell, z, S),
                             hist_y, hist_t, t_new, h, tol, max_iter, y_start)
