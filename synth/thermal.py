"""Inputs of the coupled-temperature workloads: the temperature slot and the
heating / cooling parameters.

The paper holds the gas temperature fixed during a chemistry step and
updates the energy outside the chemical solver (Section 5).  The coupled
variant integrates T in the same implicit system as the abundances; its
energy equation (written out in oracle/thermal.py and in the library) takes
the parameters drawn or fixed here:

* the state gains one component: a species named "T" appended after the
  chemical species, with no atoms, no charge and no reactions, whose value
  is the gas temperature in K;
* heat: the constant heating rate per H nucleus in K/s (cosmic rays
  depositing about 20 eV per ionisation: zeta * 20 eV / k_B);
* line cooling by a few coolant species (two-level emitters in the
  low-density limit): per coolant an excitation temperature E_i (K) and a
  coefficient L_i (K cm^3 s^-1); zero for every other species;
* gas-grain energy exchange: coefficient lam (cm^3 s^-1) and the dust
  temperature T_dust (K).

Only inputs are produced here; the energy equation itself is computed by the
oracle and by the CUDA library independently.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .network import NetDesc

ZETA = 1.3e-17               # s^-1, the workloads' cosmic-ray ionisation rate
EV_K = 11604.518             # 1 eV / k_B in K
HEAT = ZETA * 20.0 * EV_K    # K s^-1 per H nucleus
T_DUST = 20.0                # K (the paper's PDR benchmark's dust temperature)
LAM = 3.0e-17                # cm^3 s^-1, gas-grain coupling
# coolant species: (excitation temperature K, coefficient K cm^3 s^-1)
COOLANTS = {"C+": (91.2, 1.0e-10), "O": (228.0, 2.0e-10), "C": (23.6, 5.0e-11), "CO": (5.5, 1.0e-12)}
T_NAME = "T"


def with_temperature(desc: NetDesc) -> NetDesc:
    """The network with the temperature slot appended as its last species."""
    comp = np.vstack([desc.comp, np.zeros((1, desc.comp.shape[1]), dtype=desc.comp.dtype)])
    return dataclasses.replace(desc, names=list(desc.names) + [T_NAME], comp=comp,
                               meta=dict(desc.meta, t_index=desc.n_s))


@dataclasses.dataclass(frozen=True)
class Thermal:
    """Energy-equation parameters of a network carrying the temperature slot."""
    t_index: int
    L: np.ndarray     # [n_s] line-cooling coefficients, K cm^3 s^-1 (0: not a coolant)
    E: np.ndarray     # [n_s] excitation temperatures, K
    heat: float = HEAT
    lam: float = LAM
    T_dust: float = T_DUST
    zeta: float = ZETA


def thermal_params(desc_t: NetDesc, heat=HEAT, lam=LAM, T_dust=T_DUST, coolants=None) -> Thermal:
    """Parameters for a network returned by with_temperature(); coolants
    missing from the network are skipped."""
    t = desc_t.species_index(T_NAME)
    L = np.zeros(desc_t.n_s)
    E = np.ones(desc_t.n_s)
    for name, (e, l) in (COOLANTS if coolants is None else coolants).items():
        if name in desc_t.names:
            i = desc_t.species_index(name)
            L[i], E[i] = l, e
    return Thermal(t, L, E, float(heat), float(lam), float(T_dust))


def thermal_start(desc_t: NetDesc, y0: np.ndarray, T0) -> np.ndarray:
    """Initial state with the temperature slot set: y0[n_s - 1 or n_s, C] of
    the chemical species (the slot's row, if present, is overwritten)."""
    C = y0.shape[1]
    t = desc_t.species_index(T_NAME)
    z = np.zeros((desc_t.n_s, C))
    z[: y0.shape[0]] = y0[: desc_t.n_s]
    z[t] = np.broadcast_to(np.asarray(T0, dtype=float), (C,))
    return z
