"""Seeded synthetic chemical networks shaped like the paper's UMIST rate12 network.

The paper's benchmark network (Section 3: 468 species x 6175 reactions, 13
elements, 24580 nonzeros, hub rows for H / H2 / e- of 1794 / 980 / 891
reactions, Section 5) is not available, so networks of the same shape are drawn
here from H, C, O and the electron:

* species: neutral, cationic and (small) anionic C_c H_h O_o compositions plus
  e-, small ones preferred; named by formula and stored in alphabetical order,
  the paper's "original" species order (Section 3);
* reactions, grouped by class (the paper's original reaction order):
  60 % two-body (ion-neutral / neutral-neutral), 20 % cosmic-ray
  ionisation / dissociation, 15 % photoreactions, 5 % dissociative
  recombination; 1-2 reactants, 1-4 products, every reaction conserving each
  element and charge;
* rate parameters: two-body and DR  log10 alpha ~ U[-12,-9], beta ~ U[-1,1],
  gamma ~ U[0,500] K;  cosmic ray  log10 alpha ~ U[0,3];  photo
  log10 alpha ~ U[-11,-9], gamma ~ U[1,3].

Only inputs are produced here (compositions, reactant / product lists, class
codes, rate parameters).  The stoichiometry matrix, formats, rates and every
other piece of the method are computed independently by the oracle and by the
CUDA library from these arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64, stream_key

ELEMENTS = ("H", "C", "O")
TWO_BODY, COSMIC_RAY, PHOTO, DISS_RECOMB = 0, 1, 2, 3
CLASS_NAMES = {TWO_BODY: "two-body", COSMIC_RAY: "cosmic-ray", PHOTO: "photo",
               DISS_RECOMB: "dissociative-recombination"}
MAX_REACTANTS, MAX_PRODUCTS = 2, 4


@dataclass
class NetDesc:
    """Explicit network: what `sm_net_build` and the oracle both consume.

    comp[i] = (n_H, n_C, n_O, charge) of species i; reactants / products are
    species indices padded with -1; a species listed twice appears with
    multiplicity two.
    """
    names: list
    comp: np.ndarray          # int32 [n_s, 4]
    reactants: np.ndarray     # int32 [n_r, 2]
    products: np.ndarray      # int32 [n_r, 4]
    rclass: np.ndarray        # int8  [n_r]
    alpha: np.ndarray         # float64 [n_r]
    beta: np.ndarray          # float64 [n_r]
    gamma: np.ndarray         # float64 [n_r]
    meta: dict = field(default_factory=dict)

    @property
    def n_s(self) -> int:
        return int(self.comp.shape[0])

    @property
    def n_r(self) -> int:
        return int(self.reactants.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.comp.shape[1]) - 1

    def species_index(self, name: str) -> int:
        return self.names.index(name)

    def reaction_str(self, j: int) -> str:
        lhs = " + ".join(self.names[a] for a in self.reactants[j] if a >= 0)
        rhs = " + ".join(self.names[p] for p in self.products[j] if p >= 0)
        return f"{lhs} -> {rhs}"


def formula(h: int, c: int, o: int, q: int) -> str:
    if h == 0 and c == 0 and o == 0:
        return "E-"
    s = ""
    for sym, n in (("C", c), ("H", h), ("O", o)):
        if n == 1:
            s += sym
        elif n > 1:
            s += f"{sym}{n}"
    return s + ("+" if q > 0 else "-" if q < 0 else "")


def _species_pool():
    pool = []
    for c in range(0, 9):
        for o in range(0, 5):
            for h in range(0, 11):
                n_at = h + c + o
                if n_at == 0 or n_at > 14:
                    continue
                for q in (0, 1, -1):
                    if q == -1 and n_at > 3:
                        continue
                    pool.append((h, c, o, q))
    return pool


_MANDATORY = [(1, 0, 0, 0), (1, 0, 0, 1), (2, 0, 0, 0), (0, 1, 0, 0), (0, 1, 0, 1),
              (0, 0, 1, 0), (0, 0, 1, 1), (2, 0, 0, 1), (3, 0, 0, 1), (1, 0, 0, -1)]

# Integer selection weights that create the paper's hub rows (H, H2, e-):
# Section 5 reports H in 1794, H2 in 980 and e- in 891 of 6175 reactions.
_HUB_WEIGHT = {"H": 62, "H2": 28, "H+": 8, "H3+": 8, "C+": 6, "O": 6, "C": 5,
               "O+": 3, "CO": 4, "OH": 4, "H2O": 3, "CH": 3, "H2+": 3}


def generate(seed: int, n_s: int, n_r: int) -> NetDesc:
    """Draw a conserving network of n_s species and n_r reactions."""
    if n_s < 12:
        raise ValueError("need at least 12 species (atoms, ions, e-)")
    rs = SplitMix64(stream_key(seed, 1))
    pool = _species_pool()
    mandatory = set(_MANDATORY)
    keyed = []
    for sp in pool:
        h, c, o, q = sp
        size = h + 2 * (c + o) + (1 if q != 0 else 0) + (2 if q < 0 else 0)
        jitter = rs.below(1 << 20)
        keyed.append(((-1 << 40) if sp in mandatory else (size << 22) + jitter, sp))
    keyed.sort()
    chosen = [sp for _, sp in keyed[: n_s - 1]] + [(0, 0, 0, -1)]
    names = [formula(*sp) for sp in chosen]
    order = sorted(range(n_s), key=lambda i: names[i])
    comp = np.array([chosen[i] for i in order], dtype=np.int32)
    names = [names[i] for i in order]
    by_comp = {tuple(int(v) for v in comp[i]): i for i in range(n_s)}
    atoms = comp[:, :3].astype(np.int64)
    n_atoms = atoms.sum(axis=1)
    e_idx = names.index("E-")
    w_hub = np.array([_HUB_WEIGHT.get(nm, 1) for nm in names], dtype=np.int64)
    w_hub[e_idx] = 0

    n2 = n_r * 60 // 100
    ncr = n_r * 20 // 100
    nph = n_r * 15 // 100
    ndr = n_r - n2 - ncr - nph
    rr = SplitMix64(stream_key(seed, 2))

    def pick_weighted(mask, weights):
        w = np.where(mask, weights, 0)
        cum = np.cumsum(w)
        tot = int(cum[-1])
        if tot == 0:
            return -1
        r = rr.below(tot)
        return int(np.searchsorted(cum, r, side="right"))

    def decompose(total, m):
        """Split composition `total` into m existing species (last one by lookup)."""
        rem = np.array(total, dtype=np.int64)
        out = []
        for i in range(m - 1):
            left = m - 1 - i  # pieces still to come after this one
            fits = (atoms <= rem[:3]).all(axis=1) & small
            fits &= (rem[:3].sum() - n_atoms) >= left - 1
            p = pick_weighted(fits, w_hub)
            if p < 0:
                return None
            out.append(p)
            rem = rem - comp[p].astype(np.int64)
        last = by_comp.get(tuple(int(v) for v in rem))
        if last is None:
            return None
        out.append(last)
        return out

    seen = set()
    reac_l, prod_l, cls_l = [], [], []

    def accept(reac, prods, cls):
        key = (tuple(sorted(reac)), tuple(sorted(prods)))
        if key[0] == key[1] or key in seen:
            return False
        seen.add(key)
        reac_l.append(sorted(reac))
        prod_l.append(sorted(prods))
        cls_l.append(cls)
        return True

    heavy_or_any = n_atoms >= 1
    small = (n_atoms >= 1) & (n_atoms <= 3)
    m_two = [5, 65, 22, 8]        # weights of 1..4 products, two-body
    m_diss = [70, 25, 5]          # weights of 2..4 products, dissociation

    def draw(cls):
        for _ in range(500):
            if cls == TWO_BODY:
                a = pick_weighted(heavy_or_any, np.ones(n_s, dtype=np.int64))
                b = pick_weighted(heavy_or_any, w_hub)
                tot = comp[a].astype(np.int64) + comp[b]
                m = 1 + rr.weighted(m_two)
                prods = decompose(tot, m)
                if prods is not None and accept([a, b], prods, cls):
                    return
            elif cls in (COSMIC_RAY, PHOTO):
                a = pick_weighted(heavy_or_any, np.ones(n_s, dtype=np.int64))
                ion = tuple(int(v) for v in comp[a, :3]) + (int(comp[a, 3]) + 1,)
                if rr.below(100) < 45 and ion in by_comp:
                    prods = [by_comp[ion], e_idx]
                else:
                    m = 2 + rr.weighted(m_diss)
                    prods = decompose(comp[a].astype(np.int64), m)
                if prods is not None and accept([a], prods, cls):
                    return
            else:
                cations = (comp[:, 3] == 1) & heavy_or_any
                a = pick_weighted(cations, np.ones(n_s, dtype=np.int64))
                tot = comp[a].astype(np.int64) + comp[e_idx]
                m = 1 if n_atoms[a] == 1 else 2 + rr.weighted([70, 30])
                prods = decompose(tot, m)
                if prods is not None and accept([a, e_idx], prods, cls):
                    return
        raise RuntimeError(f"could not draw a class-{cls} reaction")

    for cls, cnt in ((TWO_BODY, n2), (COSMIC_RAY, ncr), (PHOTO, nph), (DISS_RECOMB, ndr)):
        for _ in range(cnt):
            draw(cls)

    reactants = np.full((n_r, MAX_REACTANTS), -1, dtype=np.int32)
    products = np.full((n_r, MAX_PRODUCTS), -1, dtype=np.int32)
    for j in range(n_r):
        reactants[j, : len(reac_l[j])] = reac_l[j]
        products[j, : len(prod_l[j])] = prod_l[j]
    rclass = np.array(cls_l, dtype=np.int8)

    rp = SplitMix64(stream_key(seed, 3))
    alpha = np.empty(n_r)
    beta = np.zeros(n_r)
    gamma = np.zeros(n_r)
    for j in range(n_r):
        u1, u2, u3 = rp.uniform(), rp.uniform(), rp.uniform()
        c = int(rclass[j])
        if c in (TWO_BODY, DISS_RECOMB):
            alpha[j] = 10.0 ** (-12.0 + 3.0 * u1)
            beta[j] = -1.0 + 2.0 * u2
            gamma[j] = 500.0 * u3
        elif c == COSMIC_RAY:
            alpha[j] = 10.0 ** (3.0 * u1)
        else:
            alpha[j] = 10.0 ** (-11.0 + 2.0 * u1)
            gamma[j] = 1.0 + 2.0 * u3
    return NetDesc(names, comp, reactants, products, rclass, alpha, beta, gamma,
                   meta={"seed": seed, "generator": "synth.network.generate"})


def worked_example() -> NetDesc:
    """The two-reaction network of Eqs. 2-6: 2A -> B (rate k n_A^2) and
    B + photon -> 2A (rate zeta n_B).  A and B are given the compositions of
    H and H2 so that element conservation holds."""
    comp = np.array([[1, 0, 0, 0], [2, 0, 0, 0]], dtype=np.int32)
    reactants = np.array([[0, 0], [1, -1]], dtype=np.int32)
    products = np.array([[1, -1, -1, -1], [0, 0, -1, -1]], dtype=np.int32)
    rclass = np.array([TWO_BODY, PHOTO], dtype=np.int8)
    return NetDesc(["A", "B"], comp, reactants, products, rclass,
                   alpha=np.array([1e-10, 1e-10]), beta=np.zeros(2),
                   gamma=np.array([0.0, 2.0]), meta={"name": "worked example, Eqs. 2-6"})
