"""Seeded cell conditions and initial abundances for the synthetic workloads.

Cells are independent hydro cells (the paper's domain-decomposition axis,
Section 3).  Each array is drawn from its own counter-based SplitMix64
sub-stream, so the first C cells of a larger batch equal a smaller batch.
"""
from __future__ import annotations

import numpy as np

from .rng import stream_key, uniform_array

# Elemental abundances relative to hydrogen nuclei (Table 1) for the elements
# the synthetic networks carry.
ELEMENT_TOTALS = {"H": 1.0, "C": 1.0e-4, "O": 3.0e-4}


def _loguniform(key, C, lo, hi):
    u = uniform_array(key, C)
    return 10.0 ** (np.log10(lo) + u * (np.log10(hi) - np.log10(lo)))


def conditions(seed, C, T=(10.0, 300.0), nH=(1e2, 1e7), Av=(0.0, 10.0)):
    """T and n_H log-uniform, A_V uniform over the given ranges; a scalar range
    (a plain number) fixes the value for every cell."""
    def draw(stream, rng, log):
        if np.isscalar(rng):
            return np.full(C, float(rng))
        lo, hi = rng
        if log:
            return _loguniform(stream_key(seed, stream), C, lo, hi)
        return lo + (hi - lo) * uniform_array(stream_key(seed, stream), C)
    return draw(11, T, True), draw(12, nH, True), draw(13, Av, False)


def atomic_start(desc, C):
    """All elements atomic and neutral (Section 3): x_H = 1, x_C = 1e-4,
    x_O = 3e-4, everything else 0; y[n_s, C]."""
    y = np.zeros((desc.n_s, C))
    for el, tot in ELEMENT_TOTALS.items():
        y[desc.species_index(el)] = tot
    return y


def loguniform_abundances(desc, seed, C, lo=1e-20, hi=1e-4):
    """Log-uniform abundances normalised to the element totals.

    Each species is owned by the rarest element it contains (Table 1 order
    C < O < H); each owner group is scaled so that its atoms of the owner
    element add up to that element's total.  The electron abundance is then
    set to the net positive charge (anions scaled down if they outweigh the
    cations)."""
    n_s = desc.n_s
    y = _loguniform(stream_key(seed, 21), n_s * C, lo, hi).reshape(n_s, C)
    rarity = sorted(ELEMENT_TOTALS, key=lambda e: ELEMENT_TOTALS[e])
    col = {"H": 0, "C": 1, "O": 2}
    e_idx = desc.species_index("E-")
    owner = np.full(n_s, -1)
    for i in range(n_s):
        for el in rarity:
            if desc.comp[i, col[el]] > 0:
                owner[i] = col[el]
                break
    for el, tot in ELEMENT_TOTALS.items():
        grp = owner == col[el]
        atoms = desc.comp[grp, col[el]].astype(float)[:, None]
        y[grp] *= tot / (atoms * y[grp]).sum(axis=0, keepdims=True)
    charge = desc.comp[:, 3]
    cat = y[charge > 0].sum(axis=0)
    an_mask = (charge < 0) & (np.arange(n_s) != e_idx)
    an = y[an_mask].sum(axis=0)
    scale = np.where(an > cat, cat / np.maximum(an, 1e-300), 1.0)
    y[an_mask] *= scale
    y[e_idx] = cat - y[an_mask].sum(axis=0)
    y[e_idx] = np.maximum(y[e_idx], 0.0)
    return y
