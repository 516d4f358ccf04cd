"""Named synthetic workloads (sizes, ranges and seeds of the measured configs).

Network seed 2312 and cell seed 4998 throughout.  Times are in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass

YEAR = 3.15576e7
NET_SEED = 2312
CELL_SEED = 4998


@dataclass(frozen=True)
class Workload:
    name: str
    n_s: int
    n_r: int
    cells: int
    T: object
    nH: object
    Av: object
    start: str            # "atomic" or "loguniform"
    t_end: float = 0.0
    chi: float = 1.0      # FUV field scaling the photorates
    rtol: float = 1e-6
    atol: float = 1e-20


WORKLOADS = {
    "single_cell_32x180": Workload("single_cell_32x180", 32, 180, 1, 10.0, 1e4, 5.0,
                                   "atomic", 1e6 * YEAR),
    "rhs_jac_470x6000_c4096": Workload("rhs_jac_470x6000_c4096", 470, 6000, 4096,
                                       (10.0, 300.0), (1e2, 1e7), (0.0, 10.0), "loguniform"),
    "integrate_470x6000_c65536": Workload("integrate_470x6000_c65536", 470, 6000, 65536,
                                          (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0),
                                          "atomic", 1e6 * YEAR),
    "adjoint_470x6000_c1024": Workload("adjoint_470x6000_c1024", 470, 6000, 1024,
                                       (10.0, 300.0), (1e2, 1e7), (0.0, 10.0),
                                       "atomic", 1e5 * YEAR),
    "mixed_470x6000_c16384": Workload("mixed_470x6000_c16384", 470, 6000, 16384,
                                      (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0),
                                      "atomic", 1e6 * YEAR),
    # the paper's PDR benchmark geometry (Section 3, model F2 of Roellig et al.
    # 2007): a slab of 128 cells on a logarithmic A_V grid, n_H = 1e3, T = 50 K,
    # FUV field chi = 1e5, atomic start, 30 Myr; the A_V grid is pdr_av()
    "pdr_slab_470x6000_c128": Workload("pdr_slab_470x6000_c128", 470, 6000, 128,
                                       50.0, 1e3, "pdr", "atomic", 30e6 * YEAR, chi=1e5),
    # coupled gas temperature (the energy equation of synth/thermal.py as one
    # more state component): the mixed-precision workload's cells, each
    # starting at its drawn T, the temperature slot appended to the network
    "thermal_470x6000_c16384": Workload("thermal_470x6000_c16384", 470, 6000, 16384,
                                        (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0),
                                        "atomic", 1e6 * YEAR),
}

PDR_AV_MIN, PDR_AV_MAX = 1e-3, 20.0


def pdr_av(C):
    """A_V of the slab's cells: the centres (in log A_V) of C cells evenly
    spaced in log A_V between 1e-3 and 20, finest at the illuminated surface."""
    import numpy as np
    lo, hi = np.log10(PDR_AV_MIN), np.log10(PDR_AV_MAX)
    return 10.0 ** (lo + (np.arange(C) + 0.5) * (hi - lo) / C)


def make_thermal(name, cells=None):
    """(desc with the temperature slot, thermal parameters, nH, Av, z0) for a
    coupled-temperature workload; z0's slot row holds the cells' initial T."""
    from . import thermal as _th
    desc, T, nH, Av, y0 = make(name, cells)
    d_t = _th.with_temperature(desc)
    return d_t, _th.thermal_params(d_t), nH, Av, _th.thermal_start(d_t, y0, T)


def make(name, cells=None):
    """(desc, T, nH, Av, y0) for a named workload, optionally on fewer cells."""
    from . import cells as _cells
    from .network import generate
    w = WORKLOADS[name]
    C = w.cells if cells is None else cells
    desc = generate(NET_SEED, w.n_s, w.n_r)
    if w.Av == "pdr":
        import numpy as np
        T, nH, Av = np.full(C, float(w.T)), np.full(C, float(w.nH)), pdr_av(C)
    else:
        T, nH, Av = _cells.conditions(CELL_SEED, C, w.T, w.nH, w.Av)
    if w.start == "atomic":
        y0 = _cells.atomic_start(desc, C)
    else:
        y0 = _cells.loguniform_abundances(desc, CELL_SEED, C)
    return desc, T, nH, Av, y0
