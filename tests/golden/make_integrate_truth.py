"""Writes tight-tolerance oracle solutions used as the reference ("truth") by
the integrator tests: the oracle's BDF method at rtol 1e-10 / atol 1e-24 on
seeded synthetic cells.  Calls only the oracle and the input generators.

    python tests/golden/make_integrate_truth.py [small|large|strat|pdr|thermal_small|thermal_large|all]

The "strat" case is a stiffness-stratified sample of the 16,384-cell
mixed-precision workload (470 x 6000, T 10-1000 K, n_H 1e2-1e8, A_V 0-20,
atomic start, 1e6 yr): every 128th of its cells is integrated by the oracle
at rtol 1e-6, and the 32 cells at evenly spaced quantiles of those step
counts are kept.

The "pdr" case: 8 cells spread over the 128-cell PDR slab (the paper's
benchmark geometry: n_H 1e3, T 50 K, FUV field 1e5 Draine fields on the
photorates, A_V 1e-3 to 20 on a log grid, atomic start, 30 Myr).

The "thermal_*" cases integrate the coupled-temperature system
(oracle/thermal.py) from each cell's drawn T.
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bdf as ob          # noqa: E402
from oracle import kinetics as ok     # noqa: E402
from synth import cells as sc         # noqa: E402
from synth import network as sn       # noqa: E402

YEAR = 3.15576e7
CASES = {
    # name: (n_s, n_r, cells, T range, nH range, Av range, t_end)
    "small": (32, 180, 24, (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0), 1e6 * YEAR),
    "large": (470, 6000, 4, (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0), 1e6 * YEAR),
    "strat": (470, 6000, 32, (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0), 1e6 * YEAR),
}


STRAT_POOL = 16384      # cells of the workload the stratified sample is drawn from
STRAT_STRIDE = 128      # every 128th cell is a candidate
STRAT_CELLS = 32


def case_inputs(name, C=None, cells=None):
    """(desc, k'[n_r, len(cells)], y0, t_end) for the given cells (default:
    all) of the case's first C cells."""
    n_s, n_r, C0, Tr, nr, ar, t_end = CASES[name]
    C = C0 if C is None else C
    cells = np.arange(C) if cells is None else np.asarray(cells)
    d = sn.generate(2312, n_s, n_r)
    T, nH, Av = sc.conditions(4998, C, Tr, nr, ar)
    T, nH, Av = T[cells], nH[cells], Av[cells]
    return d, ok.rate_coefficients(d, T, nH, Av), sc.atomic_start(d, len(cells)), t_end


def _one(args):
    name, c, rtol, atol, C = args
    d, k, y0, t_end = case_inputs(name, C, [c])
    r = ob.integrate_cell(d, k[:, 0], y0[:, 0], t_end, ob.BDFOptions(rtol=rtol, atol=atol))
    return c, r.y.tolist(), r.status, r.steps


def _solve_all(name, rtol, atol, cells=None, C=None):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    cells = list(range(CASES[name][2])) if cells is None else list(cells)
    with mp.get_context("spawn").Pool(min(len(cells), os.cpu_count() or 1)) as pool:
        res = pool.map(_one, [(name, c, rtol, atol, C) for c in cells])
    order = {c: i for i, c in enumerate(cells)}
    return sorted(res, key=lambda r: order[r[0]])


PDR_CELLS = [0, 18, 36, 54, 72, 90, 108, 127]


def _pdr_one(args):
    c, rtol, atol = args
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["pdr_slab_470x6000_c128"]
    d, T, nH, Av, y0 = make(w.name)
    k = ok.rate_coefficients(d, T[c:c + 1], nH[c:c + 1], Av[c:c + 1], chi=w.chi)[:, 0]
    r = ob.integrate_cell(d, k, y0[:, c], w.t_end, ob.BDFOptions(rtol=rtol, atol=atol))
    return c, r.y.tolist(), r.status, r.steps


def make_pdr():
    """integrate_truth_pdr.json: PDR_CELLS of the PDR slab at rtol 1e-10
    (y) and at the tested rtol 1e-6 (y_rtol6), with both step counts."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(min(len(PDR_CELLS), os.cpu_count() or 1)) as pool:
        r10 = pool.map(_pdr_one, [(c, 1e-10, 1e-24) for c in PDR_CELLS])
        r6 = pool.map(_pdr_one, [(c, 1e-6, 1e-20) for c in PDR_CELLS])
    out = {"source": "oracle BDF at rtol 1e-10, atol 1e-24 (make_integrate_truth.py)", "case": "pdr",
           "workload": "pdr_slab_470x6000_c128", "cells": PDR_CELLS,
           "y": [r[1] for r in r10], "status": [r[2] for r in r10], "steps": [r[3] for r in r10],
           "y_rtol6": [r[1] for r in r6], "steps_rtol6": [r[3] for r in r6]}
    with open(os.path.join(HERE, "integrate_truth_pdr.json"), "w") as fh:
        json.dump(out, fh)


THERMAL_SMALL_CELLS = list(range(16))
THERMAL_POOL = 256      # the large thermal case samples the first 256 cells ...
THERMAL_LARGE_N = 8     # ... at evenly spaced quantiles of n_H


def thermal_inputs(n_s, n_r, cells):
    """(desc with the temperature slot, thermal parameters, nH, Av, z0) of the
    coupled-temperature cases: the "strat" ranges (T 10-1000 K, n_H 1e2-1e8,
    A_V 0-20), atomic start at each cell's drawn T."""
    from synth import thermal as sth
    d = sth.with_temperature(sn.generate(2312, n_s, n_r))
    cells = np.asarray(cells)
    T, nH, Av = sc.conditions(4998, int(cells.max()) + 1, (10.0, 1000.0), (1e2, 1e8), (0.0, 20.0))
    T, nH, Av = T[cells], nH[cells], Av[cells]
    return d, sth.thermal_params(d), nH, Av, sth.thermal_start(d, sc.atomic_start(d, len(cells)), T)


def thermal_large_cells():
    _, _, nH, _, _ = thermal_inputs(32, 180, np.arange(THERMAL_POOL))
    order = np.argsort(nH, kind="stable")
    return sorted(int(order[int((i + 0.5) * THERMAL_POOL / THERMAL_LARGE_N)]) for i in range(THERMAL_LARGE_N))


def _thermal_one(args):
    n_s, n_r, c, rtol, atol = args
    from oracle import thermal as oth
    d, th, nH, Av, z0 = thermal_inputs(n_s, n_r, [c])
    r = oth.integrate_cell(d, th, (float(nH[0]), float(Av[0]), 1.0), z0[:, 0], 1e6 * YEAR,
                           ob.BDFOptions(rtol=rtol, atol=atol))
    return c, r.y.tolist(), r.status, r.steps


def make_thermal(name):
    """integrate_truth_<name>.json for the coupled-temperature cases
    (thermal_small: 32 x 180, cells 0-15; thermal_large: 470 x 6000, 8 cells
    at quantiles of n_H among the first 256), to 1e6 yr: rtol-1e-10 (y) and
    rtol-1e-6 (y_rtol6) oracle solutions with their step counts."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    n_s, n_r = (32, 180) if name == "thermal_small" else (470, 6000)
    cells = THERMAL_SMALL_CELLS if name == "thermal_small" else thermal_large_cells()
    with mp.get_context("spawn").Pool(min(2 * len(cells), os.cpu_count() or 1)) as pool:
        r10 = pool.map_async(_thermal_one, [(n_s, n_r, c, 1e-10, 1e-24) for c in cells])
        r6 = pool.map_async(_thermal_one, [(n_s, n_r, c, 1e-6, 1e-20) for c in cells])
        r10, r6 = r10.get(), r6.get()
    out = {"source": "oracle BDF at rtol 1e-10, atol 1e-24 (make_integrate_truth.py)", "case": name,
           "n_s": n_s, "n_r": n_r, "cells": list(cells), "t_end": 1e6 * YEAR,
           "y": [r[1] for r in r10], "status": [r[2] for r in r10], "steps": [r[3] for r in r10],
           "y_rtol6": [r[1] for r in r6], "steps_rtol6": [r[3] for r in r6]}
    with open(os.path.join(HERE, f"integrate_truth_{name}.json"), "w") as fh:
        json.dump(out, fh)


def make_strat():
    """integrate_truth_strat.json: 32 cells of the 16,384-cell workload at
    evenly spaced quantiles of the oracle's rtol-1e-6 step count (drawn from
    every 128th cell), with the rtol-1e-10 solution (y), the oracle's own
    rtol-1e-6 solution (y_rtol6) and both step counts."""
    cand = list(range(0, STRAT_POOL, STRAT_STRIDE))
    res6 = _solve_all("strat", 1e-6, 1e-20, cand, STRAT_POOL)
    steps = np.array([r[3] for r in res6])
    order = np.argsort(steps, kind="stable")
    pick = sorted({int(order[int((i + 0.5) * len(cand) / STRAT_CELLS)]) for i in range(STRAT_CELLS)})
    cells = [cand[i] for i in pick]
    res10 = _solve_all("strat", 1e-10, 1e-24, cells, STRAT_POOL)
    out = {"source": "oracle BDF at rtol 1e-10, atol 1e-24 (make_integrate_truth.py)",
           "case": "strat", "spec": [str(v) for v in CASES["strat"]], "pool_cells": STRAT_POOL,
           "cells": cells, "candidate_steps_rtol6": steps.tolist(),
           "y": [r[1] for r in res10], "status": [r[2] for r in res10], "steps": [r[3] for r in res10],
           "y_rtol6": [res6[i][1] for i in pick], "steps_rtol6": [res6[i][3] for i in pick]}
    with open(os.path.join(HERE, "integrate_truth_strat.json"), "w") as fh:
        json.dump(out, fh)


def make(name, only_rtol6=False):
    """Writes integrate_truth_<name>.json: y = the rtol-1e-10 solution (the
    reference), y_rtol6 = the oracle's own solution at the tested tolerance
    (rtol 1e-6, atol 1e-20), whose distance to y is the bar for the GPU."""
    path = os.path.join(HERE, f"integrate_truth_{name}.json")
    if only_rtol6 and os.path.exists(path):
        with open(path) as fh:
            out = json.load(fh)
    else:
        res = _solve_all(name, 1e-10, 1e-24)
        out = {"source": "oracle BDF at rtol 1e-10, atol 1e-24 (make_integrate_truth.py)",
               "case": name, "spec": [str(v) for v in CASES[name]],
               "y": [r[1] for r in res], "status": [r[2] for r in res], "steps": [r[3] for r in res]}
    res6 = _solve_all(name, 1e-6, 1e-20)
    out["y_rtol6"] = [r[1] for r in res6]
    out["steps_rtol6"] = [r[3] for r in res6]
    with open(path, "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    only6 = "--rtol6-only" in sys.argv
    for nm in (["small", "large", "strat", "pdr", "thermal_small", "thermal_large"] if which == "all" else [which]):
        if nm == "strat":
            make_strat()
        elif nm == "pdr":
            make_pdr()
        elif nm.startswith("thermal"):
            make_thermal(nm)
        else:
            make(nm, only6)
        print("wrote", nm)
