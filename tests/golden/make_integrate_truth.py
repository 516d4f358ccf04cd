"""Writes tight-tolerance oracle solutions used as the reference ("truth") by
the integrator tests: the oracle's BDF method at rtol 1e-10 / atol 1e-24 on
seeded synthetic cells.  Calls only the oracle and the input generators.

    python tests/golden/make_integrate_truth.py [small|large|all]
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
}


def case_inputs(name):
    n_s, n_r, C, Tr, nr, ar, t_end = CASES[name]
    d = sn.generate(2312, n_s, n_r)
    T, nH, Av = sc.conditions(4998, C, Tr, nr, ar)
    return d, ok.rate_coefficients(d, T, nH, Av), sc.atomic_start(d, C), t_end


def _one(args):
    name, c, rtol, atol = args
    d, k, y0, t_end = case_inputs(name)
    r = ob.integrate_cell(d, k[:, c], y0[:, c], t_end, ob.BDFOptions(rtol=rtol, atol=atol))
    return c, r.y.tolist(), r.status, r.steps


def _solve_all(name, rtol, atol):
    C = CASES[name][2]
    with mp.get_context("spawn").Pool(min(C, os.cpu_count() or 1)) as pool:
        return sorted(pool.map(_one, [(name, c, rtol, atol) for c in range(C)]))


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
    for nm in (["small", "large"] if which == "all" else [which]):
        make(nm, only6)
        print("wrote", nm)
