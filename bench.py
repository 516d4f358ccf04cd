#!/usr/bin/env python
"""Benchmark of the batched stiff-chemistry integrator.

Headline workload: the seeded synthetic network of 470 species x 6000
reactions and 65,536 independent cells of uneven stiffness (T 10-1000 K, n_H
1e2-1e8 cm^-3, A_V 0-20, atomic start), every cell integrated to 1e6 yr with
the library's BDF/Newton method at rtol 1e-6 / atol 1e-20 in the batched
mixed-precision mode.  Metric: accepted cell-steps per second.

One bench step is one slice of a single integration of the whole batch: the
first step evaluates the rate coefficients (sm_rates_eval) and starts every
cell at t = 0 (sm_state_init); every step runs a fixed number of BDF attempts
for all unfinished cells (sm_step_bdf); the last step continues until every
cell has reached t_end.  The K timed steps therefore cover exactly one
complete integration; cell-steps are that integration's accepted steps.  The
warm-up runs W slices of a separate integration of the same batch (graph
capture and clocks) and is discarded.

After the headline line's own measurements the same JSON line carries:
  fp64_vs_mixed   16,384 cells integrated in the plain FP64 mode and in the
                  mixed mode, with the per-species error of both against the
                  oracle's rtol-1e-10 solution on 32 stiffness-stratified cells
  adjoint         1024 cells to 1e5 yr in FP64: reverse sweep for 8 targets
                  against one recorded forward integrate
  rhs_jac         rhs_eval per storage format / row order and jac_eval on
                  4096 cells, against the FP64-pipe ceiling
  pdr_slab        the paper's PDR benchmark geometry (128 cells, 30 Myr) as
                  one whole simulation, mixed and FP64
  thermal         coupled gas temperature: 4096 cells of the coupled-
                  temperature workload to 1e6 yr, beside the same cells at
                  fixed T
  single_cell     the 32 x 180 network, one cell to 1e6 yr (config 0)
  cpu_baseline    the oracle on the host cores: 64 stratified cells, each
                  integrated over the whole interval; beside it the
                  coupled-temperature oracle on 16 cells, the single cell
                  and one right-hand side of the 4096 RHS-workload cells

    python bench.py [--gpus N --steps K --warmup W] [--precision mixed|tf32|fp64]
    python bench.py --impl reference ...      # the CPU oracle on a sample

Multi-GPU (torchrun): every rank integrates its own 65,536 cells (weak
scaling, no collective on the data path); the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

YEAR = 3.15576e7
WORKLOAD = "integrate_470x6000_c65536"
MIXED_WORKLOAD = "mixed_470x6000_c16384"
METRIC = "cell-steps/s (470 sp, 6k rx) plain FP64 vs batched mixed; adjoint/forward ratio"
UNIT = "cell-steps/s"
STRAT_FILE = os.path.join(ROOT, "tests", "golden", "integrate_truth_strat.json")
CPU_CELLS = 64
# every attempt accepts a step, shrinks h or counts a failure, and each cell
# stops after max_steps (100,000) accepted steps: the last bench step never
# needs this many attempts unless something is broken
MAX_TAIL_ATTEMPTS = 2_000_000

# Peaks of the pipes that bind these kernels, from unit counts and the
# 2.07 GHz maximum SM clock of this GPU (152 SMs): FP32 128 lanes x 2 flops,
# FP64 4 flops per SM per clock.  HBM: the measured copy bandwidth.
SM_COUNT, SM_GHZ = 152, 2.07
PEAK_FP32 = SM_COUNT * 128 * 2 * SM_GHZ / 1e3     # TFLOP/s
PEAK_FP64 = SM_COUNT * 4 * SM_GHZ / 1e3           # TFLOP/s

# DRAM bytes (read + write) per processed unit of a kernel, from a committed
# ncu capture in profiles/ (named there), keyed on the kernel class, the
# precision and the hash of integrate.cu's code (comments and whitespace
# removed) at capture time: a changed kernel reports traffic null until it
# is captured again.
TRAFFIC = {
    # profiles/refresh_kernel_mixed_2048cells.md: 11.47 GB in a launch that
    # refreshed all 2048 cells
    ("refresh", "mixed", "5e9214d3aef36f79"): 5.599e6,
}


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "tf32", "fp64"])
    p.add_argument("--cells", type=int, default=65536)
    p.add_argument("--t-end-yr", type=float, default=1e6)
    p.add_argument("--attempts-est", type=int, default=1400,
                   help="expected attempts of one integration; slices are attempts-est / steps long")
    p.add_argument("--time-kernel", default="refresh",
                   choices=["none", "refresh", "rhs", "solve", "predict", "finish"])
    p.add_argument("--refresh-per-sm", type=int, default=0,
                   help="cap on resident refresh CTAs per SM for the main integration (0: as many as fit)")
    p.add_argument("--thermal-time-kernel", default="none",
                   choices=["none", "refresh", "rhs", "solve", "predict", "finish"],
                   help="kernel class timed with CUDA events in the coupled-temperature leg")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-pdr", action="store_true", help="skip the PDR-slab simulation")
    p.add_argument("--thermal-cells", type=int, default=4096,
                   help="cells of the coupled-temperature leg (0 skips it)")
    p.add_argument("--no-tune", action="store_true", help="integrate with the default gather, untuned")
    p.add_argument("--mixed-cells", type=int, default=16384,
                   help="cells of the FP64 vs mixed comparison (0 = skip)")
    p.add_argument("--adjoint-cells", type=int, default=1024,
                   help="cells of the adjoint/forward measurement (0 = skip)")
    p.add_argument("--rhs-cells", type=int, default=4096,
                   help="cells of the rhs_eval / jac_eval format grid (0 = skip)")
    p.add_argument("--budget-s", type=float, default=1200.0,
                   help="auxiliary measurements start only while the run is younger than this")
    p.add_argument("--only", default="",
                   choices=["", "rhs", "mixed", "adjoint", "cpu", "probe", "pdr", "thermal", "single"],
                   help="run one auxiliary measurement alone and print it")
    p.add_argument("--phases", action="store_true",
                   help="refresh-kernel cycles per phase over one integration (phase-clock build)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_cells(cells_per_rank, rank):
    """This rank's slice of one seeded stream of cells_per_rank * world cells
    (weak scaling: every rank integrates its own independent cells)."""
    return slice(rank * cells_per_rank, (rank + 1) * cells_per_rank)


def combine_ranks(units, ms, world, device):
    """(units summed over ranks, the slowest rank's milliseconds); the whole
    job's throughput is units / ms.  No collective on the data path: this is
    the only exchange, after the timed region."""
    if world == 1:
        return float(units), float(ms)
    import torch
    import torch.distributed as dist
    t_max = torch.tensor([ms], dtype=torch.float64, device=device)
    s_sum = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dist.all_reduce(s_sum, op=dist.ReduceOp.SUM)
    return float(s_sum.item()), float(t_max.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def slice_attempts(attempts_est, steps, per=8):
    """Attempts per bench step: attempts_est / steps rounded up to a whole
    number of captured attempt groups (`per` attempts each)."""
    a = -(-max(attempts_est, 1) // max(steps, 1))
    return -(-a // per) * per


# ---------------------------------------------------------------------------
# CPU oracle on a stratified sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def stratified_cells(n=CPU_CELLS):
    """n cells of the headline workload at evenly spaced quantiles of the
    oracle's own step count (rtol 1e-6), taken from the 128 candidates
    (every 128th of the first 16,384 cells) whose counts
    tests/golden/integrate_truth_strat.json stores; cells are independent
    draws of one seeded stream, so these represent all 65,536."""
    with open(STRAT_FILE) as fh:
        s = json.load(fh)
    steps = s["candidate_steps_rtol6"]
    stride = s["pool_cells"] // len(steps)
    order = sorted(range(len(steps)), key=lambda i: (steps[i], i))
    pick = [order[int((i + 0.5) * len(order) / n)] for i in range(n)]
    return [i * stride for i in pick], [steps[i] for i in pick]


_ORACLE_NET = None


def _oracle_cell(args):
    """One sampled cell integrated by the oracle over the whole interval:
    returns (accepted steps, seconds spent integrating)."""
    global _ORACLE_NET
    c, t_end = args
    from oracle import bdf as ob
    from oracle import kinetics as ok
    from oracle import network as on
    from synth import cells as sc
    from synth.workloads import NET_SEED, WORKLOADS
    from synth.network import generate
    w = WORKLOADS[WORKLOAD]
    if _ORACLE_NET is None:
        d = generate(NET_SEED, w.n_s, w.n_r)
        _ORACLE_NET = (d, on.stoichiometry(d))
    d, S = _ORACLE_NET
    T, nH, Av = sc.conditions(4998, c + 1, w.T, w.nH, w.Av)
    k = ok.rate_coefficients(d, T[c:], nH[c:], Av[c:])[:, 0]
    y0 = sc.atomic_start(d, 1)[:, 0]
    t0 = time.time()
    r = ob.integrate_cell(d, k, y0, t_end, ob.BDFOptions(), S)
    return r.steps, time.time() - t0


_ORACLE_THERMAL = None
THERMAL_WORKLOAD = "thermal_470x6000_c16384"


def _oracle_thermal_cell(args):
    """One cell of the coupled-temperature workload integrated by the
    coupled-temperature oracle: (accepted steps, seconds integrating)."""
    global _ORACLE_THERMAL
    c, t_end = args
    from oracle import network as on
    from oracle import thermal as oth
    from synth.workloads import make_thermal
    if _ORACLE_THERMAL is None or _ORACLE_THERMAL[2].shape[0] <= c:
        d, th, nH, Av, z0 = make_thermal(THERMAL_WORKLOAD, cells=max(64, c + 1))
        _ORACLE_THERMAL = (d, th, nH, Av, z0, on.stoichiometry(d))
    d, th, nH, Av, z0, S = _ORACLE_THERMAL
    t0 = time.time()
    r = oth.integrate_cell(d, th, (float(nH[c]), float(Av[c]), 1.0), z0[:, c], t_end, S=S)
    return r.steps, time.time() - t0


def _warm_thermal(_):
    _oracle_thermal_cell((0, 1e-9))
    time.sleep(0.5)
    return 0


def _oracle_single_cell():
    """Config 0 on the oracle: the 32 x 180 network, one cell, 1e6 yr, one
    core (seconds and accepted steps)."""
    from oracle import bdf as ob
    from oracle import kinetics as ok
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["single_cell_32x180"]
    d, T, nH, Av, y0 = make(w.name)
    t0 = time.time()
    k = ok.rate_coefficients(d, T, nH, Av)
    r = ob.integrate_cell(d, k[:, 0], y0[:, 0], w.t_end)
    return {"workload": w.name, "seconds": time.time() - t0, "steps": int(r.steps)}


def _oracle_rhs_config1():
    """Config 1 on the oracle: one right-hand side of each of the 4096 cells
    of the RHS workload (dense S @ R over all cells at once, one process);
    the rate coefficients are inputs, computed before the timed region."""
    from oracle import kinetics as ok
    from oracle import network as on
    from synth.workloads import make
    d, T, nH, Av, y = make("rhs_jac_470x6000_c4096")
    k = ok.rate_coefficients(d, T, nH, Av)
    S = on.stoichiometry(d)
    t0 = time.time()
    ok.rhs(d, k, y, S)
    dt = time.time() - t0
    return {"workload": "rhs_jac_470x6000_c4096", "cells": int(y.shape[1]), "seconds": dt,
            "rhs_per_s": y.shape[1] / dt, "sample": "every cell once, one process"}


def _pool_init():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _warm(_):
    """Imports the oracle and builds the network in a worker, then lingers
    briefly so that every worker of the pool takes one of these tasks."""
    _oracle_cell((0, 1e-9))
    time.sleep(0.5)
    return 0


class OraclePool:
    """One single-threaded oracle process per host core (spawned: no state of
    a CUDA context is inherited)."""

    def __init__(self):
        import multiprocessing as mp
        _pool_init()
        self.cores = host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init)

    def warm(self):
        self.pool.map(_warm, range(2 * self.cores), chunksize=1)

    def run(self, cells, t_end):
        """(accepted steps summed, wall seconds) for integrating `cells`."""
        t0 = time.time()
        res = self.pool.map(_oracle_cell, [(c, t_end) for c in cells], chunksize=1)
        return sum(r[0] for r in res), time.time() - t0

    def run_thermal(self, cells, t_end):
        """(accepted steps summed, wall seconds) for the coupled-temperature
        oracle on `cells` of the coupled-temperature workload."""
        self.pool.map(_warm_thermal, range(2 * self.cores), chunksize=1)
        t0 = time.time()
        res = self.pool.map(_oracle_thermal_cell, [(c, t_end) for c in cells], chunksize=1)
        return sum(r[0] for r in res), time.time() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(t_end, thermal_cells=0):
    """The oracle on the host cores: the headline workload's stratified
    sample (the line's cpu_baseline), and beside it the coupled-temperature
    oracle on the first cells of that workload (thermal_cells > 0) and the
    single-cell 32 x 180 case (config 0) on one core."""
    cells, _ = stratified_cells()
    pool = OraclePool()
    extra = {}
    try:
        pool.warm()                                 # process start-up and imports, untimed
        steps, dt = pool.run(cells, t_end)
        if thermal_cells > 0:
            from synth.workloads import WORKLOADS
            n = min(pool.cores, thermal_cells)
            tsteps, tsec = pool.run_thermal(list(range(n)), WORKLOADS[THERMAL_WORKLOAD].t_end)
            extra["thermal"] = {"value": tsteps / tsec, "unit": UNIT, "cells": n, "seconds": tsec,
                                "sample": f"cells 0-{n - 1} of {THERMAL_WORKLOAD}, whole 1e6 yr at rtol 1e-6, "
                                          "one single-threaded process per core"}
    finally:
        pool.close()
    extra["single_cell"] = _oracle_single_cell()
    extra["rhs"] = _oracle_rhs_config1()
    return {"value": steps / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle", **extra,
            "sample": (f"{len(cells)} cells of {WORKLOAD} stratified by stiffness (evenly spaced quantiles of "
                       f"the oracle's step count among every 128th of the first 16,384 cells), each integrated "
                       f"over the whole 1e6 yr at rtol 1e-6, one single-threaded process per core; "
                       f"{steps} accepted steps in {dt:.1f} s"),
            "cell_steps": steps, "seconds": dt, "steps_per_cell": steps / len(cells)}


def reference_arm(a, rank):
    """The oracle as the reference arm: each step integrates one core's worth
    of the 64 stratified cells over the whole interval (the four quarters of
    the sample in turn)."""
    if rank != 0:
        return
    t_end = a.t_end_yr * YEAR
    cells, _ = stratified_cells()
    pool = OraclePool()
    n = min(pool.cores, len(cells))
    groups = [cells[i::len(cells) // n][:n] for i in range(len(cells) // n)]
    try:
        for _ in range(a.warmup):
            pool.warm()                              # start-up only
        tot_steps, tot_s = 0, 0.0
        for s in range(a.steps):
            st, dt = pool.run(groups[s % len(groups)], t_end)
            tot_steps += st
            tot_s += dt
    finally:
        pool.close()
    v = tot_steps / tot_s
    sample = (f"{n} cells per step from {len(cells)} cells of {WORKLOAD} stratified by stiffness, each "
              f"integrated over the whole 1e6 yr at rtol 1e-6, one single-threaded process per core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_s / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "cells_per_step": n,
                                        "t_end_yr": a.t_end_yr, "rtol": 1e-6, "atol": 1e-20},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(device):
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                 "-i", str(device), "-lms", "200"], stdout=subprocess.PIPE,
                                stderr=subprocess.DEVNULL, text=True)
    except (OSError, ValueError):
        return None


def clocks_stop(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
    if not rows:
        return None
    sm = sorted(float(r[1]) for r in rows)
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for i, nm in enumerate(names):
            if r[5 + i].strip().lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
            "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed(fn, stream):
    """Runs fn() between CUDA events on `stream`; returns (result, ms)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1)


def device_conditions(B, T, nH, Av, dev):
    """Padded device copies of the cell conditions (padding: harmless values)."""
    import torch
    C = len(T)
    ld = B.pad_ld(C)

    def padded(v, fill):
        out = torch.full((ld,), fill, dtype=torch.float64, device=dev)
        out[:C] = torch.tensor(v, dtype=torch.float64, device=dev)
        return out

    return padded(T, 100.0), padded(nH, 1.0), padded(Av, 0.0)


def gpu_inputs(B, net, d, T, nH, Av, y0, dev):
    """Device k' (evaluated by sm_rates_eval) and y0 for C cells."""
    import torch
    C = y0.shape[1]
    ld = B.pad_ld(C)
    Td, nHd, Avd = device_conditions(B, T, nH, Av, dev)
    kd = torch.empty((d.n_r, ld), dtype=torch.float64, device=dev)
    net.rates_eval(Td, nHd, Avd, kd, C)
    y0d = torch.zeros((d.n_s, ld), dtype=torch.float64, device=dev)
    y0d[:, :C] = torch.tensor(y0, dtype=torch.float64, device=dev)
    return kd, y0d


def integrate_timed(B, st, kd, y0d, t_end, C, stats, stream):
    """One whole integration through sm_integrate after an untimed 8-attempt
    start (graph capture); returns (final y on the host, stats, ms)."""
    st.init(kd, y0d, t_end, C)
    st.step(kd, 8)
    yd = y0d.clone()
    _, ms = timed(lambda: st.integrate(kd, yd, t_end, C, stats), stream)
    return yd[:, :C].cpu().numpy(), B.stats_to_numpy(stats), ms


def species_error(y, truth, names):
    """Per species over the sampled cells: largest and median relative error
    for abundances above 1e-20 in the reference solution."""
    import numpy as np
    live = truth > 1e-20
    rel = np.where(live, np.abs(y - truth) / np.where(live, truth, 1.0), np.nan)
    ok = live.any(axis=1)
    mx = np.array([np.nanmax(r) if o else -1.0 for r, o in zip(rel, ok)])
    med = np.array([np.nanmedian(r) if o else -1.0 for r, o in zip(rel, ok)])
    worst = np.argsort(-mx)[:5]
    return {"species_scored": int(ok.sum()), "max_rel": float(mx[ok].max()),
            "median_of_species_max": float(np.median(mx[ok])),
            "median_of_species_median": float(np.median(med[ok])),
            "worst": [[names[i], float(mx[i]), float(med[i])] for i in worst],
            "per_species": {names[i]: [float(mx[i]), float(med[i])] for i in range(len(names)) if ok[i]}}


def fp64_vs_mixed(B, C, dev):
    """The mixed-precision workload: C cells (the first C of the headline
    stream) integrated to 1e6 yr at rtol 1e-6 in the plain FP64 mode and in
    the mixed mode, each timed with CUDA events over one whole integration;
    per-species max / median relative error of both (and of the oracle's own
    rtol-1e-6 solution) against the oracle's rtol-1e-10 solution on the 32
    stiffness-stratified cells stored in tests/golden (written by
    make_integrate_truth.py, which calls only the oracle)."""
    import numpy as np
    import torch
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS[MIXED_WORKLOAD]
    d, T, nH, Av, y0 = make(MIXED_WORKLOAD, cells=C)
    with open(STRAT_FILE) as fh:
        ref = json.load(fh)
    cells = [c for c in ref["cells"] if c < C]
    sel = [i for i, c in enumerate(ref["cells"]) if c < C]
    truth = np.array(ref["y"]).T[:, sel]
    net = B.Network(d, dev.index or 0)
    kd, y0d = gpu_inputs(B, net, d, T, nH, Av, y0, dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": MIXED_WORKLOAD, "cells": C, "t_end_yr": w.t_end / YEAR, "rtol": w.rtol,
           "reference": "oracle BDF at rtol 1e-10 (tests/golden/integrate_truth_strat.json)",
           "sampled_cells": cells,
           "oracle_rtol6": species_error(np.array(ref["y_rtol6"]).T[:, sel], truth, d.names)}
    for prec in ("fp64", "mixed"):
        st = B.State(net, C, precision=prec)
        stats = B.stats_tensor(C, dev)
        y, s, ms = integrate_timed(B, st, kd, y0d, w.t_end, C, stats, stream)
        st.close()
        out[prec] = {"value": float(s["steps"].sum()) / (ms * 1e-3), "unit": UNIT, "ms": ms,
                     "steps_per_cell": float(s["steps"].mean()), "max_steps": int(s["steps"].max()),
                     "newton_per_step": float(s["newton_iters"].sum() / max(s["steps"].sum(), 1)),
                     "jac_per_step": float(s["jac_evals"].sum() / max(s["steps"].sum(), 1)),
                     "cells_ok": int((s["status"] == 0).sum()),
                     "error_vs_oracle": species_error(y[:, cells], truth, d.names)}
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    for key in ("fp64", "mixed", "oracle_rtol6"):
        e = out[key] if key == "oracle_rtol6" else out[key]["error_vs_oracle"]
        e.pop("per_species")
    net.close()
    return out


RHS_GRID = [("crs", "none", 1, 1), ("crs", "nnz", 1, 1), ("crs", "rcm", 1, 1), ("coo", "none", 1, 1),
            ("coo", "rcm", 1, 1), ("ccs", "none", 1, 1), ("ccs", "rcm", 1, 1), ("sell", "none", 4, 1),
            ("sell", "nnz", 8, 64), ("sell", "none", 32, 470), ("sell", "rcm", 8, 64)]


def rhs_jac_grid(B, C, dev, peaks):
    """rhs_eval for every storage format x row order of the grid and jac_eval,
    on the RHS workload (470 x 6000, C cells, log-uniform abundances): median
    of 20 CUDA-event-timed calls, L2 flushed (256 MB write) before each.
    Algorithmic bytes and FP64 flops per cell come from sm_net_get_info; the
    binding ceiling is min(HBM bandwidth x intensity, FP64 peak)."""
    import numpy as np
    import torch
    from synth.workloads import make
    d, T, nH, Av, y = make("rhs_jac_470x6000_c4096", cells=C)
    net = B.Network(d, dev.index or 0)
    info = net.info()
    kd, yd = gpu_inputs(B, net, d, T, nH, Av, y, dev)
    fd = torch.empty_like(yd)
    Jd = torch.empty((info["nnz_J"], yd.shape[1]), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.int8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def med(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(20):
            flush.zero_()
            ts.append(timed(fn, stream)[1])
        return float(np.median(ts))

    def row(kind, ms, nbytes, flops):
        gbs = nbytes * C / (ms * 1e-3) / 1e9
        tf = flops * C / (ms * 1e-3) / 1e12
        ceiling = min(peaks["hbm_gbs"] * 1e9 * flops / nbytes / 1e12, peaks["fp64_tflops"])
        return {"kind": kind, "us": ms * 1e3, "GB_s": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                "fp64_TF_s": tf, "fp64_frac": tf / peaks["fp64_tflops"], "binding_frac": tf / ceiling}

    out = []
    for fmt in RHS_GRID:
        net.set_format(*fmt)
        ms = med(lambda: net.rhs_eval(kd, yd, fd, C))
        out.append(row("rhs " + "/".join(str(x) for x in fmt), ms, info["rhs_bytes"], info["rhs_flops"]))
    # the conventional right-hand side (generated per network, one explicit
    # expression per species), timed the same way; same per-cell work units
    conv = None
    try:
        from paper_2312_04998_gb300 import unrolled
        t0 = time.time()
        u = unrolled.Unrolled(d)
        build_s = time.time() - t0
        ms = med(lambda: u.rhs_eval(kd, yd, fd, C))
        out.append(row("rhs conventional (generated)", ms, info["rhs_bytes"], info["rhs_flops"]))
        conv = {"us": ms * 1e3, "kernels": u.n_kernels, "terms": u.n_terms, "build_s": build_s}
    except Exception as exc:  # noqa: BLE001
        conv = {"error": f"{type(exc).__name__}: {exc}"}
    net.set_format("crs", "none", 1, 1)
    ms = med(lambda: net.jac_eval(kd, yd, Jd, C))
    out.append(row("jac", ms, info["jac_bytes"], info["jac_flops"]))
    net.sync()
    net.close()
    best = max((r for r in out if r["kind"].startswith("rhs")), key=lambda r: r["binding_frac"])
    crs = min((r for r in out if r["kind"].startswith("rhs crs")), key=lambda r: r["us"])
    if conv and "us" in conv:
        conv["crs_speedup"] = conv["us"] / crs["us"]
    return {"workload": "rhs_jac_470x6000_c4096", "cells": C, "l2": "flushed before every call",
            "rhs_bytes_per_cell": info["rhs_bytes"], "rhs_flops_per_cell": info["rhs_flops"],
            "jac_bytes_per_cell": info["jac_bytes"], "jac_flops_per_cell": info["jac_flops"],
            "peaks": peaks, "best_rhs": best["kind"], "best_rhs_binding_frac": best["binding_frac"],
            "conventional": conv,
            "rows": out}


def pdr_slab(B, dev, precisions=("mixed", "fp64")):
    """The paper's benchmark geometry with the synthetic network: the 128-cell
    PDR slab (n_H 1e3, T 50 K, FUV field 1e5 on the photorates, A_V 1e-3 to
    20 on a log grid, atomic start) integrated to 30 Myr, as one whole
    simulation timed with CUDA events (sm_rates_eval_chi + sm_integrate) after
    an untimed run that captures the graphs.  The paper's own number for its
    PDR run (UMIST network, 468 x 6175, 2x Xeon E5-2650 v3, CRS, serial):
    232 s, context only."""
    import numpy as np
    import torch
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["pdr_slab_470x6000_c128"]
    d, T, nH, Av, y0 = make(w.name)
    C = y0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, dev.index or 0)
    Td, nHd, Avd = device_conditions(B, T, nH, Av, dev)
    chid = torch.ones(ld, dtype=torch.float64, device=dev)
    chid[:C] = w.chi
    kd = torch.empty((d.n_r, ld), dtype=torch.float64, device=dev)
    y0d = torch.zeros((d.n_s, ld), dtype=torch.float64, device=dev)
    y0d[:, :C] = torch.tensor(y0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": w.name, "cells": C, "t_end_myr": w.t_end / YEAR / 1e6, "chi": w.chi,
           "paper_cpu_s": 232.0}
    for prec in precisions:
        st = B.State(net, C, precision=prec)
        stats = B.stats_tensor(C, dev)
        yd = y0d.clone()

        def run():
            net.rates_eval_chi(Td, nHd, Avd, chid, kd, C)
            yd.copy_(y0d)
            return st.integrate(kd, yd, w.t_end, C, stats)

        run()
        code, ms = timed(run, stream)
        s = B.stats_to_numpy(stats)
        out[prec] = {"seconds": ms * 1e-3, "cell_steps_per_s": float(s["steps"].sum()) / (ms * 1e-3),
                     "steps_per_cell": float(s["steps"].mean()), "max_steps": int(s["steps"].max()),
                     "cells_ok": int((s["status"] == 0).sum()), "status": int(code)}
        st.close()
    net.close()
    return out


def single_cell(B, dev):
    """Config 0: the 32 x 180 network, one cell (T 10 K, n_H 1e4, A_V 5,
    atomic start) to 1e6 yr at rtol 1e-6: GPU wall time of sm_rates_eval +
    sm_integrate (FP64, after an untimed run that captures the graphs); the
    oracle's time for the same cell is in cpu_baseline["single_cell"]."""
    import torch
    from synth.workloads import WORKLOADS, make
    w = WORKLOADS["single_cell_32x180"]
    d, T, nH, Av, y0 = make(w.name)
    ld = B.pad_ld(1)
    net = B.Network(d, dev.index or 0)
    Td, nHd, Avd = device_conditions(B, T, nH, Av, dev)
    kd = torch.empty((d.n_r, ld), dtype=torch.float64, device=dev)
    y0d = torch.zeros((d.n_s, ld), dtype=torch.float64, device=dev)
    y0d[:, :1] = torch.tensor(y0, dtype=torch.float64, device=dev)
    st = B.State(net, 1)
    stats = B.stats_tensor(1, dev)
    yd = y0d.clone()

    def run():
        net.rates_eval(Td, nHd, Avd, kd, 1)
        yd.copy_(y0d)
        return st.integrate(kd, yd, w.t_end, 1, stats)

    run()
    code, ms = timed(run, torch.cuda.current_stream(dev))
    s = B.stats_to_numpy(stats)
    st.close()
    net.close()
    return {"workload": w.name, "gpu_ms": ms, "steps": int(s["steps"][0]), "status": int(code)}


def thermal_leg(B, dev, cells=4096, precisions=("mixed",), time_kernel="none"):
    """Coupled gas temperature (NEXT row: the energy equation as one more BDF
    component, k'(T) re-evaluated inside every Newton iteration): the first
    `cells` cells of the coupled-temperature workload integrated to 1e6 yr
    as one whole simulation timed with CUDA events (sm_state_set_cells +
    sm_integrate, after an untimed run that captures the graphs), beside the
    same cells at fixed T (the coupled-temperature oracle's time is in
    cpu_baseline["thermal"])."""
    import numpy as np
    import torch
    from synth.workloads import WORKLOADS, make_thermal
    w = WORKLOADS[THERMAL_WORKLOAD]
    d, th, nH, Av, z0 = make_thermal(w.name, cells=cells)
    C = z0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, dev.index or 0)
    net.set_thermal(th)
    vec = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    nHd, Avd = vec(nH), vec(Av)
    z0d = torch.zeros((d.n_s, ld), dtype=torch.float64, device=dev)
    z0d[:, :C] = vec(z0)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": w.name, "cells": C, "t_end_yr": w.t_end / YEAR}
    for prec in precisions:
        st = B.State(net, C, precision=prec, timing_kind=time_kernel)
        st.set_cells(nHd, Avd, None, C)
        stats = B.stats_tensor(C, dev)
        zd = z0d.clone()

        def run():
            zd.copy_(z0d)
            return st.integrate(None, zd, w.t_end, C, stats)

        run()
        st.timing_reset()
        code, ms = timed(run, stream)
        _, class_ms, class_n = st.timing()
        s = B.stats_to_numpy(stats)
        T1 = zd[th.t_index, :C].cpu().numpy()
        out[prec] = {"seconds": ms * 1e-3, "cell_steps_per_s": float(s["steps"].sum()) / (ms * 1e-3),
                     "steps_per_cell": float(s["steps"].mean()), "max_steps": int(s["steps"].max()),
                     "newton_per_step": float(s["newton_iters"].sum()) / max(float(s["steps"].sum()), 1.0),
                     "cells_ok": int((s["status"] == 0).sum()), "status": int(code),
                     "T_final_K": {"min": float(T1.min()), "median": float(np.median(T1)), "max": float(T1.max())}}
        if time_kernel != "none":
            out[prec]["timed_class"] = {"kind": time_kernel, "ms": class_ms, "launches": class_n}
        st.close()
    net.close()
    # the same cells with T held at its initial value (the paper's fixed-T
    # chemistry step): the chemical network alone, k' from each cell's T
    from synth.workloads import make
    d0, T0, _, _, y0 = make(w.name, cells=cells)
    net0 = B.Network(d0, dev.index or 0)
    Td, nHd0, Avd0 = device_conditions(B, T0, nH, Av, dev)
    kd = torch.empty((d0.n_r, ld), dtype=torch.float64, device=dev)
    y0d = torch.zeros((d0.n_s, ld), dtype=torch.float64, device=dev)
    y0d[:, :C] = vec(y0)
    st = B.State(net0, C, precision=precisions[0])
    stats = B.stats_tensor(C, dev)
    yd = y0d.clone()

    def run0():
        net0.rates_eval(Td, nHd0, Avd0, kd, C)
        yd.copy_(y0d)
        return st.integrate(kd, yd, w.t_end, C, stats)

    run0()
    code, ms = timed(run0, stream)
    s = B.stats_to_numpy(stats)
    out["fixed_T_" + precisions[0]] = {"seconds": ms * 1e-3,
                                       "cell_steps_per_s": float(s["steps"].sum()) / (ms * 1e-3),
                                       "steps_per_cell": float(s["steps"].mean()), "status": int(code)}
    st.close()
    net0.close()
    return out


def peaks_(B, dev):
    """HBM: the measured copy bandwidth (MEASURED_PEAKS.json); FP64 / FP32:
    unit counts x clock, with this run's FMA-probe rates beside them."""
    hbm, src = 6782.4, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm, src = float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json"
    except (OSError, ValueError, KeyError):
        pass
    out = {"hbm_gbs": hbm, "hbm_source": src, "fp64_tflops": PEAK_FP64, "fp32_tflops": PEAK_FP32,
           "alu_source": "152 SMs x 2.07 GHz x (FP64 4 | FP32 256) flops/clk"}
    try:
        out["probe_fp64_tflops"] = B.probe_fma(dev.index or 0, True)
        out["probe_fp32_tflops"] = B.probe_fma(dev.index or 0, False)
    except Exception as exc:  # noqa: BLE001
        out["probe_error"] = f"{type(exc).__name__}: {exc}"
    return out


def adjoint_measurement(B, C, dev):
    """Discrete adjoint on the adjoint workload (470 x 6000, 1e5 yr, FP64,
    checkpoints every 16 steps): one recorded forward integrate and one reverse
    sweep for eight log-abundance targets, each timed with CUDA events.
    Targets: the eight species above 1e-12 in the largest share of cells at
    t_end (cotangent 1/y there, 0 in cells where the species is below)."""
    import numpy as np
    import torch
    from synth.workloads import WORKLOADS, make
    name = "adjoint_470x6000_c1024"
    d, T, nH, Av, y0 = make(name, cells=C)
    t_end = WORKLOADS[name].t_end
    net = B.Network(d, dev.index or 0)
    st = B.State(net, C, precision="fp64", record_steps=8000)
    kd, y0d = gpu_inputs(B, net, d, T, nH, Av, y0, dev)
    stats = B.stats_tensor(C, dev)
    stream = torch.cuda.current_stream(dev)
    yN, s, f_ms = integrate_timed(B, st, kd, y0d, t_end, C, stats, stream)
    code_f = int((s["status"] != 0).any())
    ld = B.pad_ld(C)
    frac = (yN > 1e-12).mean(axis=1)
    targets = np.argsort(-frac, kind="stable")[:8]
    cot = np.zeros((8, d.n_s, ld))
    for v, t in enumerate(targets):
        cot[v, t, :C] = np.where(yN[t] > 1e-12, 1.0 / np.maximum(yN[t], 1e-300), 0.0)
    cot_d = torch.tensor(cot, dtype=torch.float64, device=dev)
    grad = torch.zeros((8, d.n_r, ld), dtype=torch.float64, device=dev)
    astat = torch.zeros(ld, dtype=torch.int32, device=dev)
    l0, _, _ = st.timing()
    code_a, a_ms = timed(lambda: st.adjoint(kd, cot_d, grad, astat), stream)
    l1, _, _ = st.timing()
    out = {"workload": name, "cells": C, "t_end_yr": t_end / YEAR, "n_cot": 8,
           "targets": [d.names[t] for t in targets], "forward_ms": f_ms, "adjoint_ms": a_ms,
           "adjoint_per_forward": a_ms / f_ms, "adjoint_ms_per_target": a_ms / 8,
           "steps_per_cell": float(s["steps"].mean()), "max_steps": int(s["steps"].max()),
           "cells_ok": int((astat.cpu().numpy()[:C] == 0).sum()), "forward_partial": code_f,
           "adjoint_status": int(code_a), "adjoint_launches": int(l1 - l0),
           "checkpoint_every": B.CHECKPOINT_EVERY}
    st.close()
    net.close()
    return out


def phase_profile(B, a, dev):
    """Refresh-kernel cycles per phase, per refreshed cell, over one whole
    integration of the first a.cells cells of the headline workload (thread
    0 of each CTA, between the barriers that end the phases; the phase-clock
    build of the library)."""
    import numpy as np
    import torch
    from synth.workloads import make
    d, T, nH, Av, y0 = make(WORKLOAD, cells=a.cells)
    net = B.Network(d, dev.index or 0)
    kd, y0d = gpu_inputs(B, net, d, T, nH, Av, y0, dev)
    st = B.State(net, a.cells, precision=a.precision)
    stats = B.stats_tensor(a.cells, dev)
    st.init(kd, y0d, a.t_end_yr * YEAR, a.cells)
    st.step(kd, 8)
    torch.cuda.synchronize()
    B.phase_cycles(dev.index or 0, reset=True)
    yd = y0d.clone()
    st.integrate(kd, yd, a.t_end_yr * YEAR, a.cells, stats)
    torch.cuda.synchronize()
    cyc = B.phase_cycles(dev.index or 0)
    cells = max(cyc[15], 1.0)
    per = cyc[:len(B.PHASE_NAMES)] / cells
    tot = per.sum()
    return {"what": "refresh kernel cycles per refreshed cell, by phase (thread 0 of each CTA)",
            "workload": WORKLOAD, "cells": a.cells, "precision": a.precision, "refreshed_cells": int(cyc[15]),
            "total_cycles_per_cell": float(tot),
            "phases": [[nm, float(v), float(v / tot)] for nm, v in zip(B.PHASE_NAMES, per)]}


def kernel_source_hash():
    """Hash of the integrator's kernel source (integrate.cu) with comments and
    whitespace removed, so that a comment edit keeps the key of a capture."""
    import re
    with open(os.path.join(ROOT, "paper_2312_04998_gb300", "csrc", "integrate.cu")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)      # block comments
    src = re.sub(r"//[^\n]*", " ", src)                    # line comments
    src = re.sub(r"\s+", " ", src).strip()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def roofline(info, s, kind, precision, kern_ms, kern_n, peaks):
    """Roofline of the timed kernel class over the timed integration."""
    if not kern_n:
        return None
    refreshes = float(s["jac_evals"].sum())
    newton = float(s["newton_iters"].sum())
    if kind == "refresh":
        # per refreshed cell: J gather (2 flops per term) + M assembly + LU
        unit = 2.0 * info["n_jac_terms"] + 2.0 * info["nnz_J"] + float(info["lu_flops"])
        units = refreshes
        fp32 = precision != "fp64"
    elif kind == "rhs":
        unit, units, fp32 = info["rhs_flops"], newton, False
    elif kind == "solve":
        # per Newton iteration of a cell: the packed factors once, and the
        # residual / update vectors (y, psi, f, w, wf read, y written)
        esz = 8 if precision == "fp64" else 4
        unit = esz * info["lu_packed"] + 8.0 * 6 * info["n_s"]
        units = newton
        per_launch_units = units / kern_n
        ach = unit * per_launch_units / (kern_ms * 1e-3 / kern_n) / 1e9
        tr = TRAFFIC.get((kind, precision, kernel_source_hash()))
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None if tr is None else tr * per_launch_units,
                "kernel": "solve (packed factors, warp per cell)", "avg_launch_ms": kern_ms / kern_n,
                "timed_launches": kern_n, "total_ms": kern_ms, "units_per_launch": per_launch_units,
                "bytes_per_unit": unit, "unit_name": "cell Newton iteration", "peak_source": peaks["hbm_source"]}
    else:
        return None
    per_launch_units = units / kern_n
    avg_s = kern_ms * 1e-3 / kern_n
    ach = unit * per_launch_units / avg_s / 1e12
    pk = peaks["fp32_tflops"] if fp32 else peaks["fp64_tflops"]
    tr = TRAFFIC.get((kind, precision, kernel_source_hash()))
    return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "traffic": None if tr is None else tr * per_launch_units,
            "kernel": f"{kind} ({'FP32' if fp32 else 'FP64'} pipe)", "avg_launch_ms": kern_ms / kern_n,
            "timed_launches": kern_n, "total_ms": kern_ms, "units_per_launch": per_launch_units,
            "flops_per_unit": unit, "unit_name": "refreshed cell" if kind == "refresh" else "cell RHS",
            "peak_source": peaks["alu_source"]}


def main():
    t_start = time.time()
    a = args_()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return reference_arm(a, rank)
    if a.only == "cpu":
        print(json.dumps(cpu_baseline(a.t_end_yr * YEAR, max(a.thermal_cells, 0))))
        return
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_04998_gb300 import binding as B
    from synth.workloads import make
    if a.phases:
        from paper_2312_04998_gb300 import build as _bld
        _bld.build(phase_clocks=True)
        B.use_phase_build()
        print(json.dumps(phase_profile(B, a, torch.device("cuda", local))))
        return

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if a.only:
        fn = {"rhs": lambda: rhs_jac_grid(B, a.rhs_cells, dev, peaks_(B, dev)),
              "mixed": lambda: fp64_vs_mixed(B, a.mixed_cells, dev),
              "adjoint": lambda: adjoint_measurement(B, a.adjoint_cells, dev),
              "probe": lambda: peaks_(B, dev), "pdr": lambda: pdr_slab(B, dev),
              "thermal": lambda: thermal_leg(B, dev, a.thermal_cells, ("mixed",), a.thermal_time_kernel),
              "single": lambda: single_cell(B, dev)}[a.only]
        if rank == 0:
            print(json.dumps(fn()))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    C = a.cells
    t_end = a.t_end_yr * YEAR
    # every rank takes its own slice of one seeded stream of cells
    d, T, nH, Av, y0 = make(WORKLOAD, cells=C * world)
    sl = rank_cells(C, rank)
    T, nH, Av, y0 = T[sl], nH[sl], Av[sl], np.ascontiguousarray(y0[:, sl])
    net = B.Network(d, local)
    info = net.info()
    ld = B.pad_ld(C)
    Td, nHd, Avd = device_conditions(B, T, nH, Av, dev)
    y0d = torch.zeros((d.n_s, ld), dtype=torch.float64, device=dev)
    y0d[:, :C] = torch.tensor(y0, dtype=torch.float64, device=dev)
    kd = torch.empty((d.n_r, ld), dtype=torch.float64, device=dev)
    # measured choice of the traversals (untimed set-up): the standalone
    # rhs_eval format and the integrator's gather (row order, cells per CTA)
    tune = None
    if not a.no_tune:
        net.rates_eval(Td, nHd, Avd, kd, C)
        fscr = torch.empty_like(y0d)
        tune = net.autotune(kd, y0d, fscr, C)
        del fscr
    state = B.State(net, C, precision=a.precision, timing_kind=a.time_kernel,
                    refresh_ctas_per_sm=a.refresh_per_sm)
    stats = B.stats_tensor(C, dev)
    per = state.opts.attempts_per_sync
    A = slice_attempts(a.attempts_est, a.steps, per)

    def step(s):
        """Bench step s of K: a slice of the integration (see the module
        docstring)."""
        if s == 0:
            net.rates_eval(Td, nHd, Avd, kd, C)
            state.init(kd, y0d, t_end, C)
        if s < a.steps - 1:
            state.step(kd, A)
            return 0
        n = 0
        while state.read() > 0 and n < MAX_TAIL_ATTEMPTS:
            state.step(kd, per)
            n += per
        return n

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up: the first slices of a separate integration of the same batch
    net.rates_eval(Td, nHd, Avd, kd, C)
    state.init(kd, y0d, t_end, C)
    for _ in range(a.warmup):
        state.step(kd, A)
    torch.cuda.synchronize()
    clk = clocks_start(local)
    barrier()
    torch.cuda.synchronize()
    state.timing_reset()
    l_before, _, _ = state.timing()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tail = 0
    for s in range(a.steps):
        tail = step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clocks_stop(clk)
    ms = e0.elapsed_time(e1)
    l_after, kern_ms, kern_n = state.timing()
    launches = l_after - l_before + 1          # + the rates_eval of step 1
    state.read(stats=stats)
    s = B.stats_to_numpy(stats)
    cell_steps = int(s["steps"].sum())
    attempts = int((s["steps"] + s["rejects"] + s["conv_fails"]).max())
    cell_steps_all, ms_max = combine_ranks(cell_steps, ms, world, dev)
    value = cell_steps_all / (ms_max * 1e-3)

    # end to end through the public calls with host buffers: one whole
    # integration (inputs copied in, solution and per-cell results copied out)
    e2e = None
    if not a.no_e2e:
        hT = torch.tensor(T, dtype=torch.float64).pin_memory()
        hnH = torch.tensor(nH, dtype=torch.float64).pin_memory()
        hAv = torch.tensor(Av, dtype=torch.float64).pin_memory()
        hy0 = torch.zeros((d.n_s, ld), dtype=torch.float64)
        hy0[:, :C] = torch.tensor(y0)
        hy0 = hy0.pin_memory()
        hy = torch.empty_like(hy0).pin_memory()
        hst = torch.empty(stats.numel(), dtype=torch.uint8).pin_memory()
        yd = torch.empty_like(y0d)
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        Td[:C].copy_(hT, non_blocking=True)
        nHd[:C].copy_(hnH, non_blocking=True)
        Avd[:C].copy_(hAv, non_blocking=True)
        yd.copy_(hy0, non_blocking=True)
        net.rates_eval(Td, nHd, Avd, kd, C)
        state.integrate(kd, yd, t_end, C, stats)
        hy.copy_(yd, non_blocking=True)
        hst.copy_(stats, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e_ms = f0.elapsed_time(f1)
        e_steps = int(np.frombuffer(hst.numpy().tobytes(), dtype=B.CELL_STATS_DTYPE)["steps"].sum())
        e_steps, e_ms = combine_ranks(e_steps, e_ms, world, dev)
        e2e = {"value": e_steps / (e_ms * 1e-3), "unit": UNIT, "steps": 1,
               "h2d_bytes_per_step": int(3 * C * 8 + hy0.numel() * 8),
               "d2h_bytes_per_step": int(hy.numel() * 8 + hst.numel()),
               "what": "one whole integration of the batch: host conditions and y0 copied in, "
                       "sm_rates_eval + sm_integrate, solution and per-cell results copied out"}
    state.close()
    if rank != 0:
        return

    def aux(fn, *args):
        # the auxiliary measurements must not cost the main line
        if time.time() - t_start > a.budget_s:
            return {"skipped": f"run older than --budget-s {a.budget_s:.0f} s"}
        try:
            return fn(*args)
        except Exception as exc:  # noqa: BLE001
            return {"error": f"{type(exc).__name__}: {exc}"}

    peaks = aux(peaks_, B, dev)
    roof = roofline(info, s, a.time_kernel, a.precision, kern_ms, kern_n, peaks)
    if roof is not None:
        roof["peak_kind"] = "derived (unit counts x max clock), timed inside a long step"
    mixed = aux(fp64_vs_mixed, B, a.mixed_cells, dev) if a.mixed_cells > 0 else None
    adj = aux(adjoint_measurement, B, a.adjoint_cells, dev) if a.adjoint_cells > 0 else None
    rhs = aux(rhs_jac_grid, B, a.rhs_cells, dev, peaks) if a.rhs_cells > 0 else None
    pdr = None if a.no_pdr else aux(pdr_slab, B, dev)
    therm = None if a.thermal_cells <= 0 else aux(thermal_leg, B, dev, a.thermal_cells, ("mixed",),
                                                 a.thermal_time_kernel)
    single = aux(single_cell, B, dev)
    cpu = None if a.no_cpu else aux(cpu_baseline, t_end, max(a.thermal_cells, 0))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f64+f32", "tf32": "f64+f32+tf32"}[a.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells_per_gpu": C, "n_s": d.n_s, "n_r": d.n_r,
                   "t_end_yr": a.t_end_yr, "rtol": 1e-6, "atol": 1e-20, "precision": a.precision,
                   "step": f"one slice of one whole integration: {A} attempts per step, the last step until "
                           f"every cell reached t_end ({tail} attempts)",
                   "l2": "inputs larger than L2 (k' alone is 3.1 GB per GPU)",
                   "tuned": tune},
        "stats": {"cell_steps": cell_steps, "steps_per_cell": float(s["steps"].mean()),
                  "max_steps": int(s["steps"].max()), "attempts": attempts,
                  "newton_per_cell": float(s["newton_iters"].mean()),
                  "jac_per_cell": float(s["jac_evals"].mean()),
                  "rejects_per_cell": float(s["rejects"].mean()),
                  "cells_ok": int((s["status"] == 0).sum()),
                  # per-cell distributions (config 2 asks for the histograms):
                  # deciles 0, 10, ..., 100 % over the cells
                  "deciles": {key: np.percentile(s[key], np.arange(0, 101, 10)).round(1).tolist()
                              for key in ("steps", "rejects", "newton_iters", "jac_evals")}},
        "gpu_launches": int(launches),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "fp64_vs_mixed": mixed, "adjoint": adj, "rhs_jac": rhs, "pdr_slab": pdr, "thermal": therm, "single_cell": single, "peaks": peaks,
        "wall_s": time.time() - t_start,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
