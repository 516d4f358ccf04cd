"""GPU parity of rates_eval, rhs_eval (all formats and orders) and jac_eval
against the oracle, through the C ABI.

Tolerances:
* k': rtol 1e-13.  The library evaluates exp(log alpha + beta log(T/300) -
  gamma/T) n_H; with |argument| <= 82 for the workload ranges (|log alpha| <=
  27.7, |beta log(T/300)| <= 3.4, gamma/T <= 50) its rounding is bounded by a
  few times 82 * 2^-53 ~ 3e-14 relative, the oracle's own pow/exp form by less.
* f and J: |gpu - oracle| <= 1e-12 * sum_j |S_ij term_j| (+1e-300): both are
  FP64 sums of the same terms in different orders, whose difference is bounded
  by (terms per row) * 2^-53 * sum|terms| < 3e-13 sum|terms| here.
"""
import numpy as np
import pytest

from oracle import kinetics as ok
from oracle import network as on
from synth import cells as sc
from synth import network as sn

pytestmark = pytest.mark.gpu

RTOL_K = 1e-13
RTOL_F = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "these tests need a CUDA GPU"
    return _t


@pytest.fixture(scope="module")
def B(torch):
    from paper_2312_04998_gb300 import build
    build.build()
    from paper_2312_04998_gb300 import binding
    return binding


def dev_mat(torch, a, ld, fill=np.nan):
    """[n][ld] device tensor whose first a.shape[1] columns hold a; padding
    columns hold `fill` so that writes outside [0, C) are detectable."""
    n, C = a.shape
    h = np.full((n, ld), fill)
    h[:, :C] = a
    return torch.tensor(h, dtype=torch.float64, device="cuda")


def setup_case(seed_net, n_s, n_r, C, seed_cells=4998):
    d = sn.generate(seed_net, n_s, n_r)
    T, nH, Av = sc.conditions(seed_cells, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    y = sc.loguniform_abundances(d, seed_cells, C)
    return d, T, nH, Av, y


CASES = [(2312, 32, 180, 37), (2312, 470, 6000, 100)]


@pytest.mark.parametrize("case", CASES)
def test_rates_parity(torch, B, case):
    d, T, nH, Av, _ = setup_case(*case)
    C = case[3]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    kd = torch.full((d.n_r, ld), np.nan, dtype=torch.float64, device="cuda")
    tt = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    net.rates_eval(tt(T), tt(nH), tt(Av), kd, C)
    net.sync()
    k = kd.cpu().numpy()
    ref = ok.rate_coefficients(d, T, nH, Av)
    assert np.all(np.abs(k[:, :C] - ref) <= RTOL_K * np.abs(ref))
    assert np.all(np.isnan(k[:, C:])), "padding columns must stay untouched"


FORMATS = [("crs", "none", 1, 1), ("crs", "nnz", 1, 1), ("crs", "rcm", 1, 1),
           ("coo", "none", 1, 1), ("ccs", "none", 1, 1), ("ccs", "rcm", 1, 1),
           ("sell", "none", 4, 1), ("sell", "nnz", 4, 1), ("sell", "none", 8, 64),
           ("sell", "rcm", 32, 470), ("sell", "none", 1, 1)]


@pytest.fixture(scope="module")
def rhs_case(torch, B):
    d, T, nH, Av, y = setup_case(2312, 470, 6000, 100)
    k = ok.rate_coefficients(d, T, nH, Av)
    return d, k, y, ok.rhs(d, k, y), ok.rhs_scale(d, k, y)


@pytest.mark.parametrize("fmt", FORMATS)
def test_rhs_parity_formats(torch, B, rhs_case, fmt):
    d, k, y, ref, scale = rhs_case
    C = y.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    net.set_format(*fmt)
    kd, yd = dev_mat(torch, k, ld, 0.0), dev_mat(torch, y, ld, 0.0)
    fd = torch.full((d.n_s, ld), -7.0, dtype=torch.float64, device="cuda")
    net.rhs_eval(kd, yd, fd, C)
    net.sync()
    f = fd.cpu().numpy()
    err = np.abs(f[:, :C] - ref)
    assert np.all(err <= RTOL_F * scale + 1e-300), (fmt, float((err / (scale + 1e-300)).max()))
    if fmt[0] in ("crs", "sell"):
        assert np.all(f[:, C:] == -7.0), "gather formats write only the first C columns"


@pytest.mark.parametrize("case", CASES)
def test_jac_parity(torch, B, case):
    d, T, nH, Av, y = setup_case(*case)
    C = case[3]
    ld = B.pad_ld(C)
    k = ok.rate_coefficients(d, T, nH, Av)
    net = B.Network(d, 0)
    ptr = net.export(B.X_JPAT_PTR)
    col = net.export(B.X_JPAT_COL)
    Jd = torch.full((len(col), ld), np.nan, dtype=torch.float64, device="cuda")
    net.jac_eval(dev_mat(torch, k, ld, 0.0), dev_mat(torch, y, ld, 0.0), Jd, C)
    net.sync()
    J = Jd.cpu().numpy()
    S = on.stoichiometry(d)
    rows = np.repeat(np.arange(d.n_s), np.diff(ptr))
    for c in range(0, C, max(1, C // 12)):
        Jo = ok.jacobian(d, k[:, c], y[:, c], S)
        sc_ = ok.jacobian_scale(d, k[:, c], y[:, c], S)
        g = J[:, c]
        assert np.all(np.abs(g - Jo[rows, col]) <= RTOL_F * sc_[rows, col] + 1e-300)
        mask = np.ones_like(Jo, dtype=bool)
        mask[rows, col] = False
        assert np.all(Jo[mask] == 0.0), "oracle J has no entry outside the pattern"
    assert np.all(np.isnan(J[:, C:]))


def test_rhs_worked_example_closed_form(torch, B):
    """Eqs. 4-5 through the library: f = (-2 k A^2 + 2 zeta B, k A^2 - zeta B)."""
    d = sn.worked_example()
    net = B.Network(d, 0)
    kk = np.array([[0.3, 1e-12, 5.0], [0.05, 2.0, 1e-30]])
    yy = np.array([[0.7, 1e-10, 1.0], [0.2, 0.5, 1e-20]])
    kd, yd = dev_mat(torch, kk, 32, 0.0), dev_mat(torch, yy, 32, 0.0)
    fd = torch.zeros((2, 32), dtype=torch.float64, device="cuda")
    net.rhs_eval(kd, yd, fd, 3)
    net.sync()
    f = fd.cpu().numpy()[:, :3]
    A, Bv = yy
    fa = -2 * kk[0] * A * A + 2 * kk[1] * Bv
    fb = kk[0] * A * A - kk[1] * Bv
    sc_ = 2 * kk[0] * A * A + 2 * kk[1] * Bv
    assert np.all(np.abs(f[0] - fa) <= 1e-15 * sc_) and np.all(np.abs(f[1] - fb) <= 1e-15 * sc_)


def test_edge_sizes(torch, B):
    d = sn.generate(2312, 32, 180)
    net = B.Network(d, 0)
    z = torch.zeros((d.n_r, 32), dtype=torch.float64, device="cuda")
    y = torch.zeros((d.n_s, 32), dtype=torch.float64, device="cuda")
    f = torch.full((d.n_s, 32), 3.0, dtype=torch.float64, device="cuda")
    net.rhs_eval(z, y, f, 0)            # C = 0: no-op
    net.sync()
    assert torch.all(f == 3.0)
    import ctypes as ct
    L = B.lib()
    assert L.sm_rhs_eval(net.h, 5, ct.c_void_p(z.data_ptr()), ct.c_void_p(y.data_ptr()),
                         ct.c_void_p(f.data_ptr()), 20, None) == B.SM_EINVAL   # ld % 32
    assert L.sm_rhs_eval(net.h, 40, ct.c_void_p(z.data_ptr()), ct.c_void_p(y.data_ptr()),
                         ct.c_void_p(f.data_ptr()), 32, None) == B.SM_EINVAL   # C > ld


def test_nonfinite_inputs_propagate(torch, B):
    d = sn.generate(2312, 32, 180)
    net = B.Network(d, 0)
    k = torch.ones((d.n_r, 32), dtype=torch.float64, device="cuda")
    y = torch.full((d.n_s, 32), 1e-3, dtype=torch.float64, device="cuda")
    y[0, 3] = float("nan")
    f = torch.zeros((d.n_s, 32), dtype=torch.float64, device="cuda")
    net.rhs_eval(k, y, f, 32)
    net.sync()
    assert torch.isnan(f[:, 3]).any() and torch.isfinite(f[:, 4]).all()


@pytest.mark.parametrize("fmt", [("crs", "none", 1, 1), ("sell", "nnz", 8, 470)])
def test_full_size_sampled(torch, B, fmt):
    """The 4096-cell, 470 x 6000 workload in the benchmark's launch
    configuration; 24 sampled cells checked against the oracle one by one."""
    from synth.workloads import make
    d, T, nH, Av, y = make("rhs_jac_470x6000_c4096")
    C = y.shape[1]
    net = B.Network(d, 0)
    net.set_format(*fmt)
    tt = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    kd = torch.empty((d.n_r, C), dtype=torch.float64, device="cuda")
    net.rates_eval(tt(T), tt(nH), tt(Av), kd, C)
    yd = tt(y)
    fd = torch.empty((d.n_s, C), dtype=torch.float64, device="cuda")
    net.rhs_eval(kd, yd, fd, C)
    net.sync()
    k = kd.cpu().numpy()
    f = fd.cpu().numpy()
    S = on.stoichiometry(d)
    rng = np.random.default_rng(0)
    for c in list(rng.choice(C, 22, replace=False)) + [0, C - 1]:
        ref = S @ ok.reaction_rates(d, k[:, c], y[:, c])
        scale = np.abs(S) @ np.abs(ok.reaction_rates(d, k[:, c], y[:, c]))
        assert np.all(np.abs(f[:, c] - ref) <= RTOL_F * scale + 1e-300)


def test_autotune_selects_a_measured_format_and_keeps_parity(torch, B):
    """sm_net_autotune times the candidate traversals, leaves the fastest
    selected (reported by sm_net_get_info), caches it per network / device /
    batch size, and rhs_eval keeps the usual 1e-12 bar afterwards."""
    d = sn.generate(2312, 470, 6000)
    C = 512
    ld = B.pad_ld(C)
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    y = sc.loguniform_abundances(d, 4998, C)
    k = ok.rate_coefficients(d, T, nH, Av)
    net = B.Network(d, 0)
    kd, yd = dev_mat(torch, k, ld, 0.0), dev_mat(torch, y, ld, 0.0)
    fd = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    r = net.autotune(kd, yd, fd, C)
    assert not r["cached"] and r["candidates"] >= 10 and r["us"] > 0
    info = net.info()
    assert (info["fmt"], info["order"]) == (B.FMT[r["fmt"]], B.ORDER[r["order"]])
    assert (info["sell_C"], info["sell_sigma"]) == (r["sell_C"], r["sell_sigma"])
    net.set_format("crs", "none", 1, 1)
    r2 = net.autotune(kd, yd, fd, C - 100)          # same power-of-two bucket: cached
    assert r2["cached"] and r2["candidates"] == 0
    assert (r2["fmt"], r2["order"], r2["sell_C"]) == (r["fmt"], r["order"], r["sell_C"])
    assert net.info()["fmt"] == B.FMT[r["fmt"]]
    net.rhs_eval(kd, yd, fd, C)
    net.sync()
    f = fd.cpu().numpy()[:, :C]
    assert np.all(np.abs(f - ok.rhs(d, k, y)) <= RTOL_F * ok.rhs_scale(d, k, y) + 1e-300)
    # the integrator's gather was tuned too (3 row orders x 3 block shapes)
    assert r["integ_cells_per_cta"] in (8, 16, 32) and r["integ_us"] > 0 and r["candidates"] >= 19
    assert (r2["integ_order"], r2["integ_cells_per_cta"]) == (r["integ_order"], r["integ_cells_per_cta"])


@pytest.mark.parametrize("shape", [(32, 180, 100), (470, 6000, 96)])
def test_unrolled_conventional_rhs_matches_oracle(torch, B, shape):
    """The generated conventional right-hand side (one explicit expression
    per species, the pre-matrix algorithm of Section 3) against the oracle's
    dense S R, with the bar of the stoichiometry-matrix kernels."""
    from paper_2312_04998_gb300 import unrolled
    n_s, n_r, C = shape
    d = sn.generate(2312, n_s, n_r)
    ld = B.pad_ld(C)
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    y = sc.loguniform_abundances(d, 4998, C)
    k = ok.rate_coefficients(d, T, nH, Av)
    kd, yd = dev_mat(torch, k, ld, 0.0), dev_mat(torch, y, ld, 0.0)
    fd = torch.full((d.n_s, ld), -1.0, dtype=torch.float64, device="cuda")
    u = unrolled.Unrolled(d)
    assert u.n_terms == sum(int(np.count_nonzero(on.stoichiometry(d)[i])) for i in range(d.n_s))
    u.rhs_eval(kd, yd, fd, C)
    torch.cuda.synchronize()
    f = fd.cpu().numpy()[:, :C]
    assert np.all(np.abs(f - ok.rhs(d, k, y)) <= RTOL_F * ok.rhs_scale(d, k, y) + 1e-300)
