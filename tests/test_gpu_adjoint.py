"""GPU discrete adjoint (sm_adjoint) against the oracle's adjoint.

Both sides differentiate the same frozen-step map: the GPU's recorded steps
(read back with sm_state_steps) are handed to oracle.adjoint.frozen_forward,
which re-solves every implicit step to 1e-14 from y_0, and oracle.adjoint.adjoint
sweeps it backwards.  The oracle adjoint is itself pinned to the tangent
sensitivity and to central differences (test_oracle_adjoint.py).

Tolerance.  The GPU recomputes each segment of 16 steps from the history the
forward run stored, and the forward's implicit solves stop at its Newton
tolerance (here 1e-3 in the WRMS norm with rtol 1e-6, so a relative state
error of about 1e-9 per stored point); the replayed steps are solved to 1e-4
WRMS (1e-10 relative).  A relative state error d moves each gradient term by
about d times the local condition of the step, so the bar is 1e-6 of the
largest gradient entry of the same cotangent plus 1e-6 of the entry itself:
three orders above the state error, far below any plausible mistake (a wrong
alpha, sign, transpose or missing history term changes entries at O(1)).
"""
import ctypes as ct

import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import kinetics as ok
from synth import cells as sc
from synth import network as sn

pytestmark = pytest.mark.gpu

YEAR = 3.15576e7
TARGETS = ("CO", "E-")
N_COT = len(TARGETS) + 1


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


def dev(torch, a, ld):
    n, C = a.shape
    h = np.zeros((n, ld))
    h[:, :C] = a
    return torch.tensor(h, dtype=torch.float64, device="cuda")


def forward(torch, B, d, k, y0, t_end, record, **opts):
    C = y0.shape[1]
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    st = B.State(net, C, record_steps=record, newton_tol=1e-3, newton_max=6, **opts)
    kd, yd = dev(torch, k, ld), dev(torch, y0, ld)
    stats = B.stats_tensor(C, "cuda")
    code = st.integrate(kd, yd, t_end, C, stats)
    torch.cuda.synchronize()
    return net, st, kd, yd, B.stats_to_numpy(stats), code


def log_cot(torch, d, yN, ld):
    """Cotangents: Phi_v = log y_N[target_v] for TARGETS where that abundance
    is at least 1e-12 (below it the logarithm's derivative only measures
    rounding noise; the row is 0 there), and Phi_2 = r . y_N with fixed random
    weights r in [0, 1)."""
    C = yN.shape[1]
    cot = np.zeros((N_COT, d.n_s, ld))
    for v, name in enumerate(TARGETS):
        t = d.species_index(name)
        ok_ = yN[t] >= 1e-12
        cot[v, t, :C] = np.where(ok_, 1.0 / np.where(ok_, yN[t], 1.0), 0.0)
    cot[len(TARGETS), :, :C] = np.random.default_rng(5).random(d.n_s)[:, None]
    return cot, torch.tensor(cot, dtype=torch.float64, device="cuda")


def recorded_steps(st, N, C):
    t, h, q = st.steps_log(int(N.max()), C)
    t, h, q = t.cpu().numpy(), h.cpu().numpy(), q.cpu().numpy()
    return [[(t[m, c], h[m, c], int(q[m, c])) for m in range(N[c])] for c in range(C)]


def oracle_grad(d, k, y0, steps, cot):
    ys = oa.frozen_forward(d, k, y0, steps)
    return oa.adjoint(d, k, ys, steps, cot)


def check(g, ref, what):
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
    err = np.abs(g - ref)
    bar = 1e-6 * scale + 1e-6 * np.abs(ref)
    assert np.all(err <= bar), (what, float((err / np.maximum(bar, 1e-300)).max()))


@pytest.fixture(scope="module")
def small(torch, B):
    """36 cells (one full warp of cells and a ragged tail) of the 32 x 180
    network, 1e3 yr, three cotangents."""
    d = sn.generate(2312, 32, 180)
    C = 36
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    net, st, kd, yd, stats, code = forward(torch, B, d, k, y0, 1e3 * YEAR, 4000)
    assert code == B.SM_OK
    ld = B.pad_ld(C)
    yN = yd.cpu().numpy()[:, :C]
    cot, cot_d = log_cot(torch, d, yN, ld)
    grad = torch.zeros((N_COT, d.n_r, ld), dtype=torch.float64, device="cuda")
    g0 = torch.zeros((N_COT, d.n_s, ld), dtype=torch.float64, device="cuda")
    astat = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    code = st.adjoint(kd, cot_d, grad, astat, grad_y0=g0)
    torch.cuda.synchronize()
    return dict(d=d, C=C, k=k, y0=y0, net=net, st=st, kd=kd, yN=yN, stats=stats, cot=cot, cot_d=cot_d,
                grad=grad.cpu().numpy(), grad_y0=g0.cpu().numpy(), astat=astat.cpu().numpy()[:C], code=code)


def test_adjoint_matches_oracle_small(small):
    s = small
    assert s["code"] == 0 and np.all(s["astat"] == 0)
    N = s["stats"]["steps"]
    assert N.min() > 16          # every cell spans several checkpoint segments
    steps = recorded_steps(s["st"], N, s["C"])
    for c in (0, 1, 7, 19, 31, 32, 35):
        ys = oa.frozen_forward(s["d"], s["k"][:, c], s["y0"][:, c], steps[c])
        ref, ref0 = oa.adjoint(s["d"], s["k"][:, c], ys, steps[c], s["cot"][:, :, c], with_y0=True)
        check(s["grad"][:, :, c], ref, f"cell {c}")
        check(s["grad_y0"][:, :, c], ref0, f"cell {c}, dPhi/dy0")


def test_adjoint_pass_split_is_bit_identical(torch, B, small):
    """Two passes of 32 + 4 cells give the same bits as one pass of 36, and a
    second call on the same recorded run repeats the first."""
    s = small
    d, ld = s["d"], B.pad_ld(s["C"])
    for cpp in (0, 32):
        grad = torch.zeros((N_COT, d.n_r, ld), dtype=torch.float64, device="cuda")
        assert s["st"].adjoint(s["kd"], s["cot_d"], grad, cells_per_pass=cpp) == 0
        torch.cuda.synchronize()
        assert np.array_equal(grad.cpu().numpy()[:, :, :s["C"]], s["grad"][:, :, :s["C"]]), cpp


def test_adjoint_cells_beyond_record(torch, B, small):
    """A record shorter than some cells' runs: those cells report status 1 and
    a zero gradient, the rest match the fully recorded run bit for bit."""
    s = small
    d, C = s["d"], s["C"]
    N = s["stats"]["steps"]
    R = int(np.median(N))
    net, st, kd, yd, stats, code = forward(torch, B, d, s["k"], s["y0"], 1e3 * YEAR, R)
    assert code == B.SM_OK and np.array_equal(stats["steps"], N)
    ld = B.pad_ld(C)
    grad = torch.full((N_COT, d.n_r, ld), 7.0, dtype=torch.float64, device="cuda")
    astat = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    code = st.adjoint(kd, s["cot_d"], grad, astat)
    torch.cuda.synchronize()
    assert code == B.SM_EPARTIAL
    g, a = grad.cpu().numpy()[:, :, :C], astat.cpu().numpy()[:C]
    over = N > R
    assert np.array_equal(a, np.where(over, 1, 0))
    assert np.all(g[:, :, over] == 0.0)
    assert np.array_equal(g[:, :, ~over], s["grad"][:, :, :C][:, :, ~over])


def test_adjoint_rejects_bad_calls(torch, B, small):
    s = small
    d, C = s["d"], s["C"]
    ld = B.pad_ld(C)
    L = B.lib()
    grad = torch.zeros((N_COT, d.n_r, ld), dtype=torch.float64, device="cuda")
    p = lambda t: ct.c_void_p(t.data_ptr())
    # no cotangents, too many, negative pass size
    assert L.sm_adjoint(s["st"].h, p(s["kd"]), ld, p(s["cot_d"]), 0, p(grad), None, None, 0, None) == B.SM_EINVAL
    assert L.sm_adjoint(s["st"].h, p(s["kd"]), ld, p(s["cot_d"]), B.ADJ_MAX_COT + 1, p(grad), None, None, 0,
                        None) == B.SM_EINVAL
    assert L.sm_adjoint(s["st"].h, p(s["kd"]), ld, p(s["cot_d"]), 1, p(grad), None, None, -1, None) == B.SM_EINVAL
    y0 = dev(torch, s["y0"], ld)
    # a state that records nothing
    st0 = B.State(s["net"], C)
    st0.init(s["kd"], y0, 1e3 * YEAR, C)
    assert L.sm_adjoint(st0.h, p(s["kd"]), ld, p(s["cot_d"]), 1, p(grad), None, None, 0, None) == B.SM_EINVAL
    # the adjoint runs in FP64 only
    stm = B.State(s["net"], C, precision="mixed", record_steps=100)
    stm.init(s["kd"], y0, 1e3 * YEAR, C)
    assert L.sm_adjoint(stm.h, p(s["kd"]), ld, p(s["cot_d"]), 1, p(grad), None, None, 0, None) == B.SM_ENOTSUP
    torch.cuda.synchronize()


def test_adjoint_matches_oracle_470x6000(torch, B):
    """Two cells of the 470 x 6000 network over one year: the factors here
    have the sparse head and the dense trailing block of the production
    network."""
    d = sn.generate(2312, 470, 6000)
    C = 2
    T, nH, Av = sc.conditions(4998, C, (10.0, 300.0), (1e2, 1e6), (0.0, 10.0))
    k = ok.rate_coefficients(d, T, nH, Av)
    y0 = sc.atomic_start(d, C)
    net, st, kd, yd, stats, code = forward(torch, B, d, k, y0, 1.0 * YEAR, 4000)
    assert code == B.SM_OK
    ld = B.pad_ld(C)
    yN = yd.cpu().numpy()[:, :C]
    cot, cot_d = log_cot(torch, d, yN, ld)
    grad = torch.zeros((N_COT, d.n_r, ld), dtype=torch.float64, device="cuda")
    assert st.adjoint(kd, cot_d, grad) == 0
    torch.cuda.synchronize()
    g = grad.cpu().numpy()
    N = stats["steps"]
    steps = recorded_steps(st, N, C)
    c = int(np.argmin(N))   # the oracle's dense solves make the shorter run the cheaper check
    assert N[c] > 16
    ref = oracle_grad(d, k[:, c], y0[:, c], steps[c], cot[:, :, c])
    check(g[:, :, c], ref, f"cell {c}")


def test_replay_matches_oracle_frozen_map(torch, B, small):
    """sm_replay re-solves the recorded steps; the oracle's frozen map solves
    the same steps to 1e-14.  The replay stops at 1e-4 in the run's WRMS
    norm (rtol 1e-6), and the stable map carries that along the run, so the
    bar is 1e-2 WRMS units (1e-8 relative) on every abundance."""
    s = small
    d, C = s["d"], s["C"]
    ld = B.pad_ld(C)
    y = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    assert s["st"].replay(s["kd"], y) == B.SM_OK
    torch.cuda.synchronize()
    y = y.cpu().numpy()[:, :C]
    N = s["stats"]["steps"]
    steps = recorded_steps(s["st"], N, C)
    for c in (0, 5, 20, 33, 35):
        ref = oa.frozen_forward(d, s["k"][:, c], s["y0"][:, c], steps[c])[-1]
        w = 1e-6 * np.abs(ref) + 1e-20
        assert np.max(np.abs(y[:, c] - ref) / w) <= 1e-2, c


def test_autograd_function(torch, B, small):
    """Integrate.apply + backward reproduces sm_adjoint with the same
    cotangent: d/dlog k to one rounding (k.grad is divided by k), d/dy0 bit
    for bit."""
    from paper_2312_04998_gb300.autograd import Integrate
    s = small
    d, C = s["d"], s["C"]
    ld = B.pad_ld(C)
    st = B.State(s["net"], C, record_steps=4000, newton_tol=1e-3, newton_max=6)
    k = s["kd"].clone().requires_grad_(True)
    y0 = dev(torch, s["y0"], ld).requires_grad_(True)
    y = Integrate.apply(k, y0, st, 1e3 * YEAR, C)
    t = d.species_index("CO")
    loss = torch.log(y[t, :C]).sum()
    loss.backward()
    # k.grad = (dPhi/dlog k) / k; multiplying back rounds once more
    gk = (k.grad * k.detach()).cpu().numpy()[:, :C]
    ref = s["grad"][0][:, :C]
    assert np.all(np.abs(gk - ref) <= 4e-16 * np.abs(ref))
    assert np.array_equal(y0.grad.cpu().numpy()[:, :C], s["grad_y0"][0][:, :C])
    # a second integration invalidates the record of the first
    y2 = Integrate.apply(k, y0, st, 1e3 * YEAR, C)
    st.integrate(s["kd"], dev(torch, s["y0"], ld), 1e3 * YEAR, C)
    with pytest.raises(RuntimeError):
        torch.log(y2[t, :C]).sum().backward()


def test_adjoint_central_differences_1024_cells(torch, B):
    """The 1024-cell adjoint workload (470 x 6000, 1e5 yr, eight log-abundance
    targets, checkpoints every 16 steps) against central differences of the
    frozen map on the GPU: cell c perturbs one reaction j_c (half of them among
    the largest gradient entries, half at random), so the two sm_replay calls
    give 1024 sampled derivatives; 32 distinct reactions or more are covered.
    Step h = 1e-4 in log k: the replay solves each step to 1e-10 relative, so
    the difference quotient carries at most 1e-10 / h = 1e-6 of noise, while
    the O(h^2) truncation stays near 1e-8 relative.  Bar: 1e-6 + 1e-4 |g|."""
    from synth import workloads as W
    desc, T, nH, Av, y0 = W.make("adjoint_470x6000_c1024")
    C = y0.shape[1]
    k = ok.rate_coefficients(desc, T, nH, Av)
    ld = B.pad_ld(C)
    net, st, kd, yd, stats, code = forward(torch, B, desc, k, y0, W.WORKLOADS["adjoint_470x6000_c1024"].t_end, 4000)
    assert code == B.SM_OK
    yr = torch.zeros_like(yd)
    assert st.replay(kd, yr) == B.SM_OK
    yN = yr.cpu().numpy()[:, :C]
    frac = (yN > 1e-12).mean(axis=1)
    targets = np.argsort(-frac, kind="stable")[:8]
    cot = np.zeros((8, desc.n_s, ld))
    for v, t in enumerate(targets):
        cot[v, t, :C] = np.where(yN[t] > 1e-12, 1.0 / np.maximum(yN[t], 1e-300), 0.0)
    grad = torch.zeros((8, desc.n_r, ld), dtype=torch.float64, device="cuda")
    astat = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    assert st.adjoint(kd, torch.tensor(cot, device="cuda"), grad, astat) == B.SM_OK
    g = grad.cpu().numpy()[:, :, :C]
    assert np.all(astat.cpu().numpy()[:C] == 0)
    rng = np.random.default_rng(4998)
    vs = np.arange(C) % 8
    js = np.array([int(np.argsort(-np.abs(g[vs[c], :, c]))[rng.integers(0, 8)]) if c % 2 == 0
                   else int(rng.integers(0, desc.n_r)) for c in range(C)])
    assert len(set(js.tolist())) >= 32
    hh = 1e-4
    out = []
    for sign in (1.0, -1.0):
        kp = k.copy()
        kp[js, np.arange(C)] *= np.exp(sign * hh)
        y = torch.zeros_like(yd)
        assert st.replay(dev(torch, kp, ld), y) == B.SM_OK
        out.append(y.cpu().numpy()[:, :C])
    live = cot[vs, targets[vs], np.arange(C)] != 0
    phi = [np.log(np.where(live, Y[targets[vs], np.arange(C)], 1.0)) for Y in out]
    fd = (phi[0] - phi[1]) / (2 * hh)
    ad = g[vs, js, np.arange(C)]
    err = np.abs(fd - ad)[live]
    bar = 1e-6 + 1e-4 * np.abs(ad[live])
    assert live.sum() >= 0.9 * C
    assert np.all(err <= bar), float((err / bar).max())
