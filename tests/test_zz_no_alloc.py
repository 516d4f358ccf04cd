"""The non-allocating right-hand side (sm_rhs_eval_static).

Some callers cannot let a library call cudaMalloc: hydro codes that reserve
the device memory up front for their own pool allocator, and time-step loops
that must not allocate because cudaMalloc can synchronise the device.  For
them sm_rhs_eval_static keeps its rate buffer in a fixed array inside the
library.
These checks call it through the C ABI and compare it with sm_rhs_eval on the
same inputs, twice in a row (the shared array keeps the previous call's data,
which must not leak into the next result), with the tolerance of the other
RHS tests: |difference| <= 1e-12 * sum_j |S_ij R_j|.  This file is collected
last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from oracle import kinetics as ok
from synth import cells as sc
from synth import network as sn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "this test needs a CUDA GPU"
    return _t


@pytest.fixture(scope="module")
def B(torch):
    from paper_2312_04998_gb300 import build
    build.build()
    from paper_2312_04998_gb300 import binding
    return binding


def inputs(torch, d, C, ld, seed):
    T, nH, Av = sc.conditions(seed, C, (10.0, 300.0), (1e2, 1e7), (0.0, 10.0))
    y = sc.loguniform_abundances(d, seed, C)
    k = ok.rate_coefficients(d, T, nH, Av)
    kd = torch.zeros((d.n_r, ld), dtype=torch.float64, device="cuda")
    yd = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
    kd[:, :C] = torch.tensor(k, device="cuda")
    yd[:, :C] = torch.tensor(y, device="cuda")
    return k, y, kd, yd


@pytest.mark.parametrize("fmt", [("crs", "none", 1, 1), ("sell", "nnz", 8, 470)])
def test_static_rhs_matches_rhs_eval_twice(torch, B, fmt):
    d = sn.generate(2312, 470, 6000)
    C = 300
    ld = B.pad_ld(C)
    net = B.Network(d, 0)
    net.set_format(*fmt)
    for call, seed in enumerate((4998, 7001)):
        k, y, kd, yd = inputs(torch, d, C, ld, seed)
        ref = torch.zeros((d.n_s, ld), dtype=torch.float64, device="cuda")
        out = torch.full((d.n_s, ld), -1.0, dtype=torch.float64, device="cuda")
        net.rhs_eval(kd, yd, ref, C)
        net.rhs_eval_static(kd, yd, out, C)
        net.sync()
        a, b = out.cpu().numpy()[:, :C], ref.cpu().numpy()[:, :C]
        scale = ok.rhs_scale(d, k, y)
        assert np.all(np.abs(a - b) <= 1e-12 * scale + 1e-300), f"call {call}"


def test_static_rhs_rejects_oversize(torch, B):
    d = sn.generate(2312, 470, 6000)
    net = B.Network(d, 0)
    C = 1024        # 6000 x 1024 doubles > SM_STATIC_SCRATCH_DOUBLES
    assert d.n_r * C > B.STATIC_SCRATCH_DOUBLES
    z = torch.zeros((d.n_r, C), dtype=torch.float64, device="cuda")
    y = torch.zeros((d.n_s, C), dtype=torch.float64, device="cuda")
    f = torch.zeros((d.n_s, C), dtype=torch.float64, device="cuda")
    code = B.lib().sm_rhs_eval_static(net.h, C, ct.c_void_p(z.data_ptr()), ct.c_void_p(y.data_ptr()),
                                      ct.c_void_p(f.data_ptr()), C, None)
    assert code == B.SM_ETOOBIG
    assert "fixed-size" in B.status_str(code)
