"""C-ABI library on the host: symbols, argument checks and bit-exact network
structures (formats, row / column orders, Jacobian pattern) against the oracle.
No kernel is launched here (networks are built with device = -1)."""
import os
import re

import numpy as np
import pytest

from oracle import network as on
from synth import network as sn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2312_04998_gb300 import build
    build.build()
    from paper_2312_04998_gb300 import binding
    return binding


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "stoich.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    L = B.lib()
    names = declared_symbols()
    assert "sm_rhs_eval" in names and "sm_net_build" in names
    for name in names:
        assert hasattr(L, name), name


def test_binding_constants_match_header(B):
    src = open(os.path.join(ROOT, "include", "stoich.h")).read()
    defs = dict(re.findall(r"#define\s+(SM_[A-Z_]+)\s+(\d+)", src))
    assert int(defs["SM_CHECKPOINT_EVERY"]) == B.CHECKPOINT_EVERY
    assert int(defs["SM_ADJ_MAX_COT"]) == B.ADJ_MAX_COT
    assert int(defs["SM_STATIC_SCRATCH_DOUBLES"]) == B.STATIC_SCRATCH_DOUBLES


def test_status_strings(B):
    assert B.status_str(B.SM_OK) == "ok"
    assert "conserve" in B.status_str(B.SM_ENOTCONS)


@pytest.fixture(scope="module")
def big():
    d = sn.generate(2312, 470, 6000)
    return d, on.stoichiometry(d)


def _oracle_orders(S, order):
    if order == "none":
        return np.arange(S.shape[0]), np.arange(S.shape[1])
    if order == "nnz":
        return on.order_nnz(S), np.arange(S.shape[1])
    return on.order_rcm(S)


@pytest.mark.parametrize("order", ["none", "nnz", "rcm"])
def test_orders_and_crs_bit_exact(B, big, order):
    d, S = big
    net = B.Network(d, device=-1)
    net.set_format("crs", order)
    ro, co = _oracle_orders(S, order)
    assert np.array_equal(net.export(B.X_ROW_ORDER), ro)
    assert np.array_equal(net.export(B.X_COL_ORDER), co)
    val, col, ptr, _ = on.to_crs(S, ro, co)
    assert np.array_equal(net.export(B.X_FMT_PTR), ptr)
    assert np.array_equal(net.export(B.X_FMT_IDX), col)
    assert np.array_equal(net.export(B.X_FMT_VAL, np.float64), val)


@pytest.mark.parametrize("order", ["none", "rcm"])
def test_ccs_and_coo_bit_exact(B, big, order):
    d, S = big
    net = B.Network(d, device=-1)
    ro, co = _oracle_orders(S, order)
    net.set_format("ccs", order)
    val, row, ptr, _ = on.to_ccs(S, ro, co)
    assert np.array_equal(net.export(B.X_FMT_PTR), ptr)
    assert np.array_equal(net.export(B.X_FMT_IDX), row)
    assert np.array_equal(net.export(B.X_FMT_VAL, np.float64), val)
    net.set_format("coo", order)
    val, row, col = on.to_coo(S, ro, co)
    assert np.array_equal(net.export(B.X_FMT_IDX), row)
    assert np.array_equal(net.export(B.X_FMT_IDX2), col)
    assert np.array_equal(net.export(B.X_FMT_VAL, np.float64), val)


@pytest.mark.parametrize("C,sigma,order", [(4, 1, "none"), (4, 1, "nnz"), (8, 64, "none"),
                                           (32, 470, "rcm"), (1, 1, "none")])
def test_sell_bit_exact(B, big, C, sigma, order):
    d, S = big
    net = B.Network(d, device=-1)
    ro, co = _oracle_orders(S, order)
    net.set_format("sell", order, C, sigma)
    val, col, sptr, slen, rid = on.to_sell(S, C, sigma, ro, co)
    assert np.array_equal(net.export(B.X_FMT_PTR), sptr)
    assert np.array_equal(net.export(B.X_FMT_LEN), slen)
    assert np.array_equal(net.export(B.X_FMT_IDX2), rid)
    assert np.array_equal(net.export(B.X_FMT_IDX), col)
    assert np.array_equal(net.export(B.X_FMT_VAL, np.float64), val)


def test_worked_example_through_library(B):
    """Eq. 6's S = [[-2, 2], [1, -1]] exported from the library in CCS."""
    d = sn.worked_example()
    net = B.Network(d, device=-1)
    net.set_format("ccs")
    assert net.export(B.X_FMT_VAL, np.float64).tolist() == [-2.0, 1.0, 2.0, -1.0]
    assert net.export(B.X_FMT_IDX).tolist() == [0, 1, 0, 1]
    assert net.export(B.X_FMT_PTR).tolist() == [0, 2, 4]


def test_jacobian_pattern_bit_exact(B, big):
    d, _ = big
    net = B.Network(d, device=-1)
    P = on.jacobian_pattern(d)
    ptr = net.export(B.X_JPAT_PTR)
    col = net.export(B.X_JPAT_COL)
    assert ptr[-1] == P.sum() == net.info()["nnz_J"]
    for i in range(d.n_s):
        assert np.array_equal(col[ptr[i]:ptr[i + 1]], np.nonzero(P[i])[0])


def test_lu_perm_is_permutation(B, big):
    d, _ = big
    net = B.Network(d, device=-1)
    p = net.export(B.X_LU_PERM)
    assert sorted(p.tolist()) == list(range(d.n_s))
    inf = net.info()
    assert inf["nnz_LU"] >= inf["nnz_J"] and inf["lu_flops"] > 0


def test_build_rejects_nonconserving(B):
    d = sn.worked_example()
    d.products = d.products.copy()
    d.products[0, 0] = 0
    with pytest.raises(B.StoichError) as e:
        B.Network(d, device=-1)
    assert e.value.code == B.SM_ENOTCONS


def test_build_rejects_bad_indices(B):
    d = sn.worked_example()
    d.reactants = d.reactants.copy()
    d.reactants[1, 0] = 7
    with pytest.raises(B.StoichError) as e:
        B.Network(d, device=-1)
    assert e.value.code == B.SM_EINVAL


def test_device_calls_rejected_on_host_only_network(B):
    import ctypes as ct
    net = B.Network(sn.worked_example(), device=-1)
    L = B.lib()
    assert L.sm_rhs_eval(net.h, 1, None, None, None, 32, None) == B.SM_EINVAL
    assert L.sm_net_set_format(net.h, 3, 0, 0, 1) == B.SM_EINVAL      # SELL C = 0
    assert L.sm_net_set_format(net.h, 9, 0, 1, 1) == B.SM_EINVAL
    assert L.sm_net_export(net.h, 99, None, 0) == B.SM_EINVAL
    del ct


def test_autotune_needs_a_device_network(B):
    """sm_net_autotune times kernels: a host-only network is refused."""
    import ctypes as ct
    d = sn.generate(2312, 32, 180)
    net = B.Network(d, device=-1)
    r = B.TuneResult_c()
    code = B.lib().sm_net_autotune(net.h, 32, None, None, None, 32, 0, None, ct.byref(r))
    assert code == B.SM_EINVAL


@pytest.mark.parametrize("seed,n_s,n_r", [(2312, 32, 180), (2312, 470, 6000), (99, 64, 700)])
def test_library_synthetic_network_equals_input_generator(B, seed, n_s, n_r):
    """sm_synth_network draws the same arrays, bit for bit, as the package's
    Python input generator for the same seed (both are integer decisions on
    the same SplitMix64 streams)."""
    a = B.synth_network(seed, n_s, n_r)
    d = sn.generate(seed, n_s, n_r)
    for key, ref in (("comp", d.comp), ("reactants", d.reactants), ("products", d.products),
                     ("rclass", d.rclass), ("alpha", d.alpha), ("beta", d.beta), ("gamma", d.gamma)):
        assert np.array_equal(a[key], ref), key


def test_build_synthetic_matches_build_from_arrays(B):
    d = sn.generate(2312, 470, 6000)
    n1 = B.Network(d, device=-1)
    n2 = B.Network.synthetic(2312, 470, 6000, device=-1)
    assert n1.info() == n2.info()
    for what in (B.X_FMT_PTR, B.X_FMT_IDX, B.X_JPAT_PTR, B.X_JPAT_COL, B.X_LU_PERM):
        assert np.array_equal(n1.export(what), n2.export(what))


def test_synthetic_network_rejects_bad_sizes(B):
    import ctypes as ct
    h = ct.c_void_p()
    assert B.lib().sm_net_build_synthetic(1, 8, 100, -1, ct.byref(h)) == B.SM_EINVAL
    assert B.lib().sm_net_build_synthetic(1, 32, 0, -1, ct.byref(h)) == B.SM_EINVAL


def test_set_thermal_checks_the_slot_and_parameters(B):
    """sm_net_set_thermal on the host: the temperature slot must have no
    atoms, no charge and no reaction; cooling coefficients must be >= 0 with
    positive excitation temperatures; the constants must be finite and >= 0;
    NULL turns the mode off."""
    import dataclasses
    from synth import thermal as sth
    d = sth.with_temperature(sn.generate(2312, 32, 180))
    th = sth.thermal_params(d)
    net = B.Network(d, device=-1)
    net.set_thermal(th)                                   # valid
    net.set_thermal(None)                                 # off
    bad = [dataclasses.replace(th, t_index=d.species_index("H")),       # has atoms
           dataclasses.replace(th, t_index=d.species_index("E-")),      # has charge and reactions
           dataclasses.replace(th, t_index=d.n_s),                      # out of range
           dataclasses.replace(th, heat=-1.0),
           dataclasses.replace(th, lam=float("nan")),
           dataclasses.replace(th, L=np.where(np.arange(d.n_s) == 0, -1.0, th.L)),
           dataclasses.replace(th, E=np.where(th.L > 0, 0.0, th.E))]
    for b in bad:
        with pytest.raises(B.StoichError) as e:
            net.set_thermal(b)
        assert e.value.code == B.SM_EINVAL
    # a species that appears in a reaction cannot be the slot even without atoms
    d0 = sn.generate(2312, 32, 180)
    net0 = B.Network(d0, device=-1)
    with pytest.raises(B.StoichError):
        net0.set_thermal(dataclasses.replace(th, t_index=d0.species_index("E-"), L=th.L[:d0.n_s],
                                             E=th.E[:d0.n_s]))
