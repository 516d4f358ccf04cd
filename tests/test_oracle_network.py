"""Pins for the oracle's stoichiometry matrix, formats and row orders."""
import json
import os

import numpy as np
import pytest

from oracle import network as on
from synth import network as sn

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def test_worked_example_stoichiometry():
    """Eq. 6: S = [[-2, 2], [1, -1]] for 2A -> B, B + hv -> 2A."""
    g = _load("worked_example.json")
    S = on.stoichiometry(sn.worked_example())
    assert np.array_equal(S, np.array(g["stoichiometry"], dtype=float))


def test_listing_crs_exact():
    """Listing 3's arrays, converted to 0-based."""
    g = _load("listings.json")
    A = np.array(g["matrix"], dtype=float)
    val, col, ptr, rid = on.to_crs(A)
    assert val.tolist() == g["crs"]["A"]
    assert (col + 1).tolist() == g["crs"]["col_ind"]
    assert (ptr + 1).tolist() == g["crs"]["row_ptr"]
    assert rid.tolist() == [0, 1, 2, 3]


def test_listing_ccs_exact():
    """Listing 2's arrays, converted to 0-based."""
    g = _load("listings.json")
    A = np.array(g["matrix"], dtype=float)
    val, row, ptr, cid = on.to_ccs(A)
    assert val.tolist() == g["ccs"]["A"]
    assert (row + 1).tolist() == g["ccs"]["row_ind"]
    assert (ptr + 1).tolist() == g["ccs"]["col_ptr"]


def test_listing_coo_same_entries():
    """Listing 1 stores its 7 nonzeros in an arbitrary order: compare as a set."""
    g = _load("listings.json")
    A = np.array(g["matrix"], dtype=float)
    val, row, col = on.to_coo(A)
    mine = sorted(zip((row + 1).tolist(), (col + 1).tolist(), val.tolist()))
    theirs = sorted(zip(g["coo"]["row_ind"], g["coo"]["col_ind"], g["coo"]["A"]))
    assert mine == theirs and len(val) == g["coo"]["n_nz"]


def test_listing_sell_values_and_slices():
    """Listing 4 (slice width 2): values, slice lengths and real columns match;
    the padding column indices follow no stated rule and are not compared."""
    g = _load("listings.json")
    A = np.array(g["matrix"], dtype=float)
    val, col, sptr, slen, rid = on.to_sell(A, C=g["sell"]["wid_sl"], sigma=1)
    assert val.tolist() == g["sell"]["A"]
    assert slen.tolist() == g["sell"]["len_sl"]
    assert len(slen) == g["sell"]["n_sl"]
    real = np.array(g["sell"]["A"]) != 0
    assert ((col + 1)[real]).tolist() == np.array(g["sell"]["col_ind"])[real].tolist()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_format_loops_match_dense_product(seed):
    """Each format's own loop reproduces A @ x for a random sparse A, under
    random row and column orders and several SELL slice heights / windows."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-3, 4, size=(13, 17)) * (rng.random((13, 17)) < 0.25)
    A = A.astype(float)
    x = rng.standard_normal(17)
    ref = A @ x
    ro, co = rng.permutation(13), rng.permutation(17)
    assert np.allclose(on.crs_matvec(on.to_crs(A, ro, co), x, 13), ref, rtol=0, atol=1e-12)
    assert np.allclose(on.ccs_matvec(on.to_ccs(A, ro, co), x, 13), ref, rtol=0, atol=1e-12)
    assert np.allclose(on.coo_matvec(on.to_coo(A, ro, co), x, 13), ref, rtol=0, atol=1e-12)
    for C, sigma in ((1, 1), (4, 1), (4, 8), (8, 13), (32, 13)):
        fmt = on.to_sell(A, C, sigma, ro, co)
        assert np.allclose(on.sell_matvec(fmt, x, 13, C), ref, rtol=0, atol=1e-12)


def test_sell_sigma_sorts_within_windows():
    A = np.zeros((6, 6))
    nnz = [1, 3, 2, 5, 4, 0]
    for i, n in enumerate(nnz):
        A[i, :n] = 1.0
    assert on.sell_row_order(A, 2, 1).tolist() == [0, 1, 2, 3, 4, 5]
    assert on.sell_row_order(A, 2, 3).tolist() == [1, 2, 0, 3, 4, 5]
    assert on.sell_row_order(A, 2, 6).tolist() == [3, 4, 1, 2, 0, 5]


def test_nnz_order_descending_stable():
    A = np.zeros((5, 4))
    for i, n in enumerate([2, 4, 2, 1, 4]):
        A[i, :n] = 1.0
    assert on.order_nnz(A).tolist() == [1, 4, 0, 2, 3]


def _bandwidth(S, order):
    adj = on.species_graph(S)
    pos = np.empty(len(order), dtype=int)
    pos[order] = np.arange(len(order))
    return max((abs(pos[i] - pos[l]) for i in range(len(adj)) for l in adj[i]), default=0)


def test_rcm_path_graph_bandwidth_one():
    """A shuffled path graph: Cuthill-McKee from a peripheral node gives
    bandwidth 1, the optimum."""
    rng = np.random.default_rng(7)
    n = 12
    lab = rng.permutation(n)
    S = np.zeros((n, n - 1))
    for e in range(n - 1):       # reaction e links path nodes e and e+1
        S[lab[e], e] = -1.0
        S[lab[e + 1], e] = 1.0
    rows, cols = on.order_rcm(S)
    assert sorted(rows.tolist()) == list(range(n))
    assert _bandwidth(S, rows) == 1
    assert sorted(cols.tolist()) == list(range(n - 1))


def test_rcm_hand_example():
    """Graph worked by hand: star centre 0 with leaves 1,2,3; leaf 3 also
    linked to 4; 5 isolated.  Degrees: 0:3, 1:1, 2:1, 3:2, 4:1, 5:0.
    Component {0..4}: lowest-index min-degree node 1 (levels [1],[0],[2,3],[4]);
    last level's min-degree node 4 gives levels [4],[3],[0],[1,2] (no longer),
    so root stays 1.  CM from 1: 1, 0, then 0's neighbours by (deg, idx): 2, 3,
    then 4.  Component {5}: 5.  CM = 1,0,2,3,4,5; reversed 5,4,3,2,0,1."""
    edges = [(0, 1), (0, 2), (0, 3), (3, 4)]
    S = np.zeros((6, len(edges) + 1))
    for e, (a, b) in enumerate(edges):
        S[a, e] = -1.0
        S[b, e] = 1.0
    S[5, len(edges)] = -1.0      # an isolated species with a sink reaction
    rows, _ = on.order_rcm(S)
    assert rows.tolist() == [5, 4, 3, 2, 0, 1]


@pytest.mark.parametrize("n_s,n_r", [(32, 180), (120, 1200)])
def test_generated_networks_conserve(n_s, n_r):
    d = sn.generate(2312, n_s, n_r)
    assert d.n_s == n_s and d.n_r == n_r
    assert on.conserves(d)
    S = on.stoichiometry(d)
    assert np.all(np.any(S != 0, axis=0)), "every reaction changes something"
    d2 = sn.generate(2312, n_s, n_r)
    assert np.array_equal(d.reactants, d2.reactants) and np.array_equal(d.alpha, d2.alpha)


def test_nonconserving_network_detected():
    d = sn.worked_example()
    d.products = d.products.copy()
    d.products[0, 0] = 0          # 2A -> A loses an H atom
    assert not on.conserves(d)


def test_jacobian_pattern_matches_numeric_structure():
    from oracle import kinetics as ok
    d = sn.generate(5, 32, 180)
    rng = np.random.default_rng(0)
    k = 10 ** rng.uniform(-3, 0, d.n_r)
    y = 10 ** rng.uniform(-3, 0, d.n_s)
    J = ok.jacobian(d, k, y)
    P = on.jacobian_pattern(d)
    assert np.all(P[J != 0])               # numeric nonzeros lie in the pattern
    off = P & ~np.eye(d.n_s, dtype=bool)
    # generic positive values leave no structural entry at exactly zero
    # unless contributions cancel; allow a handful of cancellations only
    assert np.count_nonzero(off & (J == 0)) <= 2
