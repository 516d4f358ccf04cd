"""Stoichiometry matrix, element matrix, storage formats and row orders.

Test infrastructure (oracle): see the package docstring.

* `stoichiometry` writes out Eq. 7: alpha_ij = (copies of i among the products
  of reaction j) - (copies of i among its reactants); negative for reactants,
  positive for products, zero otherwise.  Reactant multiplicity enters both the
  rate power and S, as in the worked example of Eqs. 2-6 (2A -> B gives
  alpha_A = -2 and R = k n_A^2).
* `to_coo / to_ccs / to_crs / to_sell` build the four formats of Section 2.2
  (Listings 1-4) from the dense matrix, with 0-based indices.
* `order_nnz` is the row reordering of Section 3 ("in order of the number of
  nonzero elements"; read as descending, ties by original index).
* `order_rcm` is reverse Cuthill-McKee on the species graph pattern(S S^T),
  an added reordering (the paper reorders by nonzero count only).

Every routine here is a direct loop over the dense matrix; none of it is tuned.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Eq. 7: the stoichiometry matrix and the conservation matrix
# ----------------------------------------------------------------------------

def stoichiometry(desc) -> np.ndarray:
    """Dense S (n_s x n_r, float64): products minus reactants, per Eq. 7."""
    S = np.zeros((desc.n_s, desc.n_r))
    for j in range(desc.n_r):
        for a in desc.reactants[j]:
            if a >= 0:
                S[a, j] -= 1.0
        for p in desc.products[j]:
            if p >= 0:
                S[p, j] += 1.0
    return S


def element_matrix(desc) -> np.ndarray:
    """E[(elements + charge), species]: element counts and charge per species."""
    return desc.comp.T.astype(np.int64)


def conserves(desc) -> bool:
    """Every reaction conserves every element and charge: E.S == 0 exactly."""
    return bool(np.all(element_matrix(desc) @ stoichiometry(desc).astype(np.int64) == 0))


def jacobian_pattern(desc) -> np.ndarray:
    """Boolean structure of J = S.dR/dy plus the diagonal: (i, l) is set when
    some reaction with alpha_ij != 0 has species l among its reactants."""
    S = stoichiometry(desc)
    P = np.zeros((desc.n_s, desc.n_s), dtype=bool)
    for j in range(desc.n_r):
        rows = [i for i in range(desc.n_s) if S[i, j] != 0.0]
        for a in desc.reactants[j]:
            if a >= 0:
                for i in rows:
                    P[i, a] = True
    for i in range(desc.n_s):
        P[i, i] = True
    return P


# ----------------------------------------------------------------------------
# Section 2.2: storage formats (0-based versions of Listings 1-4)
# ----------------------------------------------------------------------------

def _orders(A, row_order, col_order):
    n_row, n_col = A.shape
    ro = np.arange(n_row) if row_order is None else np.asarray(row_order)
    co = np.arange(n_col) if col_order is None else np.asarray(col_order)
    return ro, co


def to_crs(A, row_order=None, col_order=None):
    """CRS (Listing 3): rows visited in `row_order`, each row's nonzeros in
    `col_order` order.  Returns (val, col_ind, row_ptr, row_id) where row_id[p]
    is the matrix row stored at position p and col_ind holds matrix columns."""
    ro, co = _orders(A, row_order, col_order)
    val, col_ind, row_ptr = [], [], [0]
    for i in ro:
        for j in co:
            if A[i, j] != 0:
                val.append(A[i, j])
                col_ind.append(j)
        row_ptr.append(len(val))
    return (np.array(val, dtype=float), np.array(col_ind, dtype=np.int64),
            np.array(row_ptr, dtype=np.int64), np.array(ro, dtype=np.int64))


def to_ccs(A, row_order=None, col_order=None):
    """CCS (Listing 2): columns visited in `col_order`, each column's nonzeros
    in `row_order` order.  Returns (val, row_ind, col_ptr, col_id)."""
    ro, co = _orders(A, row_order, col_order)
    val, row_ind, col_ptr = [], [], [0]
    for j in co:
        for i in ro:
            if A[i, j] != 0:
                val.append(A[i, j])
                row_ind.append(i)
        col_ptr.append(len(val))
    return (np.array(val, dtype=float), np.array(row_ind, dtype=np.int64),
            np.array(col_ptr, dtype=np.int64), np.array(co, dtype=np.int64))


def to_coo(A, row_order=None, col_order=None):
    """COO (Listing 1) in column-major order (the paper allows any order).
    Returns (val, row_ind, col_ind)."""
    val, row_ind, col_ptr, col_id = to_ccs(A, row_order, col_order)
    col_ind = np.repeat(col_id, np.diff(col_ptr))
    return val, row_ind, col_ind


def sell_row_order(A, C, sigma, row_order=None):
    """SELL-C-sigma row order: inside consecutive windows of `sigma` rows of the
    base order, rows are sorted by nonzero count, descending and stable."""
    ro, _ = _orders(A, row_order, None)
    nnz = [(int(np.count_nonzero(A[i])), i) for i in ro]
    out = []
    for w0 in range(0, len(ro), sigma):
        win = list(range(w0, min(w0 + sigma, len(ro))))
        win.sort(key=lambda p: -nnz[p][0])       # Python's sort is stable
        out.extend(ro[p] for p in win)
    return np.array(out, dtype=np.int64)


def to_sell(A, C, sigma=1, row_order=None, col_order=None):
    """Sliced ELLPACK (Listing 4) generalised to SELL-C-sigma.

    Rows (in `sell_row_order`) are cut into slices of C rows; each slice is
    padded to its longest row and stored column-major: entry k of the r-th row
    of slice s sits at slice_ptr[s] + k*C + r.  Pads hold value 0 and, as
    column, the row's last real column (0 for an empty row); rows past the end
    of the matrix have row_id -1.  Returns (val, col_ind, slice_ptr, slice_len,
    row_id)."""
    _, co = _orders(A, None, col_order)
    rows = sell_row_order(A, C, sigma, row_order)
    n = len(rows)
    n_sl = (n + C - 1) // C
    val, col_ind, slice_ptr, slice_len = [], [], [0], []
    row_id = np.full(n_sl * C, -1, dtype=np.int64)
    row_id[:n] = rows
    for s in range(n_sl):
        ents = []
        for r in range(C):
            i = row_id[s * C + r]
            ents.append([] if i < 0 else [(A[i, j], j) for j in co if A[i, j] != 0])
        L = max(len(e) for e in ents)
        slice_len.append(L)
        for k in range(L):
            for r in range(C):
                e = ents[r]
                if k < len(e):
                    v, j = e[k]
                else:
                    v, j = 0.0, (e[-1][1] if e else 0)
                val.append(v)
                col_ind.append(j)
        slice_ptr.append(len(val))
    return (np.array(val, dtype=float), np.array(col_ind, dtype=np.int64),
            np.array(slice_ptr, dtype=np.int64), np.array(slice_len, dtype=np.int64),
            row_id)


def crs_matvec(fmt, x, n_row):
    """y = A x by the CRS loop of Listing 3 (used to check formats)."""
    val, col_ind, row_ptr, row_id = fmt
    y = np.zeros(n_row)
    for p in range(len(row_id)):
        s = 0.0
        for q in range(row_ptr[p], row_ptr[p + 1]):
            s += val[q] * x[col_ind[q]]
        y[row_id[p]] = s
    return y


def ccs_matvec(fmt, x, n_row):
    """y = A x by the CCS loop of Listing 2."""
    val, row_ind, col_ptr, col_id = fmt
    y = np.zeros(n_row)
    for p in range(len(col_id)):
        for q in range(col_ptr[p], col_ptr[p + 1]):
            y[row_ind[q]] += val[q] * x[col_id[p]]
    return y


def coo_matvec(fmt, x, n_row):
    """y = A x by the COO loop of Listing 1."""
    val, row_ind, col_ind = fmt
    y = np.zeros(n_row)
    for k in range(len(val)):
        y[row_ind[k]] += val[k] * x[col_ind[k]]
    return y


def sell_matvec(fmt, x, n_row, C):
    """y = A x by the SELL loop of Listing 4 (slice by slice, column-major)."""
    val, col_ind, slice_ptr, slice_len, row_id = fmt
    y = np.zeros(n_row)
    for s in range(len(slice_len)):
        for k in range(slice_len[s]):
            for r in range(C):
                q = slice_ptr[s] + k * C + r
                i = row_id[s * C + r]
                if i >= 0:
                    y[i] += val[q] * x[col_ind[q]]
    return y


# ----------------------------------------------------------------------------
# Section 3: row reorderings
# ----------------------------------------------------------------------------

def order_nnz(S) -> np.ndarray:
    """Rows by number of nonzeros, descending; equal counts keep their order."""
    nnz = [int(np.count_nonzero(S[i])) for i in range(S.shape[0])]
    return np.array(sorted(range(S.shape[0]), key=lambda i: -nnz[i]), dtype=np.int64)


def species_graph(S):
    """Adjacency lists of pattern(S S^T) without self loops, ascending."""
    n = S.shape[0]
    nz = (S != 0).astype(np.int64)
    G = (nz @ nz.T) > 0
    return [[l for l in range(n) if l != i and G[i, l]] for i in range(n)]


def _bfs_levels(adj, root, allowed):
    level = {root: 0}
    frontier = [root]
    levels = [[root]]
    while frontier:
        nxt = []
        for v in frontier:
            for u in adj[v]:
                if allowed[u] and u not in level:
                    level[u] = level[v] + 1
                    nxt.append(u)
        if nxt:
            levels.append(nxt)
        frontier = nxt
    return levels


def order_rcm(S):
    """Reverse Cuthill-McKee on pattern(S S^T).

    Per connected component (components taken in order of their lowest
    species index): start from the lowest-index node of minimum degree, move to
    a George-Liu pseudo-peripheral node (repeat: take the minimum-degree node,
    lowest index on ties, of the last BFS level; keep it while the level count
    grows), then Cuthill-McKee BFS visiting each node's unvisited neighbours by
    (degree, index).  The concatenated order is reversed at the end.

    Returns (row_order, col_order): reactions are stably sorted by the smallest
    new position of their species."""
    n = S.shape[0]
    adj = species_graph(S)
    deg = [len(a) for a in adj]
    visited = [False] * n
    cm = []
    for v0 in range(n):
        if visited[v0]:
            continue
        comp_nodes = sorted(x for lv in _bfs_levels(adj, v0, [not b for b in visited]) for x in lv)
        allowed = [False] * n
        for x in comp_nodes:
            allowed[x] = True
        root = min(comp_nodes, key=lambda x: (deg[x], x))
        levels = _bfs_levels(adj, root, allowed)
        while True:
            cand = min(levels[-1], key=lambda x: (deg[x], x))
            lv2 = _bfs_levels(adj, cand, allowed)
            if len(lv2) > len(levels):
                root, levels = cand, lv2
            else:
                break
        visited[root] = True
        queue = [root]
        head = 0
        while head < len(queue):
            v = queue[head]
            head += 1
            nb = sorted((u for u in adj[v] if not visited[u]), key=lambda x: (deg[x], x))
            for u in nb:
                visited[u] = True
                queue.append(u)
        cm.extend(queue)
    rows = np.array(cm[::-1], dtype=np.int64)
    pos = np.empty(n, dtype=np.int64)
    pos[rows] = np.arange(n)
    keys = []
    for j in range(S.shape[1]):
        sp = np.nonzero(S[:, j])[0]
        keys.append(int(pos[sp].min()) if len(sp) else n)
    cols = np.array(sorted(range(S.shape[1]), key=lambda j: keys[j]), dtype=np.int64)
    return rows, cols
