// Host-side network construction: validation, the stoichiometry matrix (Eq. 7),
// row / column orders (Section 3 reordering, plus reverse Cuthill-McKee), the
// four storage formats of Section 2.2, the Jacobian pattern with its gather
// lists, and the symbolic LU of the Newton matrix.  Everything here runs once
// per network; the results are uploaded and shared by all cells.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace {

// ---------------------------------------------------------------------------
// Orders
// ---------------------------------------------------------------------------

// Rows by nonzero count, descending, equal counts in original order.
std::vector<int32_t> order_by_nnz(const std::vector<int32_t>& row_nnz) {
  std::vector<int32_t> o(row_nnz.size());
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(),
                   [&](int32_t a, int32_t b) { return row_nnz[a] > row_nnz[b]; });
  return o;
}

// Number of BFS levels from `root` inside the nodes flagged in `inside`, and
// the nodes of the last level.
int bfs_depth(const std::vector<std::vector<int32_t>>& adj, const std::vector<char>& inside,
              int32_t root, std::vector<int32_t>* last) {
  std::vector<int32_t> lvl(adj.size(), -1);
  std::vector<int32_t> cur{root}, nxt;
  lvl[root] = 0;
  int depth = 1;
  for (;;) {
    nxt.clear();
    for (int32_t v : cur)
      for (int32_t u : adj[v])
        if (inside[u] && lvl[u] < 0) {
          lvl[u] = lvl[v] + 1;
          nxt.push_back(u);
        }
    if (nxt.empty()) break;
    ++depth;
    cur.swap(nxt);
  }
  if (last) *last = cur;
  return depth;
}

// Reverse Cuthill-McKee on the species graph pattern(S S^T) (no self loops).
// Per component (in order of lowest species index): start at the lowest-index
// minimum-degree node, walk to a George-Liu pseudo-peripheral node, then BFS
// visiting unvisited neighbours by (degree, index).  The full order is
// reversed; reactions are then stably sorted by their smallest new row.
void order_rcm(const sm_net& net, std::vector<int32_t>* rows, std::vector<int32_t>* cols) {
  const int32_t n = net.n_s;
  std::vector<std::vector<char>> g(n, std::vector<char>(n, 0));
  for (int32_t j = 0; j < net.n_r; ++j)
    for (int32_t p = net.s_colptr[j]; p < net.s_colptr[j + 1]; ++p)
      for (int32_t q = net.s_colptr[j]; q < net.s_colptr[j + 1]; ++q)
        if (p != q) g[net.s_row[p]][net.s_row[q]] = 1;
  std::vector<std::vector<int32_t>> adj(n);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t l = 0; l < n; ++l)
      if (g[i][l]) adj[i].push_back(l);
  std::vector<int32_t> deg(n);
  for (int32_t i = 0; i < n; ++i) deg[i] = (int32_t)adj[i].size();
  auto less_dm = [&](int32_t a, int32_t b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };

  std::vector<char> visited(n, 0);
  std::vector<int32_t> cm;
  cm.reserve(n);
  for (int32_t v0 = 0; v0 < n; ++v0) {
    if (visited[v0]) continue;
    // component of v0 among unvisited nodes
    std::vector<char> inside(n, 0);
    std::vector<int32_t> stack{v0}, comp_nodes;
    inside[v0] = 1;
    while (!stack.empty()) {
      int32_t v = stack.back();
      stack.pop_back();
      comp_nodes.push_back(v);
      for (int32_t u : adj[v])
        if (!visited[u] && !inside[u]) {
          inside[u] = 1;
          stack.push_back(u);
        }
    }
    int32_t root = *std::min_element(comp_nodes.begin(), comp_nodes.end(), less_dm);
    std::vector<int32_t> last;
    int depth = bfs_depth(adj, inside, root, &last);
    for (;;) {
      int32_t cand = *std::min_element(last.begin(), last.end(), less_dm);
      std::vector<int32_t> last2;
      int d2 = bfs_depth(adj, inside, cand, &last2);
      if (d2 > depth) {
        root = cand;
        depth = d2;
        last.swap(last2);
      } else {
        break;
      }
    }
    size_t head = cm.size();
    visited[root] = 1;
    cm.push_back(root);
    while (head < cm.size()) {
      int32_t v = cm[head++];
      std::vector<int32_t> nb;
      for (int32_t u : adj[v])
        if (!visited[u]) nb.push_back(u);
      std::sort(nb.begin(), nb.end(), less_dm);
      for (int32_t u : nb) {
        visited[u] = 1;
        cm.push_back(u);
      }
    }
  }
  rows->assign(cm.rbegin(), cm.rend());
  std::vector<int32_t> pos(n);
  for (int32_t k = 0; k < n; ++k) pos[(*rows)[k]] = k;
  std::vector<int32_t> key(net.n_r);
  for (int32_t j = 0; j < net.n_r; ++j) {
    int32_t m = n;
    for (int32_t p = net.s_colptr[j]; p < net.s_colptr[j + 1]; ++p) m = std::min(m, pos[net.s_row[p]]);
    key[j] = m;
  }
  cols->resize(net.n_r);
  std::iota(cols->begin(), cols->end(), 0);
  std::stable_sort(cols->begin(), cols->end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
}

// ---------------------------------------------------------------------------
// Jacobian pattern and symbolic LU
// ---------------------------------------------------------------------------

void build_jacobian_lists(sm_net& net) {
  const int32_t n = net.n_s;
  // terms[i] : (l, j, partner, coef) for every contribution to row i
  struct Term { int32_t l, j, partner; int8_t coef; };
  std::vector<std::vector<Term>> terms(n);
  for (int32_t j = 0; j < net.n_r; ++j) {
    int32_t a = net.reac[2 * j], b = net.reac[2 * j + 1];
    for (int32_t p = net.s_colptr[j]; p < net.s_colptr[j + 1]; ++p) {
      int32_t i = net.s_row[p];
      int8_t s = net.s_coef[p];
      if (b < 0) {
        terms[i].push_back({a, j, -1, s});
      } else if (a == b) {
        terms[i].push_back({a, j, a, (int8_t)(2 * s)});
      } else {
        terms[i].push_back({a, j, b, s});
        terms[i].push_back({b, j, a, s});
      }
    }
  }
  net.jp_ptr.assign(1, 0);
  net.jp_col.clear();
  net.jt_ptr.assign(1, 0);
  net.jt_rx.clear();
  net.jt_partner.clear();
  net.jt_coef.clear();
  for (int32_t i = 0; i < n; ++i) {
    auto& t = terms[i];
    std::stable_sort(t.begin(), t.end(), [](const Term& x, const Term& y) { return x.l < y.l; });
    std::vector<int32_t> cols;
    for (auto& e : t) cols.push_back(e.l);
    cols.push_back(i);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    size_t q = 0;
    for (int32_t l : cols) {
      net.jp_col.push_back(l);
      while (q < t.size() && t[q].l == l) {
        net.jt_rx.push_back(t[q].j);
        net.jt_partner.push_back(t[q].partner);
        net.jt_coef.push_back(t[q].coef);
        ++q;
      }
      net.jt_ptr.push_back((int32_t)net.jt_rx.size());
    }
    net.jp_ptr.push_back((int32_t)net.jp_col.size());
  }
}

// Greedy minimum degree on the symmetric pattern of J + J^T (ties: lowest
// index), then right-looking symbolic elimination without pivoting.
void build_lu_symbolic(sm_net& net) {
  const int32_t n = net.n_s;
  LUSymbolic& lu = net.lu;
  std::vector<std::vector<char>> g(n, std::vector<char>(n, 0));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = net.jp_ptr[i]; p < net.jp_ptr[i + 1]; ++p) {
      int32_t l = net.jp_col[p];
      if (l != i) g[i][l] = g[l][i] = 1;
    }
  std::vector<char> alive(n, 1);
  std::vector<int32_t> degree(n, 0);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t l = 0; l < n; ++l) degree[i] += g[i][l];
  lu.perm.clear();
  for (int32_t step = 0; step < n; ++step) {
    int32_t v = -1;
    for (int32_t i = 0; i < n; ++i)
      if (alive[i] && (v < 0 || degree[i] < degree[v])) v = i;
    lu.perm.push_back(v);
    alive[v] = 0;
    std::vector<int32_t> nb;
    for (int32_t u = 0; u < n; ++u)
      if (alive[u] && g[v][u]) nb.push_back(u);
    for (int32_t a : nb)
      for (int32_t b : nb)
        if (a != b && !g[a][b]) g[a][b] = 1;
    for (int32_t u = 0; u < n; ++u)
      if (g[v][u]) {
        g[v][u] = g[u][v] = 0;
      }
    for (int32_t i = 0; i < n; ++i) {
      if (!alive[i]) continue;
      int32_t d = 0;
      for (int32_t l = 0; l < n; ++l) d += alive[l] && g[i][l];
      degree[i] = d;
    }
  }
  lu.n = n;
  lu.ld = (n + 7) / 8 * 8;
  lu.iperm.assign(n, 0);
  for (int32_t p = 0; p < n; ++p) lu.iperm[lu.perm[p]] = p;
  // permuted structural pattern (unsymmetric) + diagonal
  std::vector<std::vector<char>> f(n, std::vector<char>(n, 0));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = net.jp_ptr[i]; p < net.jp_ptr[i + 1]; ++p)
      f[lu.iperm[i]][lu.iperm[net.jp_col[p]]] = 1;
  for (int32_t i = 0; i < n; ++i) f[i][i] = 1;
  lu.lptr.assign(1, 0);
  lu.uptr.assign(1, 0);
  lu.lidx.clear();
  lu.uidx.clear();
  lu.flops = 0;
  for (int32_t k = 0; k < n; ++k) {
    std::vector<int32_t> L, U;
    for (int32_t i = k + 1; i < n; ++i)
      if (f[i][k]) L.push_back(i);
    for (int32_t j = k + 1; j < n; ++j)
      if (f[k][j]) U.push_back(j);
    for (int32_t i : L)
      for (int32_t j : U) f[i][j] = 1;
    lu.lidx.insert(lu.lidx.end(), L.begin(), L.end());
    lu.uidx.insert(lu.uidx.end(), U.begin(), U.end());
    lu.lptr.push_back((int32_t)lu.lidx.size());
    lu.uptr.push_back((int32_t)lu.uidx.size());
    lu.flops += (int64_t)L.size() + 2 * (int64_t)L.size() * (int64_t)U.size();
  }
  lu.nnz = n + (int64_t)lu.lidx.size() + (int64_t)lu.uidx.size();
  // row-wise view of L (for row-oriented forward substitution)
  {
    std::vector<std::vector<int32_t>> rows(n);
    for (int32_t k = 0; k < n; ++k)
      for (int32_t p = lu.lptr[k]; p < lu.lptr[k + 1]; ++p) rows[lu.lidx[p]].push_back(k);
    lu.lrptr.assign(1, 0);
    lu.lridx.clear();
    for (int32_t i = 0; i < n; ++i) {
      lu.lridx.insert(lu.lridx.end(), rows[i].begin(), rows[i].end());
      lu.lrptr.push_back((int32_t)lu.lridx.size());
    }
  }
  // head: first pivot from which the trailing block is at least 90 % filled
  lu.head = n;
  for (int32_t k = 0; k < n; ++k) {
    int64_t cnt = 0, m = n - k;
    for (int32_t i = k; i < n; ++i)
      for (int32_t j = k; j < n; ++j) cnt += f[i][j];
    if (cnt * 10 >= m * m * 9) {
      lu.head = k;
      break;
    }
  }
  // column-wise view of the U entries of head rows in tail columns
  {
    const int32_t h = lu.head;
    std::vector<std::vector<int32_t>> cols(n);
    for (int32_t k = 0; k < h; ++k)
      for (int32_t p = lu.uptr[k]; p < lu.uptr[k + 1]; ++p)
        if (lu.uidx[p] >= h) cols[lu.uidx[p]].push_back(k);
    lu.ucptr.assign(1, 0);
    lu.ucidx.clear();
    for (int32_t j = h; j < n; ++j) {
      lu.ucidx.insert(lu.ucidx.end(), cols[j].begin(), cols[j].end());
      lu.ucptr.push_back((int32_t)lu.ucidx.size());
    }
  }
  // per head row: where each 32-wide tail panel's columns start in its U list
  {
    const int32_t h = lu.head, np = (n - h + 31) / 32;
    lu.uoff.assign((size_t)h * (np + 1), 0);
    for (int32_t k = 0; k < h; ++k)
      for (int32_t b = 0; b <= np; ++b) {
        const int32_t c0 = h + 32 * b;
        int32_t p = lu.uptr[k];
        while (p < lu.uptr[k + 1] && lu.uidx[p] < c0) ++p;
        lu.uoff[(size_t)k * (np + 1) + b] = p;
      }
  }
  lu.lrhead.assign(n - lu.head, 0);
  for (int32_t i = lu.head; i < n; ++i) {
    int32_t cnt = 0;
    for (int32_t p = lu.lrptr[i]; p < lu.lrptr[i + 1] && lu.lridx[p] < lu.head; ++p) ++cnt;
    lu.lrhead[i - lu.head] = cnt;
  }
  lu.lrhoff.assign(1, 0);
  for (int32_t v : lu.lrhead) lu.lrhoff.push_back(lu.lrhoff.back() + v);
  lu.lrhk.clear();
  for (int32_t i = lu.head; i < n; ++i)
    for (int32_t q = 0; q < lu.lrhead[i - lu.head]; ++q) lu.lrhk.push_back(lu.lridx[lu.lrptr[i] + q]);
  // tail rows that receive head contributions, longest L21 row first (the
  // refresh kernel deals them to warps round-robin)
  lu.srow.clear();
  for (int32_t i = 0; i < n - lu.head; ++i)
    if (lu.lrhead[i] > 0) lu.srow.push_back(i);
  std::stable_sort(lu.srow.begin(), lu.srow.end(),
                   [&](int32_t a, int32_t b) { return lu.lrhead[a] > lu.lrhead[b]; });
  {
    const int32_t np1 = (n - lu.head + 31) / 32 + 1;
    lu.u12off.assign(1, 0);
    for (int32_t k = 0; k < lu.head; ++k)
      lu.u12off.push_back(lu.u12off.back() + lu.uptr[k + 1] - lu.uoff[(size_t)k * np1]);
  }
  // packed factor layout of the substitution and the level sets of its
  // sparse head: a head row's level is one more than the highest level among
  // the rows its L11 (forward) or U11 (backward) entries refer to, so all
  // rows of one level can be resolved at once
  {
    const int32_t h = lu.head, nt = n - h, np1 = (nt + 31) / 32 + 1;
    lu.u11ptr.assign(1, 0);
    for (int32_t k = 0; k < h; ++k) lu.u11ptr.push_back(lu.u11ptr.back() + lu.uoff[(size_t)k * np1] - lu.uptr[k]);
    auto group = [](const std::vector<int32_t>& lev, std::vector<int32_t>& ptr, std::vector<int32_t>& rows) {
      int32_t top = 0;
      for (int32_t v : lev) top = std::max(top, v + 1);
      ptr.assign(top + 1, 0);
      for (int32_t v : lev) ++ptr[v + 1];
      for (int32_t l = 0; l < top; ++l) ptr[l + 1] += ptr[l];
      rows.assign(lev.size(), 0);
      std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
      for (int32_t i = 0; i < (int32_t)lev.size(); ++i) rows[fill[lev[i]]++] = i;
    };
    std::vector<int32_t> fl(h, 0), bl(h, 0);
    for (int32_t i = 0; i < h; ++i)
      for (int32_t p = lu.lrptr[i]; p < lu.lrptr[i + 1]; ++p) fl[i] = std::max(fl[i], fl[lu.lridx[p]] + 1);
    for (int32_t k = h - 1; k >= 0; --k)
      for (int32_t p = lu.uptr[k]; p < lu.uoff[(size_t)k * np1]; ++p) bl[k] = std::max(bl[k], bl[lu.uidx[p]] + 1);
    group(fl, lu.flev_ptr, lu.flev);
    group(bl, lu.blev_ptr, lu.blev);
    auto up32 = [](int64_t v) { return (v + 31) / 32 * 32; };
    lu.p_l11 = 0;
    lu.p_u11 = (int32_t)up32(lu.p_l11 + (h > 0 ? lu.lrptr[h] : 0));
    lu.p_dinv = (int32_t)up32(lu.p_u11 + lu.u11ptr[h]);
    lu.p_l21 = (int32_t)up32(lu.p_dinv + h);
    lu.p_u12 = (int32_t)up32(lu.p_l21 + lu.lrhoff.back());
    lu.p_d = (int32_t)up32(lu.p_u12 + lu.u12off.back());
    lu.ldd = (int32_t)up32(nt);
    lu.p_size = up32((int64_t)lu.p_d + (int64_t)nt * lu.ldd);

    // head program: packed index of every head factor entry, pivot levels,
    // and the product terms of each entry's left-looking update
    const int32_t ld = lu.ld;
    std::vector<int32_t> lpos((size_t)n * std::max(h, 1), -1), upos((size_t)std::max(h, 1) * n, -1);
    for (int32_t i = 0; i < h; ++i)
      for (int32_t p = lu.lrptr[i]; p < lu.lrptr[i + 1]; ++p) lpos[(size_t)i * h + lu.lridx[p]] = lu.p_l11 + p;
    for (int32_t i = h; i < n; ++i)
      for (int32_t q = 0; q < lu.lrhead[i - h]; ++q)
        lpos[(size_t)i * h + lu.lridx[lu.lrptr[i] + q]] = lu.p_l21 + lu.lrhoff[i - h] + q;
    for (int32_t k = 0; k < h; ++k)
      for (int32_t p = lu.uptr[k]; p < lu.uptr[k + 1]; ++p) {
        const int32_t j = lu.uidx[p];
        const int32_t q12 = lu.uoff[(size_t)k * np1];
        upos[(size_t)k * n + j] = j < h ? lu.p_u11 + lu.u11ptr[k] + (p - lu.uptr[k])
                                        : lu.p_u12 + lu.u12off[k] + (p - q12);
      }
    // U11 columns: head rows m < k with u_mk != 0
    std::vector<std::vector<int32_t>> ucol11(h);
    for (int32_t m = 0; m < h; ++m)
      for (int32_t p = lu.uptr[m]; p < lu.uoff[(size_t)m * np1]; ++p) ucol11[lu.uidx[p]].push_back(m);
    std::vector<int32_t> lev(h, 0);
    for (int32_t k = 0; k < h; ++k) {
      for (int32_t p = lu.lrptr[k]; p < lu.lrptr[k + 1]; ++p) lev[k] = std::max(lev[k], lev[lu.lridx[p]] + 1);
      for (int32_t m : ucol11[k]) lev[k] = std::max(lev[k], lev[m] + 1);
    }
    int32_t nl = 0;
    for (int32_t v : lev) nl = std::max(nl, v + 1);
    lu.n_hlev = nl;
    lu.hop.clear();
    lu.hop_piv.clear();
    lu.hterm.clear();
    lu.hop_ptr.assign(1, 0);
    auto add_op = [&](int32_t dst, int32_t src, int32_t piv, const std::vector<std::pair<int32_t, int32_t>>& t) {
      lu.hop.push_back(dst);
      lu.hop.push_back(src);
      lu.hop.push_back((int32_t)lu.hterm.size() / 2);
      for (auto& e : t) {
        lu.hterm.push_back(e.first);
        lu.hterm.push_back(e.second);
      }
      lu.hop.push_back((int32_t)lu.hterm.size() / 2);
      lu.hop_piv.push_back(piv);
    };
    for (int32_t l = 0; l < nl; ++l) {
      // pivots: u_kk = a_kk - sum_m l_km u_mk
      for (int32_t k = 0; k < h; ++k) {
        if (lev[k] != l) continue;
        std::vector<std::pair<int32_t, int32_t>> t;
        for (int32_t p = lu.lrptr[k]; p < lu.lrptr[k + 1]; ++p) {
          const int32_t m = lu.lridx[p];
          if (upos[(size_t)m * n + k] >= 0) t.push_back({lpos[(size_t)k * h + m], upos[(size_t)m * n + k]});
        }
        add_op(lu.p_dinv + k, k * ld + k, -1, t);
      }
      lu.hop_ptr.push_back((int32_t)lu.hop_piv.size());
      for (int32_t k = 0; k < h; ++k) {
        if (lev[k] != l) continue;
        // U row k: u_kj = a_kj - sum_m l_km u_mj
        for (int32_t p = lu.uptr[k]; p < lu.uptr[k + 1]; ++p) {
          const int32_t j = lu.uidx[p];
          std::vector<std::pair<int32_t, int32_t>> t;
          for (int32_t q = lu.lrptr[k]; q < lu.lrptr[k + 1]; ++q) {
            const int32_t m = lu.lridx[q];
            if (upos[(size_t)m * n + j] >= 0) t.push_back({lpos[(size_t)k * h + m], upos[(size_t)m * n + j]});
          }
          add_op(upos[(size_t)k * n + j], k * ld + j, -1, t);
        }
        // L column k: l_ik = (a_ik - sum_m l_im u_mk) / u_kk
        for (int32_t p = lu.lptr[k]; p < lu.lptr[k + 1]; ++p) {
          const int32_t i = lu.lidx[p];
          std::vector<std::pair<int32_t, int32_t>> t;
          for (int32_t m : ucol11[k])
            if (lpos[(size_t)i * h + m] >= 0) t.push_back({lpos[(size_t)i * h + m], upos[(size_t)m * n + k]});
          add_op(lpos[(size_t)i * h + k], i * ld + k, lu.p_dinv + k, t);
        }
      }
      lu.hop_ptr.push_back((int32_t)lu.hop_piv.size());
    }
  }
  lu.jpos.resize(net.jp_col.size());
  lu.jrc.resize(net.jp_col.size());
  for (int32_t i = 0; i < n; ++i)
    for (int32_t p = net.jp_ptr[i]; p < net.jp_ptr[i + 1]; ++p)
    {
      lu.jpos[p] = lu.iperm[i] * lu.ld + lu.iperm[net.jp_col[p]];
      lu.jrc[p] = (lu.iperm[i] << 16) | lu.iperm[net.jp_col[p]];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Build
// ---------------------------------------------------------------------------

sm_status net_build_host(const sm_net_desc* d, sm_net* net) {
  if (!d || d->n_s <= 0 || d->n_r <= 0 || d->n_elem < 0 || !d->comp || !d->reactants ||
      !d->products || !d->rclass || !d->alpha || !d->beta || !d->gamma)
    return SM_EINVAL;
  if (d->n_s >= (1 << 23) || d->n_r >= (1 << 23)) return SM_EINVAL;
  const int32_t n_s = d->n_s, n_r = d->n_r, ne = d->n_elem + 1;
  net->n_s = n_s;
  net->n_r = n_r;
  net->n_elem = d->n_elem;
  net->comp.assign(d->comp, d->comp + (size_t)n_s * ne);
  net->reac.assign(d->reactants, d->reactants + 2 * (size_t)n_r);
  net->prod.assign(d->products, d->products + 4 * (size_t)n_r);
  net->cls.assign(d->rclass, d->rclass + n_r);
  net->alpha.assign(d->alpha, d->alpha + n_r);
  net->beta.assign(d->beta, d->beta + n_r);
  net->gamma.assign(d->gamma, d->gamma + n_r);
  net->order.assign(n_r, 0);
  for (int32_t j = 0; j < n_r; ++j) {
    int32_t a = net->reac[2 * j], b = net->reac[2 * j + 1];
    if (a < 0 || a >= n_s || b < -1 || b >= n_s) return SM_EINVAL;
    net->order[j] = b >= 0 ? 2 : 1;
    for (int q = 0; q < 4; ++q) {
      int32_t p = net->prod[4 * j + q];
      if (p < -1 || p >= n_s) return SM_EINVAL;
    }
    if (net->cls[j] < 0 || net->cls[j] > 3) return SM_EINVAL;
    if (!std::isfinite(net->alpha[j]) || !(net->alpha[j] > 0.0) || !std::isfinite(net->beta[j]) ||
        !std::isfinite(net->gamma[j]))
      return SM_EINVAL;
  }
  // Eq. 7: net coefficient = products - reactants; zero entries dropped.
  net->s_colptr.assign(1, 0);
  net->s_row.clear();
  net->s_coef.clear();
  std::vector<int32_t> cnt(n_s, 0);
  for (int32_t j = 0; j < n_r; ++j) {
    std::vector<int32_t> touched;
    for (int q = 0; q < 2; ++q) {
      int32_t a = net->reac[2 * j + q];
      if (a >= 0) { cnt[a] -= 1; touched.push_back(a); }
    }
    for (int q = 0; q < 4; ++q) {
      int32_t p = net->prod[4 * j + q];
      if (p >= 0) { cnt[p] += 1; touched.push_back(p); }
    }
    std::sort(touched.begin(), touched.end());
    touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
    // conservation: sum_i comp[i][e] * S_ij == 0 for every element and charge
    for (int32_t e = 0; e < ne; ++e) {
      int64_t s = 0;
      for (int32_t i : touched) s += (int64_t)net->comp[(size_t)i * ne + e] * cnt[i];
      if (s != 0) return SM_ENOTCONS;
    }
    for (int32_t i : touched) {
      if (cnt[i] != 0) {
        net->s_row.push_back(i);
        net->s_coef.push_back((int8_t)cnt[i]);
      }
      cnt[i] = 0;
    }
    net->s_colptr.push_back((int32_t)net->s_row.size());
  }
  // orders
  std::vector<int32_t> row_nnz(n_s, 0);
  for (int32_t r : net->s_row) row_nnz[r]++;
  net->row_order[SM_ORDER_NONE].resize(n_s);
  std::iota(net->row_order[SM_ORDER_NONE].begin(), net->row_order[SM_ORDER_NONE].end(), 0);
  net->col_order[SM_ORDER_NONE].resize(n_r);
  std::iota(net->col_order[SM_ORDER_NONE].begin(), net->col_order[SM_ORDER_NONE].end(), 0);
  net->row_order[SM_ORDER_NNZ] = order_by_nnz(row_nnz);
  net->col_order[SM_ORDER_NNZ] = net->col_order[SM_ORDER_NONE];
  order_rcm(*net, &net->row_order[SM_ORDER_RCM], &net->col_order[SM_ORDER_RCM]);

  build_jacobian_lists(*net);
  build_lu_symbolic(*net);

  sm_net_info& in = net->info;
  in.n_s = n_s;
  in.n_r = n_r;
  in.nnz_S = (int64_t)net->s_row.size();
  in.nnz_J = (int64_t)net->jp_col.size();
  in.n_jac_terms = (int64_t)net->jt_rx.size();
  in.nnz_LU = net->lu.nnz;
  in.lu_flops = net->lu.flops;
  in.lu_head = net->lu.head;
  in.max_row_nnz = *std::max_element(row_nnz.begin(), row_nnz.end());
  int64_t sum_order = 0;
  for (int32_t j = 0; j < n_r; ++j) sum_order += net->order[j];
  in.rhs_bytes = 8.0 * (n_r + 2.0 * n_s);
  in.rhs_flops = 2.0 * in.nnz_S + (double)sum_order;
  in.jac_bytes = 8.0 * (n_r + n_s + (double)in.nnz_J);
  in.jac_flops = 2.0 * in.n_jac_terms + (double)sum_order;
  in.lu_packed = net->lu.p_size;
  return SM_OK;
}

// ---------------------------------------------------------------------------
// Formats
// ---------------------------------------------------------------------------

namespace {

inline uint32_t pack(int32_t index, int32_t coef) {
  return ((uint32_t)index & 0xFFFFFFu) | ((uint32_t)(uint8_t)(int8_t)coef << 24);
}

}  // namespace

sm_status build_format(const sm_net* net, int32_t fmt, int32_t order, int32_t C, int32_t sigma,
                       Format* out) {
  if (fmt < SM_FMT_CRS || fmt > SM_FMT_SELL || order < SM_ORDER_NONE || order > SM_ORDER_RCM)
    return SM_EINVAL;
  if (fmt == SM_FMT_SELL && (C < 1 || C > 32 || sigma < 1)) return SM_EINVAL;
  const int32_t n_s = net->n_s, n_r = net->n_r;
  const std::vector<int32_t>& ro = net->row_order[order];
  const std::vector<int32_t>& co = net->col_order[order];
  std::vector<int32_t> rpos(n_s), cpos(n_r);
  for (int32_t k = 0; k < n_s; ++k) rpos[ro[k]] = k;
  for (int32_t k = 0; k < n_r; ++k) cpos[co[k]] = k;
  // rows of S as (column, coefficient), columns in traversal order
  std::vector<std::vector<std::pair<int32_t, int32_t>>> rows(n_s);
  for (int32_t j = 0; j < n_r; ++j)
    for (int32_t p = net->s_colptr[j]; p < net->s_colptr[j + 1]; ++p)
      rows[net->s_row[p]].push_back({j, net->s_coef[p]});
  for (auto& r : rows)
    std::sort(r.begin(), r.end(), [&](const std::pair<int32_t, int32_t>& a,
                                      const std::pair<int32_t, int32_t>& b) {
      return cpos[a.first] < cpos[b.first];
    });

  Format f;
  f.fmt = fmt;
  f.order = order;
  f.C = fmt == SM_FMT_SELL ? C : 1;
  f.sigma = fmt == SM_FMT_SELL ? sigma : 1;
  if (fmt == SM_FMT_CRS) {
    f.ptr.push_back(0);
    for (int32_t k = 0; k < n_s; ++k) {
      for (auto& e : rows[ro[k]]) {
        f.idx.push_back(e.first);
        f.val.push_back((double)e.second);
        f.packed.push_back(pack(e.first, e.second));
      }
      f.ptr.push_back((int32_t)f.idx.size());
    }
    f.aux = ro;
  } else if (fmt == SM_FMT_CCS || fmt == SM_FMT_COO) {
    f.ptr.push_back(0);
    for (int32_t k = 0; k < n_r; ++k) {
      int32_t j = co[k];
      std::vector<std::pair<int32_t, int32_t>> ents;
      for (int32_t p = net->s_colptr[j]; p < net->s_colptr[j + 1]; ++p)
        ents.push_back({net->s_row[p], net->s_coef[p]});
      std::sort(ents.begin(), ents.end(), [&](const std::pair<int32_t, int32_t>& a,
                                              const std::pair<int32_t, int32_t>& b) {
        return rpos[a.first] < rpos[b.first];
      });
      for (auto& e : ents) {
        f.idx.push_back(e.first);
        f.val.push_back((double)e.second);
        f.packed.push_back(pack(e.first, e.second));
        if (fmt == SM_FMT_COO) f.idx2.push_back(j);
      }
      f.ptr.push_back((int32_t)f.idx.size());
    }
    f.aux = (fmt == SM_FMT_COO) ? f.idx2 : co;
  } else {
    // SELL-C-sigma: stable sort by nonzero count inside windows of sigma rows
    std::vector<int32_t> srow;
    for (int32_t w0 = 0; w0 < n_s; w0 += sigma) {
      std::vector<int32_t> win(ro.begin() + w0, ro.begin() + std::min(n_s, w0 + sigma));
      std::stable_sort(win.begin(), win.end(), [&](int32_t a, int32_t b) {
        return rows[a].size() > rows[b].size();
      });
      srow.insert(srow.end(), win.begin(), win.end());
    }
    const int32_t n_sl = (n_s + C - 1) / C;
    f.idx2.assign((size_t)n_sl * C, -1);
    std::copy(srow.begin(), srow.end(), f.idx2.begin());
    f.aux = f.idx2;
    f.ptr.push_back(0);
    for (int32_t s = 0; s < n_sl; ++s) {
      int32_t L = 0;
      for (int32_t r = 0; r < C; ++r) {
        int32_t i = f.idx2[(size_t)s * C + r];
        if (i >= 0) L = std::max(L, (int32_t)rows[i].size());
      }
      f.len.push_back(L);
      for (int32_t k = 0; k < L; ++k)
        for (int32_t r = 0; r < C; ++r) {
          int32_t i = f.idx2[(size_t)s * C + r];
          int32_t col = 0, coef = 0;
          if (i >= 0 && k < (int32_t)rows[i].size()) {
            col = rows[i][k].first;
            coef = rows[i][k].second;
          } else if (i >= 0 && !rows[i].empty()) {
            col = rows[i].back().first;
          }
          f.idx.push_back(col);
          f.val.push_back((double)coef);
          f.packed.push_back(pack(col, coef));
        }
      f.ptr.push_back((int32_t)f.idx.size());
    }
  }
  // CRS warp partition: chunks of about equal nonzero count (used by the
  // merge-style CRS kernel; row boundaries are found on the device).
  if (fmt == SM_FMT_CRS) {
    const int32_t nnz = (int32_t)f.idx.size();
    auto part = [&](int32_t n_chunks, std::vector<int32_t>& v) {
      for (int32_t c = 0; c <= n_chunks; ++c) v.push_back((int32_t)((int64_t)nnz * c / n_chunks));
    };
    part(32, f.chunk_nz);    // must match the CRS kernels' chunks per CTA
    part(64, f.chunk_nz64);
    part(16, f.chunk_nz16);
  }
  // upload (skipped for host-only networks, device < 0)
  out->d_ptr.release();
  out->d_packed.release();
  out->d_aux.release();
  out->d_chunk.release();
  out->d_chunk64.release();
  out->d_chunk16.release();
  *out = std::move(f);
  Format& g = *out;
  if (net->device < 0) return SM_OK;
  sm_status st;
  if (!g.ptr.empty() && (st = g.d_ptr.upload(g.ptr.data(), g.ptr.size() * 4)) != SM_OK) return st;
  if ((st = g.d_packed.upload(g.packed.data(), g.packed.size() * 4)) != SM_OK) return st;
  if (!g.aux.empty() && (st = g.d_aux.upload(g.aux.data(), g.aux.size() * 4)) != SM_OK) return st;
  if (!g.chunk_nz.empty() && (st = g.d_chunk.upload(g.chunk_nz.data(), g.chunk_nz.size() * 4)) != SM_OK)
    return st;
  if (!g.chunk_nz64.empty() && (st = g.d_chunk64.upload(g.chunk_nz64.data(), g.chunk_nz64.size() * 4)) != SM_OK)
    return st;
  if (!g.chunk_nz16.empty() && (st = g.d_chunk16.upload(g.chunk_nz16.data(), g.chunk_nz16.size() * 4)) != SM_OK)
    return st;
  return SM_OK;
}

sm_status net_select_format(sm_net* net, int32_t fmt, int32_t order, int32_t C, int32_t sigma) {
  sm_status st = build_format(net, fmt, order, C, sigma, &net->cur);
  if (st != SM_OK) return st;
  net->info.fmt = net->cur.fmt;
  net->info.order = net->cur.order;
  net->info.sell_C = net->cur.C;
  net->info.sell_sigma = net->cur.sigma;
  net->info.fmt_entries = (int64_t)net->cur.idx.size();
  return SM_OK;
}

sm_status net_upload(sm_net* net) {
  const int32_t n_r = net->n_r;
  std::vector<int32_t> reac2(2 * (size_t)n_r);
  std::vector<double> rate(4 * (size_t)n_r);
  for (int32_t j = 0; j < n_r; ++j) {
    reac2[2 * j] = net->reac[2 * j];
    reac2[2 * j + 1] = net->reac[2 * j + 1];
    int c = net->cls[j];
    // two-body classes keep log(alpha) (rate = exp(log alpha + ...)), others alpha
    rate[4 * j + 0] = (c == SM_TWO_BODY || c == SM_DISS_RECOMB) ? std::log(net->alpha[j]) : net->alpha[j];
    rate[4 * j + 1] = net->beta[j];
    rate[4 * j + 2] = net->gamma[j];
    rate[4 * j + 3] = (double)c;
  }
  sm_status st;
  if ((st = rhs_prepare_device(net->device)) != SM_OK) return st;
  if ((st = net->d_reac.upload(reac2.data(), reac2.size() * 4)) != SM_OK) return st;
  if ((st = net->d_rate.upload(rate.data(), rate.size() * 8)) != SM_OK) return st;
  // Jacobian gather words: reaction (low 23 bits) | partner+1 ... packed as two
  // int32 per term: (reaction | coef << 24, partner)
  std::vector<int32_t> words(2 * net->jt_rx.size());
  for (size_t t = 0; t < net->jt_rx.size(); ++t) {
    words[2 * t] = (int32_t)pack(net->jt_rx[t], net->jt_coef[t]);
    words[2 * t + 1] = net->jt_partner[t];
  }
  {
    std::vector<uint32_t> ent(net->s_row.size());
    for (size_t p = 0; p < ent.size(); ++p) ent[p] = pack(net->s_row[p], net->s_coef[p]);
    if ((st = net->d_sc_ptr.upload(net->s_colptr.data(), net->s_colptr.size() * 4)) != SM_OK) return st;
    if ((st = net->d_sc_ent.upload(ent.data(), ent.size() * 4)) != SM_OK) return st;
  }
  if ((st = net->d_jp_ptr.upload(net->jp_ptr.data(), net->jp_ptr.size() * 4)) != SM_OK) return st;
  if ((st = net->d_jt_ptr.upload(net->jt_ptr.data(), net->jt_ptr.size() * 4)) != SM_OK) return st;
  if ((st = net->d_jt_word.upload(words.data(), words.size() * 4)) != SM_OK) return st;
  // the same terms with the reactant slot whose derivative they use: slot 0 =
  // d/d(first reactant) = k' x_second (or k'), slot 1 = d/d(second reactant)
  {
    std::vector<int32_t> ws(2 * net->jt_rx.size());
    for (int32_t i = 0; i < net->n_s; ++i)
      for (int32_t e = net->jp_ptr[i]; e < net->jp_ptr[i + 1]; ++e) {
        const int32_t l = net->jp_col[e];
        for (int32_t t = net->jt_ptr[e]; t < net->jt_ptr[e + 1]; ++t) {
          const int32_t j = net->jt_rx[t];
          ws[2 * t] = (int32_t)pack(j, net->jt_coef[t]);
          ws[2 * t + 1] = net->reac[2 * j] == l ? 0 : 1;
        }
      }
    if ((st = net->d_jt_slot.upload(ws.data(), ws.size() * 4)) != SM_OK) return st;
  }
  // gather chunks of about equal term count over the J pattern entries
  {
    const int64_t n_e = (int64_t)net->jp_col.size(), n_t = (int64_t)net->jt_rx.size();
    const int64_t n_ch = std::max<int64_t>(1, std::min<int64_t>(256, n_e));
    net->jchunk.assign(1, 0);
    int64_t e = 0;
    for (int64_t c = 1; c < n_ch; ++c) {
      const int64_t target = n_t * c / n_ch;
      while (e < n_e && net->jt_ptr[e + 1] <= target) ++e;
      net->jchunk.push_back((int32_t)std::max<int64_t>(e, net->jchunk.back()));
    }
    net->jchunk.push_back((int32_t)n_e);
    if ((st = net->d_jchunk.upload(net->jchunk.data(), net->jchunk.size() * 4)) != SM_OK) return st;
  }
  LUSymbolic& lu = net->lu;
  if ((st = lu.d_lptr.upload(lu.lptr.data(), lu.lptr.size() * 4)) != SM_OK) return st;
  if (!lu.lidx.empty() && (st = lu.d_lidx.upload(lu.lidx.data(), lu.lidx.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_uptr.upload(lu.uptr.data(), lu.uptr.size() * 4)) != SM_OK) return st;
  if (!lu.uidx.empty() && (st = lu.d_uidx.upload(lu.uidx.data(), lu.uidx.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_lrptr.upload(lu.lrptr.data(), lu.lrptr.size() * 4)) != SM_OK) return st;
  if (!lu.lridx.empty() && (st = lu.d_lridx.upload(lu.lridx.data(), lu.lridx.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_ucptr.upload(lu.ucptr.data(), lu.ucptr.size() * 4)) != SM_OK) return st;
  if (!lu.ucidx.empty() && (st = lu.d_ucidx.upload(lu.ucidx.data(), lu.ucidx.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_jpos.upload(lu.jpos.data(), lu.jpos.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_jrc.upload(lu.jrc.data(), lu.jrc.size() * 4)) != SM_OK) return st;
  // one 16-byte descriptor per Jacobian entry for the refresh gather: term
  // range, (row, column) in elimination order, (row, column) species; and
  // the entries with more than kJLong terms, which a warp gathers
  {
    const size_t n_e = net->jp_col.size();
    std::vector<int32_t> desc(4 * n_e);
    net->jlong.clear();
    for (int32_t i = 0; i < net->n_s; ++i)
      for (int32_t e = net->jp_ptr[i]; e < net->jp_ptr[i + 1]; ++e) {
        desc[4 * e] = net->jt_ptr[e];
        desc[4 * e + 1] = net->jt_ptr[e + 1];
        desc[4 * e + 2] = lu.jrc[e];
        desc[4 * e + 3] = (i << 16) | net->jp_col[e];
        if (net->jt_ptr[e + 1] - net->jt_ptr[e] > kJLong) net->jlong.push_back(e);
      }
    if ((st = net->d_jdesc.upload(desc.data(), desc.size() * 4)) != SM_OK) return st;
    if (!net->jlong.empty() && (st = net->d_jlong.upload(net->jlong.data(), net->jlong.size() * 4)) != SM_OK)
      return st;
  }
  if (!lu.uoff.empty() && (st = lu.d_uoff.upload(lu.uoff.data(), lu.uoff.size() * 4)) != SM_OK) return st;
  if (!lu.lrhead.empty() && (st = lu.d_lrhead.upload(lu.lrhead.data(), lu.lrhead.size() * 4)) != SM_OK)
    return st;
  if ((st = lu.d_lrhoff.upload(lu.lrhoff.data(), lu.lrhoff.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_u12off.upload(lu.u12off.data(), lu.u12off.size() * 4)) != SM_OK) return st;
  if (!lu.lrhk.empty() && (st = lu.d_lrhk.upload(lu.lrhk.data(), lu.lrhk.size() * 4)) != SM_OK) return st;
  if (!lu.srow.empty() && (st = lu.d_srow.upload(lu.srow.data(), lu.srow.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_u11ptr.upload(lu.u11ptr.data(), lu.u11ptr.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_hop_ptr.upload(lu.hop_ptr.data(), lu.hop_ptr.size() * 4)) != SM_OK) return st;
  if (!lu.hop.empty() && (st = lu.d_hop.upload(lu.hop.data(), lu.hop.size() * 4)) != SM_OK) return st;
  if (!lu.hop_piv.empty() && (st = lu.d_hop_piv.upload(lu.hop_piv.data(), lu.hop_piv.size() * 4)) != SM_OK)
    return st;
  if (!lu.hterm.empty() && (st = lu.d_hterm.upload(lu.hterm.data(), lu.hterm.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_flev_ptr.upload(lu.flev_ptr.data(), lu.flev_ptr.size() * 4)) != SM_OK) return st;
  if (!lu.flev.empty() && (st = lu.d_flev.upload(lu.flev.data(), lu.flev.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_blev_ptr.upload(lu.blev_ptr.data(), lu.blev_ptr.size() * 4)) != SM_OK) return st;
  if (!lu.blev.empty() && (st = lu.d_blev.upload(lu.blev.data(), lu.blev.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_perm.upload(lu.perm.data(), lu.perm.size() * 4)) != SM_OK) return st;
  if ((st = lu.d_iperm.upload(lu.iperm.data(), lu.iperm.size() * 4)) != SM_OK) return st;
  int32_t zero = 0;
  if ((st = net->d_status.upload(&zero, 4)) != SM_OK) return st;
  return integ_format(net, SM_ORDER_NONE);
}

sm_status integ_format(sm_net* net, int32_t order) {
  if (order < SM_ORDER_NONE || order > SM_ORDER_RCM) return SM_EINVAL;
  if (!net->integ_fmt[order].packed.empty()) return SM_OK;
  return build_format(net, SM_FMT_CRS, order, 1, 1, &net->integ_fmt[order]);
}
