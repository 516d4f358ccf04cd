// Internal structures of the stoichiometry-matrix library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "stoich.h"

// Jacobian entries with more terms than this are gathered by a whole warp.
constexpr int kJLong = 32;

// Device status word bits written by kernels (never trap).
enum : int32_t {
  DEV_ERR_NONE = 0,
  DEV_ERR_BOUNDS = 1,   // an index check failed; the access was skipped
  DEV_ERR_TIMEOUT = 2,  // a bounded wait ran out
};

#define SM_TRY_CUDA(expr)                                      \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) {                                   \
      sm_set_last_cuda_error(_e, #expr);                       \
      return (_e == cudaErrorMemoryAllocation) ? SM_ENOMEM : SM_ECUDA; \
    }                                                          \
  } while (0)

void sm_set_last_cuda_error(cudaError_t e, const char* what);

// Rate-law parameters of one reaction: (log alpha for two-body classes,
// alpha otherwise; beta; gamma; class as a double).
struct __align__(32) RatePar {
  double x, y, z, w;
};

// A device allocation owned by a handle.
struct DevArray {
  void* p = nullptr;
  size_t bytes = 0;
  sm_status upload(const void* h, size_t n);
  sm_status ensure(size_t n);  // grow (no copy) to at least n bytes
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Traversal format as uploaded: see the sm_net_export documentation.
struct Format {
  int32_t fmt = SM_FMT_CRS, order = SM_ORDER_NONE, C = 1, sigma = 1;
  std::vector<int32_t> ptr, idx, idx2, len;
  std::vector<double> val;
  // Device-only companion indices: CRS row ids, CCS column ids, COO column
  // per nonzero, SELL row ids (-1 = padding row).
  std::vector<int32_t> aux;
  // Packed device entries: column (or row) in the low 24 bits, signed
  // coefficient in the high 8 bits.
  std::vector<uint32_t> packed;
  // CRS partitions: per chunk the first nonzero, for 32 chunks (chunk_nz,
  // the default 16-cell gather) and for 64 / 16 chunks (the 8- and 32-cell
  // gathers of the integrator), n_chunks + 1 entries each.
  std::vector<int32_t> chunk_nz, chunk_nz64, chunk_nz16;
  DevArray d_ptr, d_packed, d_aux, d_chunk, d_chunk64, d_chunk16;
};

// Symbolic LU of the Newton matrix M = I - gamma J (no pivoting).
struct LUSymbolic {
  int32_t n = 0, ld = 0, head = 0;
  std::vector<int32_t> perm, iperm;       // perm[p] = species at position p
  std::vector<int32_t> lptr, lidx;        // per pivot: rows below it (positions)
  std::vector<int32_t> uptr, uidx;        // per pivot: columns right of it
  std::vector<int32_t> lrptr, lridx;      // per row: columns of L left of the diagonal
  std::vector<int32_t> ucptr, ucidx;      // per tail column j >= head: head rows k with U(k, j) != 0
  std::vector<int32_t> jrc;               // per J pattern entry: (row position << 16) | column position
  std::vector<int32_t> lrhead;            // per tail row: entries of its L row in head columns
  std::vector<int32_t> lrhoff;            // exclusive prefix sum of lrhead (n - head + 1 entries)
  std::vector<int32_t> u12off;            // per head row: start of its tail-column U entries, packed
  std::vector<int32_t> lrhk;              // head column of each L21 entry in compact row order
  std::vector<int32_t> srow;              // tail rows with L21 entries, longest first
  std::vector<int32_t> uoff;              // per head row k: [n_panels + 1] offsets into its U list where
                                          // the tail columns of each 32-wide panel start
  std::vector<int32_t> jpos;              // per J pattern entry: dense offset p*ld+q
  // Packed factor layout read by the substitution (per cell, values only,
  // in the precision of the factors), segment offsets in elements:
  //   [p_l11, +lrptr[head])   L11: head rows' L entries, order of lrptr/lridx
  //   [p_u11, +u11ptr[head])  U11: head rows' U entries in head columns
  //   [p_dinv, +head)         inverse pivots of the head
  //   [p_l21, +lrhoff[nt])    L21: tail rows' L entries in head columns
  //   [p_u12, +u12off[head])  U12: head rows' U entries in tail columns
  //   [p_d, +nt * ldd)        the dense tail block, column-major (L below the
  //                           diagonal, U above, inverse pivots on it)
  int32_t p_l11 = 0, p_u11 = 0, p_dinv = 0, p_l21 = 0, p_u12 = 0, p_d = 0, ldd = 0;
  int64_t p_size = 0;
  std::vector<int32_t> u11ptr;            // per head row: start of its U11 entries (head + 1)
  std::vector<int32_t> flev_ptr, flev;    // head rows grouped by forward-substitution level
  std::vector<int32_t> blev_ptr, blev;    // head rows grouped by backward-substitution level
  // Head program of the refresh: the sparse head's factors (L11, U11, inverse
  // pivots, L21, U12) computed in the packed layout, level by level.  Pivot k
  // depends on the pivots m < k with l_km or u_mk nonzero; all pivots of one
  // level are independent.  Per level l, ops [hop_ptr[2l], hop_ptr[2l+1]) are
  // the level's pivots, [hop_ptr[2l+1], hop_ptr[2l+2]) its U-row and L-column
  // entries.  An op is {packed index written, offset in the dense working
  // matrix read, first term, end of terms}; its value is
  //   a - sum over its terms (x, y) of H[x] * H[y]
  // (H = the packed head values), inverted for a pivot, times H[hop_piv]
  // (the inverse pivot) for an L entry (hop_piv = -1 otherwise).
  std::vector<int32_t> hop_ptr, hop, hop_piv, hterm;   // hop: 4 ints per op, hterm: 2 per term
  int32_t n_hlev = 0;
  int64_t nnz = 0, flops = 0;
  DevArray d_u11ptr, d_flev_ptr, d_flev, d_blev_ptr, d_blev, d_hop_ptr, d_hop, d_hop_piv, d_hterm;
  DevArray d_lptr, d_lidx, d_uptr, d_uidx, d_lrptr, d_lridx, d_ucptr, d_ucidx, d_jpos, d_perm, d_iperm,
      d_jrc, d_uoff, d_lrhead, d_lrhoff, d_u12off, d_lrhk, d_srow;
};

struct sm_net {
  int device = 0;
  int32_t n_s = 0, n_r = 0, n_elem = 0;
  std::vector<int32_t> comp, reac, prod;
  std::vector<int8_t> cls;
  std::vector<double> alpha, beta, gamma;
  std::vector<int32_t> order;  // reactants per reaction
  // S in column-compressed form, original order, rows ascending.
  std::vector<int32_t> s_colptr, s_row;
  std::vector<int8_t> s_coef;
  // Row orders and column orders for SM_ORDER_NONE / NNZ / RCM.
  std::vector<int32_t> row_order[3], col_order[3];
  Format cur;
  // The integrator's masked CRS gather: CRS in each row order (NONE, NNZ,
  // RCM; built on first use and kept for the network's life, so that a
  // captured graph never refers to released arrays), the selected order and
  // the cells per CTA of the gather (8, 16 or 32), chosen by sm_net_autotune.
  Format integ_fmt[3];
  int32_t integ_order = SM_ORDER_NONE, integ_kc = 16;
  // Jacobian pattern (CRS, species order) and contribution list per entry:
  // term = coef * k'[j] * (partner >= 0 ? y[partner] : 1).
  std::vector<int32_t> jp_ptr, jp_col, jt_ptr, jt_rx, jt_partner;
  std::vector<int8_t> jt_coef;
  LUSymbolic lu;
  // Device copies used by the kernels.
  DevArray d_reac;        // int2 per reaction: reactant indices (-1 = none)
  DevArray d_rate;        // RatePar per reaction: (log alpha | alpha, beta, gamma, class)
  DevArray d_jp_ptr, d_jt_ptr, d_jt_word;  // Jacobian gather lists
  DevArray d_jt_slot;                      // (reaction | coef << 24, reactant slot) per term
  std::vector<int32_t> jlong;              // Jacobian entries with more than kJLong terms
  DevArray d_jdesc, d_jlong;               // per entry {t0, t1, jrc, row << 16 | col}; long entries
  DevArray d_sc_ptr, d_sc_ent;             // S by columns: pointers and (species | coef << 24)
  std::vector<int32_t> jchunk;             // J entries per gather chunk (balanced by terms)
  DevArray d_jchunk;
  DevArray d_status;      // int32 device status word
  DevArray d_scratch;     // reaction-rate scratch for rhs_eval
  sm_net_info info{};
  // Coupled temperature (sm_net_set_thermal; states copy it at creation):
  // slot th_t holds T (-1: off), line-cooling coefficients and excitation
  // temperatures per species, and the constant parameters.
  int32_t th_t = -1;
  double th_heat = 0.0, th_lam = 0.0, th_Td = 0.0, th_zeta = 0.0;
  std::vector<double> th_L, th_E;
};

// Host-side builders (net_build.cpp).
sm_status net_build_host(const sm_net_desc* d, sm_net* net);
sm_status net_upload(sm_net* net);
sm_status net_select_format(sm_net* net, int32_t fmt, int32_t order, int32_t C, int32_t sigma);
sm_status build_format(const sm_net* net, int32_t fmt, int32_t order, int32_t C, int32_t sigma,
                       Format* out);
// Builds (once) the integrator's CRS format in row order `order`.
sm_status integ_format(sm_net* net, int32_t order);

// Kernel launchers (one per .cu file).
sm_status launch_rates(const sm_net* net, int64_t C, const double* T, const double* nH,
                       const double* Av, const double* chi, double zeta, double* k, int64_t ld, cudaStream_t s);
sm_status launch_rhs(const sm_net* net, int64_t C, const double* k, const double* y,
                     double* f, int64_t ld, double* scratch, int64_t ld_scratch, cudaStream_t s);
// Masked CRS right-hand side for the integrator: cells whose mask word has
// `bit` set are evaluated; whole thread blocks without such a cell exit, and
// with cact (device, may be null) so do blocks of cells at or past *cact.
sm_status launch_rhs_masked(const sm_net* net, int64_t C, const double* k, int64_t ldk,
                            const double* y, double* f, int64_t ld, double* scratch, int64_t ldr,
                            const int* mask, int bit, const int* cact, cudaStream_t s);
// Per-device set-up of the right-hand-side kernels (constant tables); called
// when a network is uploaded.
sm_status rhs_prepare_device(int device);
sm_status launch_jac(const sm_net* net, int64_t C, const double* k, const double* y,
                     double* J, int64_t ld, cudaStream_t s);

inline bool ld_ok(int64_t C, int64_t ld) { return C >= 0 && ld >= C && ld % 32 == 0; }
