// Batched variable-order BDF integration with simplified Newton iterations
// (the stiff-solver role of DLSODES in Section 3), one independent state
// machine per cell.
//
// One "attempt" advances every unfinished cell by one trial step:
//   predict   32 cells per CTA, the species split over 8 warps: Lagrange
//             predictor, BDF coefficients, weights, and the decision whether
//             the Newton matrix must be refreshed;
//   refresh   one CTA per cell on the compacted refresh list: J at the
//             predicted state, M = I - gamma J (FP64, equilibrated and
//             rounded to FP32 in mixed precision), LU without pivoting in
//             the minimum-degree order, written as packed factors;
//   newton    up to newton_max rounds of: reaction rates + CRS gather of
//             S R(y) (cells fast axis, masked to iterating cells), then one
//             warp per cell forming the FP64 residual, forward/backward
//             substitution and the WRMS convergence test;
//   finish    32 cells per CTA, the species split over 8 warps: error test,
//             order / step selection, history.
// With a coupled temperature (sm_net_set_thermal) the rate coefficients of
// the T-dependent reactions are recomputed from the state before every
// right-hand side, the temperature row follows each gather, and T is
// eliminated last in the Newton solve (th_* kernels below).
// The host enqueues attempts in groups (captured once in a CUDA graph) and
// reads back only the number of running cells between groups.  The same file
// holds the step recording and the discrete adjoint of the frozen-step map
// (sm_state_steps, sm_adjoint, sm_replay) and checkpoint / resume
// (sm_state_save, sm_state_load).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int QMAX = 5;  // highest BDF order; the history keeps QMAX + 1 points
// counters[] entries of the compaction (0..3 belong to the attempt loop and
// the adjoint)
constexpr int kCAct = 8;     // slots holding the running cells: [0, counters[kCAct])
constexpr int kCHoles = 9;   // finished cells below the new boundary
constexpr int kCRun = 10;    // running cells above it
constexpr int kCLive = 11;   // running cells counted for the compaction
constexpr int kCounters = 16;
constexpr int kCkpt = SM_CHECKPOINT_EVERY;
enum : int {
  F_NEED_J = 1, F_REJECTED = 2, F_HAS_EPREV = 4, F_NEWTON = 8, F_CONV = 16,
  F_FINAL = 32, F_REFRESH = 64, F_FAILED = 128, F_ATTEMPT = 256
};

struct Dev {
  int n, n_r, nnz_j, mixed, tf32, head;
  int64_t C, ld;
  double rtol, atol, gamma_tol, newton_tol, eta_max, eta_keep, t_end;
  int q_max, max_steps, j_age_max, newton_max, max_conv_fails;
  // per-cell scalars [ld] (tn, alpha: [QMAX+1][ld])
  double *t, *h, *gam, *gam_J, *crate, *dprev, *tn, *alpha;
  int *q, *nh, *n_at_q, *j_age, *flags, *crej, *ccf, *status, *m_it;
  int *steps, *rejects, *conv_fails, *newton_iters, *jac_evals;
  // per-cell vectors [n][ld]; Y is [QMAX+1][n][ld]
  double *Y, *ypred, *y, *psi, *f, *f0, *eprev, *w, *wf;
  int *list, *counters;  // counters[0] = refresh list length, [1] = running cells
  // compaction of the running cells (states that record no steps): cell
  // slots are permuted so that running cells occupy slots [0, counters[kCAct])
  int* slot_cell;        // [ld] slot -> cell of the caller's arrays (and of the packed factors)
  int compact;           // 1: compaction on
  double* kslot;         // [n_r][ld] rate coefficients in slot order (compaction on), else null
  int *holes, *runners;  // [ld] each: the slot pairs of one compaction
  // recording (record > 0): per accepted step m (1-based) at [m-1][ld]; the
  // step history after every kCkpt-th accepted step at checkpoint m / kCkpt
  int record;
  double *log_t, *log_h;
  int* log_q;
  double *ck_Y, *ck_t;   // [K][QMAX+1][n][ld], [K][QMAX+1][ld]
  int* ck_nh;            // [K][ld]
  void* lu;
  int64_t lu_stride;
  int ldm;
  // packed factors read by the substitution (see LUSymbolic): per cell
  // lup_stride values from lup; null when the state keeps dense factors only
  void* lup;
  int64_t lup_stride;
  int lu_cta;   // 1: lu holds one dense working matrix per refresh CTA (not per cell)
  int p_l11, p_u11, p_dinv, p_l21, p_u12, p_d, ldd, n_flev, n_blev;
  const int *u11ptr, *flev_ptr, *flev, *blev_ptr, *blev;
  const int *hop_ptr, *hop_piv;     // head program (see LUSymbolic)
  const int4* hop;
  const int2* hterm;
  int n_hlev;
  const int *perm, *iperm, *lptr, *lidx, *uptr, *uidx, *lrptr, *lridx, *ucptr, *ucidx, *jp_ptr, *jt_ptr,
      *jpos, *jrc, *uoff, *lrhead, *lrhoff, *u12off, *lrhk, *srow;
  int n_srow;
  const int2 *jt_word, *jt_slot, *reac;
  const int* sc_ptr;
  const uint32_t* sc_ent;
  const int4* jdesc;     // per Jacobian entry {t0, t1, jrc, row << 16 | col}
  const int* jlong;      // entries with more than kJLong terms
  int n_jlong;
  // coupled temperature (therm = 1, see sm_net_set_thermal): row t_idx of
  // every state vector holds T; k' of the T-dependent reactions is
  // recomputed from it (into kslot) before every right-hand side
  int therm, t_idx, n_cool, bpad;
  double th_heat, th_lam, th_Td, th_zeta;
  const RatePar* rpar;
  const double *th_L, *th_E, *th_dn;   // [n] cooling coefficients, [n] excitation temperatures, [n_r] net particle change
  const int* th_cool;                  // [n_cool] the coolant species
  const double *c_nH, *c_Av, *c_chi;   // [ld] cell conditions, cell order
  double *bz, *bgv, *bs;               // per cell (cell order): z, gamma_J v ([ld][bpad]) and the Schur complement ([ld])
};

__device__ __forceinline__ double& V(double* a, const Dev& d, int s, int64_t c) {
  return a[(int64_t)s * d.ld + c];
}
__device__ __forceinline__ double* Yh(const Dev& d, int i) { return d.Y + (int64_t)i * d.n * d.ld; }

// Weights of the polynomial through (T[i], .), i < m, evaluated at t.
__device__ void lagrange(const double* T, int m, double t, double* wts) {
  for (int i = 0; i < m; ++i) {
    double num = 1.0, den = 1.0;
    for (int j = 0; j < m; ++j)
      if (j != i) {
        num *= t - T[j];
        den *= T[i] - T[j];
      }
    wts[i] = num / den;
  }
}

// alpha_i = h l_i'(tau_0) on nodes tau_0 = tnew, tau_i = T[i-1] (i = 1..q).
__device__ void bdf_alphas(double tnew, const double* T, int q, double h, double* al) {
  double tau[QMAX + 1];
  tau[0] = tnew;
  for (int i = 1; i <= q; ++i) tau[i] = T[i - 1];
  double s = 0.0;
  for (int i = 1; i <= q; ++i) s += 1.0 / (tau[0] - tau[i]);
  al[0] = h * s;
  for (int i = 1; i <= q; ++i) {
    double num = 1.0, den = 1.0;
    for (int m = 1; m <= q; ++m)
      if (m != i) num *= tau[0] - tau[m];
    for (int m = 0; m <= q; ++m)
      if (m != i) den *= tau[i] - tau[m];
    al[i] = h * num / den;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// init: copy y0 into the history, validate inputs; then (after f0 = f(y0))
// pick h0 = min(0.01 / |f0|_wrms, t_end).
// ---------------------------------------------------------------------------
__global__ void init_copy_kernel(Dev d, const double* __restrict__ yin, int64_t ldu,
                                 const double* __restrict__ k, int64_t ldk) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  bool ok = true;
  double* Y0 = Yh(d, 0);
  for (int s = 0; s < d.n; ++s) {
    const double v = yin[(int64_t)s * ldu + c];
    V(Y0, d, s, c) = v;
    ok = ok && isfinite(v);
  }
  if (k) {
    for (int j = 0; j < d.n_r; ++j) {
      const double kv = k[(int64_t)j * ldk + c];
      ok = ok && isfinite(kv);
      if (d.kslot) d.kslot[(int64_t)j * d.ld + c] = kv;
    }
  }
  if (d.therm) {
    const int64_t oc = c;
    ok = ok && V(Y0, d, d.t_idx, c) > 0.0 && isfinite(d.c_nH[oc]) && d.c_nH[oc] > 0.0 && isfinite(d.c_Av[oc]) &&
         isfinite(d.c_chi[oc]);
  }
  d.slot_cell[c] = (int)c;
  d.status[c] = ok ? SM_CELL_RUNNING : SM_CELL_NAN;
  d.flags[c] = ok ? F_NEWTON : 0;  // F_NEWTON selects the cells for f0
  d.t[c] = 0.0;
  d.steps[c] = d.rejects[c] = d.conv_fails[c] = d.newton_iters[c] = d.jac_evals[c] = 0;
  d.q[c] = 1;
  d.h[c] = 0.0;
}

// Copies the step history of cell c into checkpoint slot kk.
__device__ void store_checkpoint(const Dev& d, int64_t c, int kk) {
  const int nh = d.nh[c];
  const int64_t vs = (int64_t)d.n * d.ld;
  double* dst = d.ck_Y + (int64_t)kk * (QMAX + 1) * vs;
  for (int i = 0; i < nh; ++i) {
    for (int s = 0; s < d.n; ++s) dst[i * vs + (int64_t)s * d.ld + c] = Yh(d, i)[(int64_t)s * d.ld + c];
    d.ck_t[((int64_t)kk * (QMAX + 1) + i) * d.ld + c] = d.tn[(int64_t)i * d.ld + c];
  }
  d.ck_nh[(int64_t)kk * d.ld + c] = nh;
}

__global__ void init_finish_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) {
    d.counters[kCAct] = (int)d.C;
    d.counters[kCHoles] = d.counters[kCRun] = d.counters[kCLive] = 0;
  }
  if (c >= d.C) return;
  if (d.status[c] != SM_CELL_RUNNING) {
    d.flags[c] = 0;
    return;
  }
  const double* Y0 = Yh(d, 0);
  double acc = 0.0;
  for (int s = 0; s < d.n; ++s) {
    const double y0 = Y0[(int64_t)s * d.ld + c];
    const double v = d.f0[(int64_t)s * d.ld + c] / (d.rtol * fabs(y0) + d.atol);
    acc += v * v;
  }
  const double nrm = sqrt(acc / d.n);
  d.h[c] = fmin(0.01 / fmax(nrm, 1e-300), d.t_end);
  d.t[c] = 0.0;
  d.q[c] = 1;
  d.nh[c] = 1;
  d.tn[c] = 0.0;
  d.n_at_q[c] = 0;
  d.j_age[c] = 0;
  d.flags[c] = F_NEED_J;
  d.gam_J[c] = 1.0;
  d.crate[c] = 1.0;
  d.crej[c] = d.ccf[c] = 0;
  if (d.record) store_checkpoint(d, c, 0);
}

// ---------------------------------------------------------------------------
// predict
// ---------------------------------------------------------------------------
// Predict and finish work on 32 cells per CTA with kCoopWarps warps: every
// warp derives a cell's step scalars from the same inputs (identical
// results), warp 0 alone writes them back, and the species loops are split
// over the warps (lane = cell, so every row access is a coalesced 256-byte
// line).  A thread per cell over all species left too few warps to hide
// the memory latency when few cells run.
constexpr int kCoopWarps = 8;

__global__ void __launch_bounds__(32 * kCoopWarps) predict_kernel(Dev d) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const bool live = c < d.C && !(d.compact && c >= d.counters[kCAct]);
  int fl = 0, q = 1, nh = 1, state = 0;   // state: 0 idle, 1 max steps, 2 step too small, 3 attempt
  double h = 0.0, gamma = 0.0;
  bool fin = false, refresh = false;
  double T[QMAX + 1], wts[QMAX + 1], al[QMAX + 1];
  if (live) {
    fl = d.flags[c] & ~(F_CONV | F_FAILED | F_REFRESH | F_FINAL | F_NEWTON | F_ATTEMPT);
    if (d.status[c] == SM_CELL_RUNNING) {
      if (d.steps[c] >= d.max_steps) {
        state = 1;
      } else {
        const double t = d.t[c];
        h = d.h[c];
        q = d.q[c];
        nh = d.nh[c];
        fin = t + h >= d.t_end;
        if (fin) h = d.t_end - t;
        const double tnew = fin ? d.t_end : t + h;
        if (tnew == t || !(h > 0.0)) {
          state = 2;
        } else {
          state = 3;
          for (int i = 0; i < nh; ++i) T[i] = d.tn[(int64_t)i * d.ld + c];
          if (nh > 1) lagrange(T, q + 1, tnew, wts);
          bdf_alphas(tnew, T, q, h, al);
          gamma = h / al[0];
          refresh = (fl & F_NEED_J) || d.j_age[c] >= d.j_age_max || fabs(gamma / d.gam_J[c] - 1.0) > d.gamma_tol;
        }
      }
    }
  }
  __syncthreads();   // every warp has read the cell before warp 0 rewrites it
  if (wi == 0 && live) {
    if (d.status[c] == SM_CELL_RUNNING) atomicAdd(&d.counters[1], 1);
    if (state == 1) d.status[c] = SM_CELL_MAXSTEPS;
    if (state == 2) d.status[c] = SM_CELL_HMIN;
    if (state == 3) {
      d.h[c] = h;
      d.gam[c] = gamma;
      for (int i = 0; i <= q; ++i) d.alpha[(int64_t)i * d.ld + c] = al[i];
      fl |= F_NEWTON | F_ATTEMPT | (fin ? F_FINAL : 0) | (refresh ? F_REFRESH : 0);
      d.m_it[c] = 0;
      d.dprev[c] = 0.0;
      if (refresh) d.list[atomicAdd(&d.counters[0], 1)] = (int)c;
    }
    d.flags[c] = fl;
  }
  if (state != 3) return;
  // kPU species at a time with the history loops unrolled, so that each
  // thread has kPU * (q + 1) loads in flight
  constexpr int kPU = 4;
  const bool euler = nh == 1;
  for (int s0 = wi * kPU; s0 < d.n; s0 += kCoopWarps * kPU) {
    double Yv[kPU][QMAX + 1], fv[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int64_t o = (int64_t)(s0 + u) * d.ld + c;
      const bool in = s0 + u < d.n;
#pragma unroll
      for (int i = 0; i <= QMAX; ++i) Yv[u][i] = (in && i <= q && i < nh) ? Yh(d, i)[o] : 0.0;
      fv[u] = (in && euler) ? d.f0[o] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      if (s0 + u >= d.n) break;
      const int64_t o = (int64_t)(s0 + u) * d.ld + c;
      const double y0 = Yv[u][0];
      double yp = euler ? y0 + h * fv[u] : 0.0, ps = 0.0;
#pragma unroll
      for (int i = 0; i <= QMAX; ++i) {
        if (!euler && i <= q) yp += wts[i] * Yv[u][i];
        if (i >= 1 && i <= q) ps += al[i] * Yv[u][i - 1];
      }
      d.ypred[o] = yp;
      d.y[o] = yp;
      d.psi[o] = ps;
      d.w[o] = 1.0 / (d.rtol * fabs(y0) + d.atol);
    }
  }
}

// ---------------------------------------------------------------------------
// refresh: J, M = I - gamma J and its LU without pivoting (elimination order
// = minimum degree), worked in a dense matrix (one per refresh CTA, or one
// per cell in recording states) and written out as the cell's packed
// factors.  One CTA per cell on the compacted refresh list (grid-stride).
// The first kJPre term words of the Jacobian entries a thread holds are
// loaded before any is used.  With M = [A11 A12; A21 A22]
// split at the first `head` pivots (sparse) and the >= 90 % dense trailing
// block:
//  A  dR_j/dx for both reactant slots of every reaction is formed once in
//     shared memory (FP64) and M is gathered at the Jacobian pattern;
//  B  the head's factors (L11, U11, pivots, L21, U12) are computed in
//     shared memory in the packed layout by the head program: pivots in
//     dependency levels, every entry of a level at once (left-looking);
//  S  the head's Schur complement A22 -= L21 U12 (sparse: about 1 % of a
//     dense product) is applied panel by panel from shared memory: U12's
//     panel columns as a dense tile, L21 in compact row order, one warp per
//     tail row (lanes = columns), rows dealt longest first;
//  C  the trailing block is factorised right-looking by panels of kNB
//     columns; panel and U12 block live in shared memory, the trailing
//     update is a register-tiled GEMM.
// Inverse pivots replace the diagonal.
// ---------------------------------------------------------------------------
// Optional per-phase cycle counters of the refresh kernel (build option
// SM_PHASE_CLOCKS, see build.py): thread 0 of every CTA adds the clock64()
// cycles between consecutive phase marks (taken right after the CTA-wide
// barriers that end the phases) to g_phase_cycles[phase]; slot 15 counts the
// refreshed cells.  Compiled out otherwise.
constexpr int kPhaseSlots = 16;
#ifdef SM_PHASE_CLOCKS
__device__ unsigned long long g_phase_cycles[kPhaseSlots];
#define PHASE_START() long long ph_t = clock64()
#define PHASE_MARK(k)                                                                         \
  do {                                                                                        \
    if (threadIdx.x == 0) {                                                                   \
      const long long ph_now = clock64();                                                     \
      atomicAdd(&g_phase_cycles[(k)], (unsigned long long)(ph_now - ph_t));                   \
      ph_t = ph_now;                                                                          \
    }                                                                                         \
  } while (0)
#else
#define PHASE_START() do {} while (0)
#define PHASE_MARK(k) do {} while (0)
#endif

constexpr int kRefreshThreads = 256;
constexpr int kNB = 32;
constexpr int kTM = 4, kTN = 4;
constexpr int kBM = 16 * kTM, kBN = 16 * kTN;
constexpr int kPS = 3;                    // panels per pass of the head Schur complement (phase S)

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Shared-memory plan (bytes) shared by host and device.
struct RefreshPlan {
  int pitch;          // column pitch of the panel buffer
  int upitch;         // row pitch of the U block buffer
  int n_panels;       // 32-wide panels of the trailing block
  int hv_off;         // byte offset of the packed head factors H in phases B / S
  int ix_off;         // byte offset of the Schur pass's staged indices (after H)
  int n_l21, n_u12;   // L21 / U12 entries
  bool head_smem;     // phase B runs the head program in shared memory (else pivot by pivot)
  size_t bytes;
};

template <class T> struct Vec4;
template <> struct Vec4<float> {
  float a[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
  }
};
template <> struct Vec4<double> {
  double a[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 v0 = *reinterpret_cast<const double2*>(p);
    const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
    a[0] = v0.x; a[1] = v0.y; a[2] = v1.x; a[3] = v1.y;
  }
};

template <class T> __device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Tensor-core trailing update C -= L U with K = kNB for the FP32 factors
// (precision mode TF32): L (r x kNB) column-major in shared memory (element
// (i, k) at L[k * pl + i]), U (kNB x r) row-major (element (k, j) at U[k * pu
// + j]), C (r x r) in global memory with row stride ldc.  One warp per 32 x 32
// tile of C: 2 x 4 mma.m16n8k8 TF32 fragments, each operand split into TF32
// high and low parts (three products per pair: FP32-level accuracy), FP32
// accumulators loaded from and stored back to C.  Fragment layouts of m16n8k8 .tf32 (g = lane / 4,
// t = lane % 4): A {(g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4)}, B {(t, g),
// (t + 4, g)}, C {(g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1)}.  Rows
// and columns of a tile past r read whatever follows in shared memory and are
// neither loaded from nor stored to C.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ void tf32_trailing_update(float* C, int ldc, int r, const float* L, int pl, const float* U, int pu,
                                     int warp, int nwarps, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int nb = (r + 31) / 32;
  for (int tile = warp; tile < nb * nb; tile += nwarps) {
    const int i0 = (tile / nb) * 32, j0 = (tile % nb) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = i0 + mt * 16 + g + (e >> 1) * 8, col = j0 + nt * 8 + 2 * t + (e & 1);
          acc[mt][nt][e] = (row < r && col < r) ? C[(int64_t)row * ldc + col] : 0.f;
        }
#pragma unroll
    for (int k0 = 0; k0 < kNB; k0 += 8) {
      // each operand x = hi + lo with hi = tf32(x), lo = tf32(x - hi); the
      // products hi*hi + hi*lo + lo*hi keep FP32-level accuracy
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
      const float* l0 = L + (k0 + t) * pl + i0 + g;
      const float* l4 = l0 + 4 * pl;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const float v[4] = {-l0[mt * 16], -l0[mt * 16 + 8], -l4[mt * 16], -l4[mt * 16 + 8]};
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(v[e], ah[mt][e], al[mt][e]);
      }
      const float* u0 = U + (k0 + t) * pu + j0 + g;
      const float* u4 = u0 + 4 * pu;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        split_tf32(u0[nt * 8], bh[nt][0], bl[nt][0]);
        split_tf32(u4[nt * 8], bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_tf32(acc[mt][nt], al[mt], bh[nt]);
          mma_tf32(acc[mt][nt], ah[mt], bl[nt]);
          mma_tf32(acc[mt][nt], ah[mt], bh[nt]);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = i0 + mt * 16 + g + (e >> 1) * 8, col = j0 + nt * 8 + 2 * t + (e & 1);
          if (row < r && col < r) C[(int64_t)row * ldc + col] = acc[mt][nt][e];
        }
  }
}

template <class T>
__global__ void __launch_bounds__(kRefreshThreads, 2) refresh_kernel(Dev d, const double* __restrict__ k,
                                                                 int64_t ldk, RefreshPlan plan) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int n = d.n, n_r = d.n_r, ldm = d.ldm, h = d.head, nt = n - h, pitch = plan.pitch;
  const int np1 = plan.n_panels + 1;
  T* Pt = reinterpret_cast<T*>(smem_raw);           // panel, column-major, kNB columns
  T* U = Pt + (size_t)kNB * pitch;                  // U12 block, kNB rows, pitch upitch
  const int upitch = plan.upitch;
  double* dR = reinterpret_cast<double*>(smem_raw); // phase A: [n_r][2]
  float* wsf;
  float* wif;
  T* Hv = reinterpret_cast<T*>(smem_raw + plan.hv_off);  // phases B / S: packed head factors
  // phase S indices, staged after H: per L21 entry its head column, per U12
  // entry its tail column, per head row and panel the start of its U12 entries
  unsigned short* sx_l21 = reinterpret_cast<unsigned short*>(smem_raw + plan.ix_off);
  unsigned short* sx_u12 = sx_l21 + plan.n_l21;
  int* sx_off = reinterpret_cast<int*>(smem_raw + plan.ix_off + 4 * ((plan.n_l21 + plan.n_u12 + 1) / 2));
  double* coef = dR + 2 * n_r;                      // (double)(int8_t)i, J coefficients
  wsf = reinterpret_cast<float*>(coef + 256);
  wif = wsf + n;
  const int count = d.counters[0];
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t c = d.list[e];
    T* A = static_cast<T*>(d.lu) + (d.lu_cta ? (int64_t)blockIdx.x : c) * d.lu_stride;
    T* P = d.lup ? static_cast<T*>(d.lup) + (int64_t)d.slot_cell[c] * d.lup_stride : nullptr;
    T* D = P ? P + d.p_d : nullptr;   // packed tail block, column-major
    PHASE_START();
    const double gamma = d.gam[c];
    // zero the dense trailing block and the head's pattern entries
    for (int r = warp; r < nt; r += nwarps) {
      T* row = A + (int64_t)(h + r) * ldm + h;
      for (int q = lane; q < nt; q += 32) row[q] = T(0);
    }
    for (int kp = warp; kp < h; kp += nwarps) {
      for (int p = __ldg(d.lptr + kp) + lane; p < __ldg(d.lptr + kp + 1); p += 32)
        A[(int64_t)__ldg(d.lidx + p) * ldm + kp] = T(0);
      for (int p = __ldg(d.uptr + kp) + lane; p < __ldg(d.uptr + kp + 1); p += 32)
        A[(int64_t)kp * ldm + __ldg(d.uidx + p)] = T(0);
      if (lane == 0) A[(int64_t)kp * ldm + kp] = T(0);
    }
    // ---- phase A
    for (int i = tid; i < 256; i += nthr) coef[i] = (double)(int8_t)i;
    for (int j = tid; j < n_r; j += nthr) {
      const int2 rc = __ldg(d.reac + j);
      const double kv = k[(int64_t)j * ldk + c];
      dR[2 * j] = rc.y >= 0 ? kv * d.ypred[(int64_t)rc.y * d.ld + c] : kv;
      dR[2 * j + 1] = rc.y >= 0 ? kv * d.ypred[(int64_t)rc.x * d.ld + c] : 0.0;
    }
    if (d.mixed)
      for (int s = tid; s < n; s += nthr) {
        const double wv = V(d.w, d, s, c);
        V(d.wf, d, s, c) = wv;
        wsf[s] = (float)wv;
        wif[s] = (float)(1.0 / wv);
      }
    __syncthreads();
    PHASE_MARK(0);   // zero the working matrix, dR/dx, weights
    // M_ij = delta_ij - gamma sum_terms coef dR, stored in elimination order
    // (W M W^-1 with this step's error weights, scaled in FP32, when mixed)
    auto store_m = [&](const int4 ds, double acc) {
      const int pi = ds.z >> 16, pj = ds.z & 0xFFFF;
      const double m = fma(-gamma, acc, pi == pj ? 1.0 : 0.0);
      T* dst = A + (int64_t)pi * ldm + pj;
      if (d.mixed) *dst = T((float)m * (wsf[ds.w >> 16] * wif[ds.w & 0xFFFF]));
      else *dst = T(m);
    };
    auto term = [&](double acc, int t) {
      const int2 w = __ldg(d.jt_slot + t);
      return fma(coef[(uint32_t)w.x >> 24], dR[2 * (w.x & 0xFFFFFF) + w.y], acc);
    };
    // entries with more than kJLong terms (the hub species'): a warp each
    for (int q = warp; q < d.n_jlong; q += nwarps) {
      const int4 ds = __ldg(d.jdesc + __ldg(d.jlong + q));
      double acc = 0.0;
      for (int t = ds.x + lane; t < ds.y; t += 32) acc = term(acc, t);
      acc = warp_sum(acc);
      if (lane == 0) store_m(ds, acc);
    }
    // the others: a thread each, two entries at a time; the first kJPre term
    // words of both entries are loaded before any is used, so that their
    // loads overlap (most entries have at most kJPre terms)
    constexpr int kJPre = 4;
    for (int p = tid; p < d.nnz_j; p += 2 * nthr) {
      const bool hb = p + nthr < d.nnz_j;
      const int4 da = __ldg(d.jdesc + p);
      const int4 db = hb ? __ldg(d.jdesc + p + nthr) : make_int4(0, 0, 0, 0);
      const bool la = da.y - da.x <= kJLong, lb = hb && db.y - db.x <= kJLong;
      double aa = 0.0, ab = 0.0;
      const int na = la ? da.y - da.x : 0, nb = lb ? db.y - db.x : 0;
      int2 wa[kJPre], wb[kJPre];
#pragma unroll
      for (int u = 0; u < kJPre; ++u) {
        wa[u] = u < na ? __ldg(d.jt_slot + da.x + u) : make_int2(0, 0);
        wb[u] = u < nb ? __ldg(d.jt_slot + db.x + u) : make_int2(0, 0);
      }
#pragma unroll
      for (int u = 0; u < kJPre; ++u) {
        if (u < na) aa = fma(coef[(uint32_t)wa[u].x >> 24], dR[2 * (wa[u].x & 0xFFFFFF) + wa[u].y], aa);
        if (u < nb) ab = fma(coef[(uint32_t)wb[u].x >> 24], dR[2 * (wb[u].x & 0xFFFFFF) + wb[u].y], ab);
      }
      for (int u = kJPre; u < max(na, nb); ++u) {
        if (u < na) aa = term(aa, da.x + u);
        if (u < nb) ab = term(ab, db.x + u);
      }
      if (la) store_m(da, aa);
      if (lb) store_m(db, ab);
    }
    __syncthreads();
    PHASE_MARK(1);   // Jacobian gather, M = I - gamma J
    // ---- phase B: sparse head.  The head program (see LUSymbolic) computes
    // every head factor entry in the packed layout, in shared memory: level
    // by level, first the level's pivots (stored inverted), then the U rows
    // and L columns of those pivots, each entry a thread's
    //   a - sum of its product terms (times the inverse pivot for L).
    if (plan.head_smem) {
      for (int e = tid; e < plan.n_l21; e += nthr) sx_l21[e] = (unsigned short)__ldg(d.lrhk + e);
      for (int kr = warp; kr < h; kr += nwarps) {
        const int base = __ldg(d.uoff + kr * np1), o12 = __ldg(d.u12off + kr), cnt = __ldg(d.u12off + kr + 1) - o12;
        for (int q = lane; q < cnt; q += 32) sx_u12[o12 + q] = (unsigned short)(__ldg(d.uidx + base + q) - h);
        for (int b = lane; b < np1; b += 32) sx_off[kr * np1 + b] = o12 + __ldg(d.uoff + kr * np1 + b) - base;
      }
      for (int l = 0; l < d.n_hlev; ++l) {
        for (int part = 0; part < 2; ++part) {
          const int o1 = __ldg(d.hop_ptr + 2 * l + part + 1);
          for (int o = __ldg(d.hop_ptr + 2 * l + part) + tid; o < o1; o += nthr) {
            const int4 op = __ldg(d.hop + o);
            T v = A[op.y];
            for (int t = op.z; t < op.w; ++t) {
              const int2 tm = __ldg(d.hterm + t);
              v -= Hv[tm.x] * Hv[tm.y];
            }
            if (part == 0) {
              v = T(1) / v;
            } else {
              const int pv = __ldg(d.hop_piv + o);
              if (pv >= 0) v *= Hv[pv];
            }
            Hv[op.x] = v;
          }
          __syncthreads();
        }
      }
      PHASE_MARK(2);   // head program
      // ---- phase S: A22 -= L21 U12, one 32-column panel at a time.  U12's
      // panel columns are expanded into a dense h x 32 tile (in front of H);
      // each tail row with head entries is one warp's: lanes are the panel's
      // columns, the row's L21 values come from H.
      T* Ut = reinterpret_cast<T*>(smem_raw);
      for (int q0 = 0; q0 < plan.n_panels; q0 += kPS) {
        // kPS panels per pass: tile [j][k][32] for panel q0 + j
        const int np = min(kPS, plan.n_panels - q0);
        for (int e = tid; e < np * h * kNB; e += nthr) Ut[e] = T(0);
        __syncthreads();
        for (int kr = warp; kr < h; kr += nwarps) {
          // row kr's packed U12 entries of panels q0 .. q0 + np - 1
          const int e1 = sx_off[kr * np1 + q0 + np];
          for (int e = sx_off[kr * np1 + q0] + lane; e < e1; e += 32) {
            const int ct = (int)sx_u12[e] - kNB * q0;
            Ut[((ct / kNB) * h + kr) * kNB + (ct % kNB)] = Hv[d.p_u12 + e];
          }
        }
        __syncthreads();
        // kSB rows per warp at a time (rows t = t0 + u * nwarps + warp, so the
        // longest rows stay spread over the warps): their loads of A go out
        // together before any row's sums are formed
        constexpr int kSB = 8;
        for (int t0 = 0; t0 < d.n_srow; t0 += kSB * nwarps) {
          T cur[kSB][kPS];
          int ir[kSB], ro[kSB], rc[kSB];
#pragma unroll
          for (int u = 0; u < kSB; ++u) {
            const int t = t0 + u * nwarps + warp;
            ir[u] = t < d.n_srow ? __ldg(d.srow + t) : -1;
          }
#pragma unroll
          for (int u = 0; u < kSB; ++u) {
            const T* Ai = A + (int64_t)(h + max(ir[u], 0)) * ldm + h + kNB * q0 + lane;
#pragma unroll
            for (int j = 0; j < kPS; ++j)
              cur[u][j] = (ir[u] >= 0 && j < np && h + kNB * (q0 + j) + lane < n) ? Ai[kNB * j] : T(0);
            ro[u] = ir[u] >= 0 ? __ldg(d.lrhoff + ir[u]) : 0;
            rc[u] = ir[u] >= 0 ? __ldg(d.lrhead + ir[u]) : 0;
          }
#pragma unroll
          for (int u = 0; u < kSB; ++u) {
            if (ir[u] < 0) continue;
            const int o = ro[u], cnt = rc[u];
            T acc[kPS];
#pragma unroll
            for (int j = 0; j < kPS; ++j) acc[j] = T(0);
            for (int e = 0; e < cnt; ++e) {
              const T l = Hv[d.p_l21 + o + e];
              const T* ut = Ut + (int)sx_l21[o + e] * kNB + lane;
#pragma unroll
              for (int j = 0; j < kPS; ++j)
                if (j < np) acc[j] += l * ut[j * h * kNB];
            }
            T* Ai = A + (int64_t)(h + ir[u]) * ldm + h + kNB * q0 + lane;
#pragma unroll
            for (int j = 0; j < kPS; ++j)
              if (j < np && h + kNB * (q0 + j) + lane < n) Ai[kNB * j] = cur[u][j] - acc[j];
          }
        }
        __syncthreads();
      }
    } else {
      // pivot by pivot, Schur complement applied immediately
      for (int kp = 0; kp < h; ++kp) {
        const T inv = T(1) / A[(int64_t)kp * ldm + kp];
        const int l0 = __ldg(d.lptr + kp), l1 = __ldg(d.lptr + kp + 1);
        for (int p = l0 + tid; p < l1; p += nthr) A[(int64_t)__ldg(d.lidx + p) * ldm + kp] *= inv;
        __syncthreads();
        if (tid == 0) A[(int64_t)kp * ldm + kp] = inv;
        const int u0 = __ldg(d.uptr + kp), nU = __ldg(d.uptr + kp + 1) - u0;
        const T* Ak = A + (int64_t)kp * ldm;
        for (int a = l0 + warp; a < l1; a += nwarps) {
          T* Ai = A + (int64_t)__ldg(d.lidx + a) * ldm;
          const T l = Ai[kp];
          for (int b = lane; b < nU; b += 32) {
            const int j = __ldg(d.uidx + u0 + b);
            Ai[j] -= l * Ak[j];
          }
        }
        __syncthreads();
      }
    }
    PHASE_MARK(3);   // head Schur complement (or the pivot-by-pivot head)
    // the head's factors are final.  Packed output: copy them out (from H, or
    // from the dense matrix after the pivot-by-pivot head); dense output: put
    // H's values back at their dense positions
    if (plan.head_smem) {
      if (P) {
        for (int i = tid; i < d.p_d; i += nthr) P[i] = Hv[i];
      } else {
        const int o1 = __ldg(d.hop_ptr + 2 * d.n_hlev);
        for (int o = tid; o < o1; o += nthr) {
          const int4 op = __ldg(d.hop + o);
          A[op.y] = Hv[op.x];
        }
      }
      __syncthreads();
    } else if (P) {
      __syncthreads();
      for (int i = warp; i < h; i += nwarps) {
        const T* Ai = A + (int64_t)i * ldm;
        for (int q = __ldg(d.lrptr + i) + lane; q < __ldg(d.lrptr + i + 1); q += 32)
          P[d.p_l11 + q] = Ai[__ldg(d.lridx + q)];
        const int u0 = __ldg(d.uptr + i), o11 = __ldg(d.u11ptr + i), n11 = __ldg(d.u11ptr + i + 1) - o11;
        for (int q = lane; q < n11; q += 32) P[d.p_u11 + o11 + q] = Ai[__ldg(d.uidx + u0 + q)];
        const int q12 = __ldg(d.uoff + i * np1), o12 = __ldg(d.u12off + i), n12 = __ldg(d.u12off + i + 1) - o12;
        for (int q = lane; q < n12; q += 32) P[d.p_u12 + o12 + q] = Ai[__ldg(d.uidx + q12 + q)];
        if (lane == 0) P[d.p_dinv + i] = Ai[i];
      }
      for (int i = h + warp; i < n; i += nwarps) {
        const T* Ai = A + (int64_t)i * ldm;
        const int p0 = __ldg(d.lrptr + i), o = __ldg(d.lrhoff + i - h), cnt = __ldg(d.lrhead + i - h);
        for (int q = lane; q < cnt; q += 32) P[d.p_l21 + o + q] = Ai[__ldg(d.lridx + p0 + q)];
      }
    }
    PHASE_MARK(4);   // packed head factors
    // ---- phase C: dense trailing block, blocked right-looking LU
    for (int pb = 0; pb * kNB < nt; ++pb) {
      const int p0 = h + pb * kNB;
      const int w = min(kNB, n - p0), m = n - p0, r = m - w;
#pragma unroll 4
      for (int a = warp; a < m; a += nwarps)
        if (lane < w) Pt[lane * pitch + a] = A[(int64_t)(p0 + a) * ldm + p0 + lane];
      for (int a = m + tid; a < pitch; a += nthr)
        for (int b = 0; b < w; ++b) Pt[b * pitch + a] = T(0);
      __syncthreads();
      PHASE_MARK(5);   // panel loads
      if (sizeof(T) == 4 && w == kNB) {
        // full FP32 panel.  (1) warp 0 factors the kNB x kNB diagonal block in
        // registers (lane = row, pivot rows broadcast by shuffles); (2) every
        // row below solves l U11 = a on its own (thread per row, U11 read as
        // shared-memory broadcasts), with no barrier between columns
        if (warp == 0) {
          T rv[kNB];
#pragma unroll
          for (int b = 0; b < kNB; ++b) rv[b] = Pt[b * pitch + lane];
#pragma unroll
          for (int kk = 0; kk < kNB; ++kk) {
            const T inv = T(1) / shfl(rv[kk], kk);
            const T l = rv[kk] * inv;
            const bool below = lane > kk;
            if (below) rv[kk] = l;
#pragma unroll
            for (int b = 0; b < kNB; ++b)
              if (b > kk) {
                const T pb = shfl(rv[b], kk);
                if (below) rv[b] -= l * pb;
              }
          }
#pragma unroll
          for (int b = 0; b < kNB; ++b) Pt[b * pitch + lane] = b == lane ? T(1) / rv[b] : rv[b];
        }
        __syncthreads();
        for (int a = kNB + tid; a < m; a += nthr) {
          T rv[kNB];
#pragma unroll
          for (int b = 0; b < kNB; ++b) rv[b] = Pt[b * pitch + a];
#pragma unroll
          for (int kk = 0; kk < kNB; ++kk) {
            const T l = rv[kk] * Pt[kk * pitch + kk];   // inverse pivot
            rv[kk] = l;
#pragma unroll
            for (int b = 0; b < kNB; ++b)
              if (b > kk) rv[b] -= l * Pt[b * pitch + kk];
          }
#pragma unroll
          for (int b = 0; b < kNB; ++b) Pt[b * pitch + a] = rv[b];
        }
        __syncthreads();
      } else {
        for (int kk = 0; kk < w; ++kk) {
          // row kk is final after the previous barrier; the inverse pivot is
          // stored after this step's barrier (no later step reads it)
          const T inv = T(1) / Pt[kk * pitch + kk];
          for (int a = kk + 1 + tid; a < m; a += nthr) {
            const T l = Pt[kk * pitch + a] * inv;
            Pt[kk * pitch + a] = l;
            for (int b = kk + 1; b < w; ++b) Pt[b * pitch + a] -= l * Pt[b * pitch + kk];
          }
          __syncthreads();
          if (tid == 0) Pt[kk * pitch + kk] = inv;
        }
        __syncthreads();
      }
      PHASE_MARK(6);   // panel LU
      if (D) {
        // the panel's columns (diagonal block and L below it) are final
        for (int b = warp; b < w; b += nwarps)
          for (int a = lane; a < m; a += 32) D[(int64_t)(p0 - h + b) * d.ldd + (p0 - h + a)] = Pt[b * pitch + a];
      } else {
        for (int a = warp; a < m; a += nwarps)
          if (lane < w) A[(int64_t)(p0 + a) * ldm + p0 + lane] = Pt[lane * pitch + a];
      }
      if (r > 0) {
        const int rp = round_up(r, 4);
        for (int a = warp; a < w; a += nwarps)
          for (int b = lane; b < rp; b += 32)
            U[a * upitch + b] = b < r ? A[(int64_t)(p0 + a) * ldm + p0 + w + b] : T(0);
        __syncthreads();
        PHASE_MARK(7);   // panel stored, U block loaded
        // U12 = L11^-1 A12, one thread per column
        if (w == kNB) {
          for (int b = tid; b < r; b += nthr) {
            T col[kNB];
#pragma unroll
            for (int a = 0; a < kNB; ++a) col[a] = U[a * upitch + b];
#pragma unroll
            for (int kk = 0; kk < kNB; ++kk)
#pragma unroll
              for (int a = kk + 1; a < kNB; ++a) col[a] -= Pt[kk * pitch + a] * col[kk];
#pragma unroll
            for (int a = 0; a < kNB; ++a) U[a * upitch + b] = col[a];
          }
        } else {
          for (int b = tid; b < r; b += nthr)
            for (int kk = 0; kk < w; ++kk) {
              const T u = U[kk * upitch + b];
              for (int a = kk + 1; a < w; ++a) U[a * upitch + b] -= Pt[kk * pitch + a] * u;
            }
        }
        __syncthreads();
        PHASE_MARK(8);   // U block solved
        if (D) {
          // the panel's U rows are final: column b of the block, rows p0..p0+w
          for (int e = tid; e < r * 32; e += nthr) {
            const int b = e >> 5, a = e & 31;
            if (a < w) D[(int64_t)(p0 - h + w + b) * d.ldd + (p0 - h + a)] = U[a * upitch + b];
          }
        } else {
          for (int a = warp; a < w; a += nwarps)
            for (int b = lane; b < r; b += 32) A[(int64_t)(p0 + a) * ldm + p0 + w + b] = U[a * upitch + b];
        }
        // A22 -= L21 U12; L21 column kk is Pt[kk * pitch + w + i]
        bool done = false;
        if constexpr (sizeof(T) == 4) {
          if (d.tf32 && w == kNB) {
            tf32_trailing_update(A + (int64_t)(p0 + w) * ldm + p0 + w, ldm, r, Pt + w, pitch, U, upitch, warp,
                                 nwarps, lane);
            done = true;
          }
        }
        // 64 x 64 tiles of the trailing block in turn, a 4 x 4 sub-tile per
        // thread; the next tile's values of A are loaded while this tile's
        // products are formed
        const int ty = tid / 16, tx = tid % 16;
        const int nbu = (r + kBN - 1) / kBN, ntile = done ? 0 : ((r + kBM - 1) / kBM) * nbu;
        T nxt[kTM][kTN];
        auto load_c = [&](int tt) {
          const int i0 = (tt / nbu) * kBM + ty * kTM, j0 = (tt % nbu) * kBN + tx * kTN;
#pragma unroll
          for (int a = 0; a < kTM; ++a)
#pragma unroll
            for (int b = 0; b < kTN; ++b)
              nxt[a][b] = (i0 + a < r && j0 + b < r) ? A[(int64_t)(p0 + w + i0 + a) * ldm + p0 + w + j0 + b] : T(0);
        };
        if (ntile > 0) load_c(0);
        for (int tt = 0; tt < ntile; ++tt) {
          T acc[kTM][kTN];
#pragma unroll
          for (int a = 0; a < kTM; ++a)
#pragma unroll
            for (int b = 0; b < kTN; ++b) acc[a][b] = nxt[a][b];
          if (tt + 1 < ntile) load_c(tt + 1);
          const int i0 = (tt / nbu) * kBM + ty * kTM, j0 = (tt % nbu) * kBN + tx * kTN;
          if (i0 >= r || j0 >= r) continue;
          const T* lp = Pt + w + i0;
          const T* up = U + j0;
          for (int kk = 0; kk < w; ++kk) {
            Vec4<T> lv, uv;
            lv.load(lp + kk * pitch);
            uv.load(up + kk * upitch);
#pragma unroll
            for (int a = 0; a < kTM; ++a)
#pragma unroll
              for (int b = 0; b < kTN; ++b) acc[a][b] -= lv.a[a] * uv.a[b];
          }
#pragma unroll
          for (int a = 0; a < kTM; ++a)
#pragma unroll
            for (int b = 0; b < kTN; ++b)
              if (i0 + a < r && j0 + b < r)
                A[(int64_t)(p0 + w + i0 + a) * ldm + p0 + w + j0 + b] = acc[a][b];
        }
      }
      __syncthreads();
      PHASE_MARK(9);   // trailing update
    }
    if (tid == 0) {
      d.gam_J[c] = gamma;
      d.j_age[c] = 0;
      d.crate[c] = 1.0;
      d.flags[c] &= ~F_NEED_J;
      d.jac_evals[c] += 1;
    }
    __syncthreads();
#ifdef SM_PHASE_CLOCKS
    if (tid == 0) atomicAdd(&g_phase_cycles[kPhaseSlots - 1], 1ull);
#endif
    PHASE_MARK(10);  // epilogue
  }
}

// ---------------------------------------------------------------------------
// Newton: residual, substitution, update and convergence test (warp per cell)
// ---------------------------------------------------------------------------
constexpr int kSolveWarps = 4;

// sum_{c in [c0, c1)} row[c] * x[c]: scalar ends, 16-byte vector middle.
__device__ __forceinline__ float dense_dot(const float* __restrict__ row, const float* x, int c0, int c1) {
  float s0 = 0.f, s1 = 0.f;
  int c = c0;
  for (; c < c1 && (c & 3); ++c) s0 += row[c] * x[c];
  for (; c + 4 <= c1; c += 4) {
    const float4 a = *reinterpret_cast<const float4*>(row + c);
    const float4 b = *reinterpret_cast<const float4*>(x + c);
    s0 = fmaf(a.x, b.x, s0);
    s1 = fmaf(a.y, b.y, s1);
    s0 = fmaf(a.z, b.z, s0);
    s1 = fmaf(a.w, b.w, s1);
  }
  for (; c < c1; ++c) s0 += row[c] * x[c];
  return s0 + s1;
}
__device__ __forceinline__ double dense_dot(const double* __restrict__ row, const double* x, int c0, int c1) {
  double s0 = 0.0, s1 = 0.0;
  int c = c0;
  for (; c < c1 && (c & 1); ++c) s0 += row[c] * x[c];
  for (; c + 2 <= c1; c += 2) {
    const double2 a = *reinterpret_cast<const double2*>(row + c);
    const double2 b = *reinterpret_cast<const double2*>(x + c);
    s0 = fma(a.x, b.x, s0);
    s1 = fma(a.y, b.y, s1);
  }
  for (; c < c1; ++c) s0 += row[c] * x[c];
  return s0 + s1;
}

// Substitution with the factors of one cell (warp per cell).  Sparse head rows
// run one row at a time with the next row's entries already in flight; the
// dense tail runs in blocks of 32 rows, one row per lane: each lane streams
// its row segment left (forward) or right (backward) of the block, then the
// 32 x 32 diagonal block is resolved with warp shuffles.
template <class T>
__device__ void lu_substitute(const Dev& d, const T* __restrict__ A, T* x, int lane) {
  const int n = d.n, ldm = d.ldm, h = d.head;
  constexpr int EPL = 4;   // head-row entries per lane (rows up to 128 entries)
  // forward, sparse head rows (unit lower triangle)
  {
    T v[EPL];
    int j[EPL];
    auto load_row = [&](int i) {
      const int p0 = __ldg(d.lrptr + i), p1 = __ldg(d.lrptr + i + 1);
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = p0 + lane + 32 * e;
        j[e] = p < p1 ? __ldg(d.lridx + p) : -1;
        v[e] = p < p1 ? A[(int64_t)i * ldm + j[e]] : T(0);
      }
    };
    if (h > 0) load_row(0);
    for (int i = 0; i < h; ++i) {
      T vc[EPL];
      int jc[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e) { vc[e] = v[e]; jc[e] = j[e]; }
      if (i + 1 < h) load_row(i + 1);
      T s = T(0);
#pragma unroll
      for (int e = 0; e < EPL; ++e)
        if (jc[e] >= 0) s += vc[e] * x[jc[e]];
      // rows longer than EPL * 32 entries finish here
      for (int p = __ldg(d.lrptr + i) + lane + 32 * EPL; p < __ldg(d.lrptr + i + 1); p += 32) {
        const int cc = __ldg(d.lridx + p);
        s += A[(int64_t)i * ldm + cc] * x[cc];
      }
      s = warp_sum(s);
      if (lane == 0) x[i] -= s;
      __syncwarp();
    }
  }
  // forward, dense tail in blocks of 32 rows
  for (int r0 = h; r0 < n; r0 += 32) {
    const int i = r0 + lane;
    const bool live = i < n;
    T xi = T(0);
    T lrow[32];
    if (live) {
      const T* Ai = A + (int64_t)i * ldm;
      T s = T(0);
      for (int p = __ldg(d.lrptr + i), p1 = __ldg(d.lrptr + i + 1); p < p1; ++p) {
        const int c = __ldg(d.lridx + p);
        if (c >= h) break;
        s += Ai[c] * x[c];
      }
      s += dense_dot(Ai, x, h, r0);
      xi = x[i] - s;
#pragma unroll
      for (int k = 0; k < 32; ++k) lrow[k] = (k < lane && r0 + k < n) ? Ai[r0 + k] : T(0);
    } else {
#pragma unroll
      for (int k = 0; k < 32; ++k) lrow[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const T xk = __shfl_sync(0xffffffffu, xi, k);
      if (lane > k) xi -= lrow[k] * xk;
    }
    if (live) x[i] = xi;
    __syncwarp();
  }
  // backward, dense tail from the last block up
  const int nb = (n - h + 31) / 32;
  for (int b = nb - 1; b >= 0; --b) {
    const int r0 = h + 32 * b, r1 = min(r0 + 32, n);
    const int i = r0 + lane;
    const bool live = i < n;
    T xi = T(0);
    T urow[32];
    if (live) {
      const T* Ai = A + (int64_t)i * ldm;
      xi = x[i] - dense_dot(Ai, x, r1, n);
#pragma unroll
      for (int k = 0; k < 32; ++k) urow[k] = (k >= lane && r0 + k < r1) ? Ai[r0 + k] : T(0);
    } else {
#pragma unroll
      for (int k = 0; k < 32; ++k) urow[k] = T(0);
    }
#pragma unroll
    for (int k = 31; k >= 0; --k) {
      if (lane == k) xi *= urow[k];  // inverse pivot on the diagonal
      const T xk = __shfl_sync(0xffffffffu, xi, k);
      if (lane < k) xi -= urow[k] * xk;
    }
    if (live) x[i] = xi;
    __syncwarp();
  }
  // backward, sparse head rows
  {
    T v[EPL];
    int j[EPL];
    auto load_row = [&](int i) {
      const int p0 = __ldg(d.uptr + i), p1 = __ldg(d.uptr + i + 1);
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = p0 + lane + 32 * e;
        j[e] = p < p1 ? __ldg(d.uidx + p) : -1;
        v[e] = p < p1 ? A[(int64_t)i * ldm + j[e]] : T(0);
      }
    };
    if (h > 0) load_row(h - 1);
    for (int i = h - 1; i >= 0; --i) {
      T vc[EPL];
      int jc[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e) { vc[e] = v[e]; jc[e] = j[e]; }
      const T piv = A[(int64_t)i * ldm + i];
      if (i > 0) load_row(i - 1);
      T s = T(0);
#pragma unroll
      for (int e = 0; e < EPL; ++e)
        if (jc[e] >= 0) s += vc[e] * x[jc[e]];
      // rows longer than EPL * 32 entries finish here
      for (int p = __ldg(d.uptr + i) + lane + 32 * EPL; p < __ldg(d.uptr + i + 1); p += 32) {
        const int c = __ldg(d.uidx + p);
        s += A[(int64_t)i * ldm + c] * x[c];
      }
      s = warp_sum(s);
      if (lane == 0) x[i] = (x[i] - s) * piv;
      __syncwarp();
    }
  }
}

// Substitution with the packed factors of one cell (warp per cell, x in
// shared memory).  The sparse head is resolved level by level (every row of a
// level at once, a lane per row), the L21 / U12 couplings a lane per row, and
// the dense tail block, stored column-major, by 32-column blocks: the
// block's 32 x 32 diagonal part with warp shuffles, then its columns applied
// to all remaining rows at once (right-looking), so every factor load is a
// coalesced 128-byte column segment and the loads of a block do not wait on
// one another.
template <class T>
__device__ void lu_substitute_packed(const Dev& d, const T* __restrict__ P, T* x, int lane) {
  const int n = d.n, h = d.head, nt = n - h, ldd = d.ldd;
  const int np1 = (nt + 31) / 32 + 1;
  T* xt = x + h;
  const T* __restrict__ D = P + d.p_d;
  // forward: L11 by levels
  for (int l = 0; l < d.n_flev; ++l) {
    const int r1 = __ldg(d.flev_ptr + l + 1);
    for (int q = __ldg(d.flev_ptr + l) + lane; q < r1; q += 32) {
      const int i = __ldg(d.flev + q);
      T s = T(0);
      for (int p = __ldg(d.lrptr + i); p < __ldg(d.lrptr + i + 1); ++p) s += P[d.p_l11 + p] * x[__ldg(d.lridx + p)];
      x[i] -= s;
    }
    __syncwarp();
  }
  // forward: L21 (tail rows, head columns)
  for (int i = lane; i < nt; i += 32) {
    const int cnt = __ldg(d.lrhead + i);
    if (cnt == 0) continue;
    const int p0 = __ldg(d.lrptr + h + i), o = d.p_l21 + __ldg(d.lrhoff + i);
    T s = T(0);
    for (int q = 0; q < cnt; ++q) s += P[o + q] * x[__ldg(d.lridx + p0 + q)];
    xt[i] -= s;
  }
  __syncwarp();
  // forward: dense tail, unit lower triangle
  constexpr int kR = 11;   // row chunks of 32 per pass over a block's columns
  for (int r0 = 0; r0 < nt; r0 += 32) {
    const int w = min(32, nt - r0);
    T lcol[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) lcol[k] = (k < w && lane < w && k < lane) ? D[(int64_t)(r0 + k) * ldd + r0 + lane] : T(0);
    T xi = lane < w ? xt[r0 + lane] : T(0);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const T xk = __shfl_sync(0xffffffffu, xi, k);
      if (lane > k) xi -= lcol[k] * xk;
    }
    if (lane < w) xt[r0 + lane] = xi;
    // rows below: x_r -= sum_k L(r, r0 + k) x_{r0+k}
    for (int rb = r0 + 32; rb < nt; rb += 32 * kR) {
      T acc[kR];
#pragma unroll
      for (int t = 0; t < kR; ++t) acc[t] = T(0);
      for (int k = 0; k < w; ++k) {
        const T xk = __shfl_sync(0xffffffffu, xi, k);
        const T* col = D + (int64_t)(r0 + k) * ldd + rb + lane;
#pragma unroll
        for (int t = 0; t < kR; ++t)
          if (rb + 32 * t + lane < nt) acc[t] += col[32 * t] * xk;
      }
#pragma unroll
      for (int t = 0; t < kR; ++t)
        if (rb + 32 * t + lane < nt) xt[rb + 32 * t + lane] -= acc[t];
    }
    __syncwarp();
  }
  // backward: dense tail, upper triangle with inverse pivots, last block first
  for (int r0 = (nt - 1) / 32 * 32; r0 >= 0; r0 -= 32) {
    const int w = min(32, nt - r0);
    T ucol[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) ucol[k] = (k < w && lane < w && k >= lane) ? D[(int64_t)(r0 + k) * ldd + r0 + lane] : T(0);
    T xi = lane < w ? xt[r0 + lane] : T(0);
#pragma unroll
    for (int k = 31; k >= 0; --k) {
      if (k < w) {
        if (lane == k) xi *= ucol[k];   // inverse pivot
        const T xk = __shfl_sync(0xffffffffu, xi, k);
        if (lane < k) xi -= ucol[k] * xk;
      }
    }
    if (lane < w) xt[r0 + lane] = xi;
    // rows above: x_r -= sum_k U(r, r0 + k) x_{r0+k}
    for (int ra = 0; ra < r0; ra += 32 * kR) {
      T acc[kR];
#pragma unroll
      for (int t = 0; t < kR; ++t) acc[t] = T(0);
      for (int k = 0; k < w; ++k) {
        const T xk = __shfl_sync(0xffffffffu, xi, k);
        const T* col = D + (int64_t)(r0 + k) * ldd + ra + lane;
#pragma unroll
        for (int t = 0; t < kR; ++t)
          if (ra + 32 * t + lane < r0) acc[t] += col[32 * t] * xk;
      }
#pragma unroll
      for (int t = 0; t < kR; ++t)
        if (ra + 32 * t + lane < r0) xt[ra + 32 * t + lane] -= acc[t];
    }
    __syncwarp();
  }
  // backward: U12 (head rows, tail columns)
  for (int i = lane; i < h; i += 32) {
    const int o = __ldg(d.u12off + i), cnt = __ldg(d.u12off + i + 1) - o, q0 = __ldg(d.uoff + i * np1);
    T s = T(0);
    for (int q = 0; q < cnt; ++q) s += P[d.p_u12 + o + q] * x[__ldg(d.uidx + q0 + q)];
    x[i] -= s;
  }
  __syncwarp();
  // backward: U11 by levels, then the inverse pivot
  for (int l = 0; l < d.n_blev; ++l) {
    const int r1 = __ldg(d.blev_ptr + l + 1);
    for (int q = __ldg(d.blev_ptr + l) + lane; q < r1; q += 32) {
      const int i = __ldg(d.blev + q);
      const int o = __ldg(d.u11ptr + i), cnt = __ldg(d.u11ptr + i + 1) - o, u0 = __ldg(d.uptr + i);
      T s = T(0);
      for (int e = 0; e < cnt; ++e) s += P[d.p_u11 + o + e] * x[__ldg(d.uidx + u0 + e)];
      x[i] = (x[i] - s) * P[d.p_dinv + i];
    }
    __syncwarp();
  }
}

template <class T>
__global__ void __launch_bounds__(32 * kSolveWarps) solve_update_kernel(Dev d, int need, int want) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * kSolveWarps + wi;
  if (c >= d.C || (d.compact && c >= d.counters[kCAct])) return;
  if ((d.flags[c] & need) != want) return;   // cells in Newton (and, in replays, on this factor set)
  const int n = d.n, xs = (n + 3) / 4 * 4;
  T* x = reinterpret_cast<T*>(smem_raw) + (int64_t)wi * xs;
  const double a0 = d.alpha[c], h = d.h[c];
  const double inv_a0 = 1.0 / a0;
  double rT = 0.0;   // the temperature row's residual, kept in FP64
  for (int s = lane; s < n; s += 32) {
    const int64_t o = (int64_t)s * d.ld + c;
    double b = -(a0 * d.y[o] + d.psi[o] - h * d.f[o]) * inv_a0;
    if (s == d.t_idx) rT = b;
    if (d.mixed) b *= d.wf[o];
    x[__ldg(d.iperm + s)] = T(b);
  }
  __syncwarp();
  if (d.lup) lu_substitute_packed<T>(d, static_cast<const T*>(d.lup) + (int64_t)d.slot_cell[c] * d.lup_stride, x, lane);
  else lu_substitute<T>(d, static_cast<const T*>(d.lu) + c * d.lu_stride, x, lane);
  const double gamma = d.gam[c], gJ = d.gam_J[c];
  const double scale = gamma != gJ ? 2.0 / (1.0 + gamma / gJ) : 1.0;
  // coupled temperature: T eliminated last (see th_border_kernel); the
  // species block's solution a0 becomes a0 - z bT, and T moves by bT
  double bT = 0.0;
  const double* bz = nullptr;
  if (d.therm) {
    const int64_t oc = d.slot_cell[c];
    const double* bgv = d.bgv + oc * d.bpad;
    bz = d.bz + oc * d.bpad;
    double dot = 0.0;
    for (int s = lane; s < n; s += 32) {
      if (s == d.t_idx) continue;
      double a = (double)x[__ldg(d.iperm + s)];
      if (d.mixed) a /= d.wf[(int64_t)s * d.ld + c];
      dot = fma(bgv[s], a, dot);
    }
    dot = warp_sum(dot);
    rT = __shfl_sync(0xffffffffu, rT, d.t_idx & 31);
    bT = (rT + dot) / d.bs[oc];
  }
  double acc = 0.0;
  for (int s = lane; s < n; s += 32) {
    const int64_t o = (int64_t)s * d.ld + c;
    double del = (double)x[__ldg(d.iperm + s)];
    if (d.mixed) del /= d.wf[o];
    if (bz) del = s == d.t_idx ? bT : fma(-bz[s], bT, del);
    del *= scale;
    d.y[o] += del;
    const double v = del * d.w[o];
    acc += v * v;
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const double dn = sqrt(acc / n);
    const int m = d.m_it[c];
    double crate = d.crate[c];
    const double dp = d.dprev[c];
    bool conv = false, fail = false;
    if (!isfinite(dn)) {
      fail = true;
    } else {
      if (m > 0) crate = fmax(0.3 * crate, dn / dp);
      if (dn * fmin(1.0, crate) <= d.newton_tol) conv = true;
      else if (m > 0 && dn > 2.0 * dp) fail = true;
      else if (m + 1 >= d.newton_max) fail = true;
    }
    d.crate[c] = crate;
    d.dprev[c] = dn;
    d.m_it[c] = m + 1;
    d.newton_iters[c] += 1;
    if (conv || fail) d.flags[c] = (d.flags[c] & ~F_NEWTON) | (conv ? F_CONV : F_FAILED);
  }
}

// ---------------------------------------------------------------------------
// coupled temperature (sm_net_set_thermal)
//
// T is component t_idx of the state.  Before every right-hand side the
// T-dependent coefficients (two-body, dissociative recombination) are
// recomputed from the slot's T into kslot; after the CRS gather of the
// chemical rows, th_energy_kernel sets the temperature row
//   f_t = (heat - n_H sum_i x_i L_i exp(-E_i/T) - lam n_H (T - T_dust)
//          - 3/2 T sum_{i != t} f_i) / (3/2 x_tot);
// after a refresh, th_border_kernel adds T to the Newton matrix by block
// elimination.
// ---------------------------------------------------------------------------
constexpr int kThRatesChunk = 64;
constexpr int kBorderWarps = 2;

// k' in slot order from the slots' temperatures Trow[slot] (a row of a
// state vector).  init = 1 (start of an integration): every class, every
// slot below C; else the T-dependent classes of the slots in Newton
// iterations.
__global__ void __launch_bounds__(128) th_rates_kernel(Dev d, const double* __restrict__ Trow, int init) {
  const int64_t c = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= d.C) return;
  if (!init && ((d.compact && c >= d.counters[kCAct]) || !(d.flags[c] & F_NEWTON))) return;
  const int j0 = blockIdx.y * kThRatesChunk, j1 = min(d.n_r, j0 + kThRatesChunk);
  const int64_t oc = d.slot_cell[c];
  const double T = Trow[c], nH = d.c_nH[oc];
  const double lt = log(T * (1.0 / 300.0)), it = 1.0 / T;
  for (int j = j0; j < j1; ++j) {
    const RatePar p = d.rpar[j];   // (log alpha | alpha, beta, gamma, class)
    const int cls = (int)p.w;
    double v;
    if (cls == SM_TWO_BODY || cls == SM_DISS_RECOMB) v = exp(fma(p.y, lt, p.x) - p.z * it) * nH;
    else if (!init) continue;
    else if (cls == SM_COSMIC_RAY) v = p.x * d.th_zeta;
    else v = d.c_chi[oc] * p.x * exp(-p.z * d.c_Av[oc]);
    d.kslot[(int64_t)j * d.ld + c] = v;
  }
}

// The temperature row f[t] from y and the chemical rows of f, for the slots
// in Newton iterations (init = 1: every slot below C).
__global__ void __launch_bounds__(128) th_energy_kernel(Dev d, const double* __restrict__ y, double* __restrict__ f,
                                                        int init) {
  const int64_t c = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= d.C) return;
  if (!init && ((d.compact && c >= d.counters[kCAct]) || !(d.flags[c] & F_NEWTON))) return;
  const int t = d.t_idx;
  const double T = y[(int64_t)t * d.ld + c];
  double xt = 0.0, F = 0.0;
  for (int s = 0; s < d.n; ++s) {
    if (s == t) continue;
    xt += y[(int64_t)s * d.ld + c];
    F += f[(int64_t)s * d.ld + c];
  }
  const int64_t oc = d.slot_cell[c];
  const double nH = d.c_nH[oc];
  double line = 0.0;
  for (int q = 0; q < d.n_cool; ++q) {
    const int i = __ldg(d.th_cool + q);
    line = fma(y[(int64_t)i * d.ld + c], d.th_L[i] * exp(-d.th_E[i] / T), line);
  }
  f[(int64_t)t * d.ld + c] = (d.th_heat - nH * line - d.th_lam * nH * (T - d.th_Td) - 1.5 * T * F) / (1.5 * xt);
}

// After a refresh, per refreshed cell (warp per cell): the temperature
// border of its Newton matrix.  With u = dF/dT (F the chemical rows),
// v = d f_t / dx and w = d f_t / dT at the predicted state, the full matrix
// is  [M, -gJ u; -gJ v^T, 1 - gJ w]  (M the species block the refresh
// factorised, gJ = gamma_J).  Eliminating T last leaves
//   z = M^-1 (-gJ u),   s = 1 - gJ w + gJ v.z,
// and the Newton correction of a residual (r, r_T) is (a0 - z b, b) with
// a0 = M^-1 r and b = (r_T + gJ v.a0) / s (solve_update_kernel).  The
// sums over the chemical rows come from the reactions: sum_i S_ij = dn_j,
// so sum_i f_i = sum_j dn_j R_j and sum_i J_il = sum_j dn_j dR_j/dx_l.
template <class T>
__global__ void __launch_bounds__(32 * kBorderWarps) th_border_kernel(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int n = d.n, t = d.t_idx, xs = (n + 3) / 4 * 4;
  double* u = reinterpret_cast<double*>(smem_raw) + (int64_t)wi * 3 * xs;   // dF/dT
  double* vv = u + xs;                                                      // sum_j dn_j dR_j/dx_l
  double* ys = vv + xs;                                                     // the predicted state
  T* x = reinterpret_cast<T*>(reinterpret_cast<double*>(smem_raw) + (int64_t)kBorderWarps * 3 * xs) +
         (int64_t)wi * xs;
  const int count = d.counters[0];
  for (int e = blockIdx.x * kBorderWarps + wi; e < count; e += gridDim.x * kBorderWarps) {
    const int64_t c = d.list[e];
    const int64_t oc = d.slot_cell[c];
    for (int s = lane; s < n; s += 32) {
      u[s] = 0.0;
      vv[s] = 0.0;
      ys[s] = d.ypred[(int64_t)s * d.ld + c];
    }
    __syncwarp();
    const double Tc = ys[t], it = 1.0 / Tc;
    double F = 0.0, U = 0.0;
    for (int j = lane; j < d.n_r; j += 32) {
      const int2 rc = __ldg(d.reac + j);
      const double kv = d.kslot[(int64_t)j * d.ld + c];
      const double ya = ys[rc.x], yb = rc.y >= 0 ? ys[rc.y] : 1.0;
      const double R = kv * ya * yb;
      const RatePar p = d.rpar[j];
      const int cls = (int)p.w;
      const double g = (cls == SM_TWO_BODY || cls == SM_DISS_RECOMB) ? (p.y + p.z * it) * it : 0.0;  // d ln k'/dT
      const double dn = __ldg(d.th_dn + j);
      F = fma(dn, R, F);
      if (g != 0.0) {
        const double Rg = R * g;
        U = fma(dn, Rg, U);
        for (int q = __ldg(d.sc_ptr + j); q < __ldg(d.sc_ptr + j + 1); ++q) {
          const uint32_t ent = __ldg(d.sc_ent + q);
          atomicAdd(&u[ent & 0xFFFFFF], (double)(int8_t)(ent >> 24) * Rg);
        }
      }
      if (dn != 0.0) {
        if (rc.y < 0) {
          atomicAdd(&vv[rc.x], dn * kv);
        } else if (rc.x == rc.y) {
          atomicAdd(&vv[rc.x], dn * 2.0 * kv * ya);
        } else {
          atomicAdd(&vv[rc.x], dn * kv * yb);
          atomicAdd(&vv[rc.y], dn * kv * ya);
        }
      }
    }
    F = warp_sum(F);
    U = warp_sum(U);
    __syncwarp();
    const double nH = d.c_nH[oc];
    double xt = 0.0, line = 0.0, dline = 0.0;
    for (int s = lane; s < n; s += 32)
      if (s != t) xt += ys[s];
    for (int q = lane; q < d.n_cool; q += 32) {
      const int i = __ldg(d.th_cool + q);
      const double cl = d.th_L[i] * exp(-d.th_E[i] * it);
      line = fma(ys[i], cl, line);
      dline = fma(ys[i] * cl, d.th_E[i] * it * it, dline);
    }
    xt = warp_sum(xt);
    line = warp_sum(line);
    dline = warp_sum(dline);
    const double i15x = 1.0 / (1.5 * xt);
    const double fT = (d.th_heat - nH * line - d.th_lam * nH * (Tc - d.th_Td) - 1.5 * Tc * F) * i15x;
    const double w = (-nH * dline - d.th_lam * nH - 1.5 * F - 1.5 * Tc * U) * i15x;
    const double gJ = d.gam_J[c];
    for (int s = lane; s < n; s += 32) {
      double b = s == t ? 0.0 : -gJ * u[s];
      if (d.mixed) b *= d.wf[(int64_t)s * d.ld + c];
      x[__ldg(d.iperm + s)] = T(b);
    }
    __syncwarp();
    lu_substitute_packed<T>(d, static_cast<const T*>(d.lup) + oc * d.lup_stride, x, lane);
    double* bz = d.bz + oc * d.bpad;
    double* bgv = d.bgv + oc * d.bpad;
    double vz = 0.0;
    for (int s = lane; s < n; s += 32) {
      double z = 0.0, v = 0.0;
      if (s != t) {
        z = (double)x[__ldg(d.iperm + s)];
        if (d.mixed) z /= d.wf[(int64_t)s * d.ld + c];
        const double cl = d.th_L[s] > 0.0 ? d.th_L[s] * exp(-d.th_E[s] * it) : 0.0;
        v = (-nH * cl - 1.5 * Tc * vv[s]) * i15x - fT / xt;
      }
      bz[s] = z;
      bgv[s] = gJ * v;
      vz = fma(v, z, vz);
    }
    vz = warp_sum(vz);
    if (lane == 0) d.bs[oc] = 1.0 - gJ * w + gJ * vz;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// finish: error test, step / order selection, history update
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kCoopWarps) finish_kernel(Dev d) {
  // partial WRMS sums of the warps (error test, then the two neighbouring orders)
  __shared__ double red_e[kCoopWarps][32], red_lo[kCoopWarps][32], red_hi[kCoopWarps][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const bool live = c < d.C && !(d.compact && c >= d.counters[kCAct]);
  const int n = d.n;
  int fl = live ? d.flags[c] : 0;
  const bool go = (fl & F_ATTEMPT) != 0;
  fl &= ~F_ATTEMPT;
  const bool work = go && !(fl & F_FAILED);   // an error test to run
  int q = 1, nh = 1;
  double h = 0.0, tnew = 0.0;
  double T[QMAX + 1];
  if (go) {
    q = d.q[c];
    nh = d.nh[c];
    h = d.h[c];
  }
  if (work) {
    tnew = (fl & F_FINAL) ? d.t_end : d.t[c] + h;
    for (int i = 0; i < nh; ++i) T[i] = d.tn[(int64_t)i * d.ld + c];
  }
  // pass 1: the error estimate, species split over the warps
  double acc = 0.0;
  if (work) {
#pragma unroll 4
    for (int s = wi; s < n; s += kCoopWarps) {
      const int64_t o = (int64_t)s * d.ld + c;
      const double v = (d.y[o] - d.ypred[o]) * d.w[o];
      acc += v * v;
    }
  }
  red_e[wi][lane] = acc;
  __syncthreads();
  acc = 0.0;
  for (int w = 0; w < kCoopWarps; ++w) acc += red_e[w][lane];   // same order in every warp
  const double err = work ? (nh >= q + 1 ? h / (tnew - T[q]) : 1.0 / (q + 1)) * sqrt(acc / n) : 0.0;
  const bool accepted = work && isfinite(err) && err <= 1.0;
  // pass 2: rate the neighbouring orders on the old history
  const int naq = accepted ? d.n_at_q[c] + 1 : 0;
  const bool lo = accepted && naq >= q + 1 && q > 1;
  const bool hi = accepted && naq >= q + 1 && q < d.q_max && (fl & F_HAS_EPREV) && nh + 1 >= q + 2;
  double wl[QMAX + 1];
  if (lo) lagrange(T, q, tnew, wl);
  double acc_lo = 0.0, acc_hi = 0.0;
  if (lo || hi) {
#pragma unroll 2
    for (int s = wi; s < n; s += kCoopWarps) {
      const int64_t o = (int64_t)s * d.ld + c;
      const double yv = d.y[o], wv = d.w[o];
      if (lo) {
        double p = 0.0;
#pragma unroll
        for (int i = 0; i < QMAX; ++i)
          if (i < q) p += wl[i] * Yh(d, i)[o];
        const double v = (yv - p) * wv;
        acc_lo += v * v;
      }
      if (hi) {
        const double v = ((yv - d.ypred[o]) - d.eprev[o]) * wv;
        acc_hi += v * v;
      }
    }
  }
  red_lo[wi][lane] = acc_lo;
  red_hi[wi][lane] = acc_hi;
  __syncthreads();
  acc_lo = acc_hi = 0.0;
  for (int w = 0; w < kCoopWarps; ++w) {
    acc_lo += red_lo[w][lane];
    acc_hi += red_hi[w][lane];
  }
  double best_eta = accepted ? 0.9 * pow(fmax(err, 1e-10), -1.0 / (q + 1)) : 0.0;
  int best_q = q;
  if (lo) {
    const double est = h / (tnew - T[q - 1]) * sqrt(acc_lo / n);
    const double eta_lo = 0.8 * pow(fmax(est, 1e-10), -1.0 / q);
    if (eta_lo > best_eta) {
      best_eta = eta_lo;
      best_q = q - 1;
    }
  }
  if (hi) {
    const double est = sqrt(acc_hi / n) / (q + 2);
    const double eta_hi = 0.7 * pow(fmax(est, 1e-10), -1.0 / (q + 2));
    if (eta_hi > best_eta) {
      best_eta = eta_hi;
      best_q = q + 1;
    }
  }
  // pass 3: shift the history of the accepted cells, newest first (each warp
  // its own species, which pass 2 read before)
  const int nh_new = min(nh + 1, d.q_max + 1);
  const bool keep_e = best_q == q;
  if (accepted) {
#pragma unroll 4
    for (int s = wi; s < n; s += kCoopWarps) {
      const int64_t o = (int64_t)s * d.ld + c;
      double Yv[QMAX];
#pragma unroll
      for (int i = 0; i < QMAX; ++i) Yv[i] = i < nh_new - 1 ? Yh(d, i)[o] : 0.0;
      const double yv = d.y[o];
      const double yp = keep_e ? d.ypred[o] : 0.0;
#pragma unroll
      for (int i = 0; i < QMAX; ++i)
        if (i < nh_new - 1) Yh(d, i + 1)[o] = Yv[i];
      if (keep_e) d.eprev[o] = yv - yp;
      Yh(d, 0)[o] = yv;
    }
  }
  __syncthreads();   // the history is complete (checkpoints read it)
  if (wi != 0 || !go) return;
  // the cell's scalars, warp 0 alone
  if (fl & F_FAILED) {
    d.conv_fails[c] += 1;
    const int cf = d.ccf[c] + 1;
    d.ccf[c] = cf;
    if (cf >= d.max_conv_fails) {
      d.status[c] = SM_CELL_CONV;
    } else {
      if (fl & F_REFRESH) h *= 0.25;
      fl |= F_NEED_J | F_REJECTED;
      d.h[c] = h;
    }
    d.flags[c] = fl;
    return;
  }
  if (!isfinite(err)) {
    d.status[c] = SM_CELL_NAN;
    d.flags[c] = fl;
    return;
  }
  if (err > 1.0) {
    d.rejects[c] += 1;
    const int cr = d.crej[c] + 1;
    d.crej[c] = cr;
    const double eta = fmax(0.2, 0.9 * pow(err, -1.0 / (q + 1)));
    if (cr >= 3 && q > 1) {
      d.q[c] = 1;
      d.n_at_q[c] = 0;
      fl &= ~F_HAS_EPREV;
    }
    d.h[c] = h * eta;
    d.flags[c] = fl | F_REJECTED;
    return;
  }
  for (int i = nh_new - 1; i >= 1; --i) d.tn[(int64_t)i * d.ld + c] = T[i - 1];
  d.tn[c] = tnew;
  d.nh[c] = nh_new;
  d.t[c] = tnew;
  d.steps[c] += 1;
  if (d.record) {
    const int m = d.steps[c];  // 1-based index of this accepted step
    if (m <= d.record) {
      d.log_t[(int64_t)(m - 1) * d.ld + c] = tnew;
      d.log_h[(int64_t)(m - 1) * d.ld + c] = h;
      d.log_q[(int64_t)(m - 1) * d.ld + c] = q;
      if (m % kCkpt == 0) store_checkpoint(d, c, m / kCkpt);
    }
  }
  d.j_age[c] += 1;
  d.crej[c] = 0;
  d.ccf[c] = 0;
  if (!keep_e) {
    d.q[c] = best_q;
    d.n_at_q[c] = 0;
    fl &= ~F_HAS_EPREV;
  } else {
    d.n_at_q[c] = naq;
    fl |= F_HAS_EPREV;
  }
  double eta = fmin(best_eta, (fl & F_REJECTED) ? 1.0 : d.eta_max);
  eta = fmax(eta, 0.2);
  if (eta >= 1.0 && eta < d.eta_keep) eta = 1.0;
  d.h[c] = h * eta;
  fl &= ~F_REJECTED;
  if (fl & F_FINAL) d.status[c] = SM_CELL_OK;
  d.flags[c] = fl;
}

__global__ void read_kernel(Dev d, double* __restrict__ yout, int64_t ldu, sm_cell_stats* __restrict__ st) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int64_t oc = d.slot_cell[c];   // the caller's cell held in slot c
  if (yout)
    for (int s = 0; s < d.n; ++s) yout[(int64_t)s * ldu + oc] = Yh(d, 0)[(int64_t)s * d.ld + c];
  if (st) {
    sm_cell_stats r;
    r.status = d.status[c];
    r.steps = d.steps[c];
    r.rejects = d.rejects[c];
    r.conv_fails = d.conv_fails[c];
    r.newton_iters = d.newton_iters[c];
    r.jac_evals = d.jac_evals[c];
    r.q_last = d.q[c];
    r.pad = 0;
    r.t = d.t[c];
    r.h = d.h[c];
    st[oc] = r;
  }
}

// After a state is loaded without its Newton factors: every cell refreshes
// its Newton matrix on its next attempt.
__global__ void need_j_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  d.flags[c] |= F_NEED_J;
}

// counters[1] = cells still running, counters[2] = cells stopped short of t_end
__global__ void count_running_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int s = d.status[c];
  if (s == SM_CELL_RUNNING) atomicAdd(&d.counters[1], 1);
  else if (s != SM_CELL_OK) atomicAdd(&d.counters[2], 1);
}

// ---------------------------------------------------------------------------
// Compaction of the running cells.  Cells finish after very different numbers
// of steps (a few dozen to over a thousand), and every kernel of an attempt
// works on whole warps or blocks of consecutive slots, so the finished cells
// scattered among the running ones cost as much as running ones.  After a
// group of attempts, once an eighth of the running range has finished, the
// finished slots below the new boundary (the number of running cells) swap
// their contents with the running slots above it; the two sets are disjoint,
// so the swaps need no ordering.  A slot's contents are its per-cell scalars
// (slot_cell included), its vectors and its rate coefficients; the packed
// factors stay where they are and are found through slot_cell.  Per-cell results do not
// depend on the slot, so compaction changes no result.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool compaction_due(int ca, int cn) { return ca - cn >= max(256, ca / 8); }

__global__ void compact_count_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C || c >= d.counters[kCAct]) return;
  if (d.status[c] == SM_CELL_RUNNING) atomicAdd(&d.counters[kCLive], 1);
}

__global__ void compact_list_kernel(Dev d) {
  const int ca = d.counters[kCAct], cn = d.counters[kCLive];
  if (!compaction_due(ca, cn)) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C || c >= ca) return;
  const bool run = d.status[c] == SM_CELL_RUNNING;
  if (c < cn && !run) d.holes[atomicAdd(&d.counters[kCHoles], 1)] = (int)c;
  else if (c >= cn && run) d.runners[atomicAdd(&d.counters[kCRun], 1)] = (int)c;
}

template <class U>
__device__ __forceinline__ void swap_rows(U* base, int rows, int64_t ld, int64_t a, int64_t b, int t, int nt) {
  for (int r = t; r < rows; r += nt) {
    U* p = base + (int64_t)r * ld;
    const U va = p[a], vb = p[b];
    p[a] = vb;
    p[b] = va;
  }
}

__global__ void __launch_bounds__(256) compact_swap_kernel(Dev d) {
  const int np = min(d.counters[kCHoles], d.counters[kCRun]);
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const int64_t a = d.holes[p], b = d.runners[p];
    // per-cell scalars: the double rows t .. alpha[QMAX] and the int rows
    // q .. slot_cell are contiguous with stride ld (see sm_state_create)
    swap_rows(d.t, 6 + 2 * (QMAX + 1), d.ld, a, b, threadIdx.x, blockDim.x);
    swap_rows(d.q, 15, d.ld, a, b, threadIdx.x, blockDim.x);
    // history and working vectors: Y[QMAX + 1], ypred, y, psi, f, f0, eprev, w, wf
    swap_rows(d.Y, (QMAX + 1 + 8) * d.n, d.ld, a, b, threadIdx.x, blockDim.x);
    swap_rows(d.kslot, d.n_r, d.ld, a, b, threadIdx.x, blockDim.x);
  }
}

__global__ void compact_commit_kernel(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int ca = d.counters[kCAct], cn = d.counters[kCLive];
    if (compaction_due(ca, cn)) d.counters[kCAct] = cn;
    d.counters[kCHoles] = d.counters[kCRun] = d.counters[kCLive] = 0;
  }
}

// After a state is loaded: every slot counts as possibly running.
__global__ void set_active_kernel(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    d.counters[kCAct] = (int)d.C;
    d.counters[kCHoles] = d.counters[kCRun] = d.counters[kCLive] = 0;
  }
}

// Rate coefficients in slot order from the caller's array (after a state
// was loaded, or when sm_step_bdf gets another k than the integration began with).
__global__ void kslot_gather_kernel(Dev d, const double* __restrict__ k, int64_t ldk) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int64_t oc = d.slot_cell[c];
  for (int j = 0; j < d.n_r; ++j) d.kslot[(int64_t)j * d.ld + c] = k[(int64_t)j * ldk + oc];
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the frozen-step map (reverse sweep).
//
// The recorded accepted steps (t_m, h_m, q_m) of the last integration are
// fixed and every implicit step alpha_0 y_m + sum_i alpha_i y_{m-i} - h_m f(y_m)
// = 0 is solved to a tight tolerance.  Segments of kCkpt steps are recomputed
// from their stored step history, last segment first; each recomputed state
// y_m gets its own factorisation of M_m = I - gamma_m J(y_m), kept in one of
// kCkpt slots, which is also the Newton matrix of step m + 1.  Walking the
// segment backwards, lambda_m solves
//   (alpha_0^m M_m)^T lambda_m = c [m = N] - sum_d alpha_d^{m+d} lambda_{m+d}
// over d = 1..QMAX with d <= q_{m+d}, and
//   dPhi / d log k_j += h_m R_j(y_m) (S^T lambda_m)_j,
// since f = S R and every R_j is proportional to k_j.
// Cells are processed in passes of at most `cells_per_pass`; inside a pass
// the cell index is local (Dev pointers are shifted to the pass's first cell)
// and the adjoint arrays use their own stride lda.
// ---------------------------------------------------------------------------
constexpr int kRing = QMAX + 1;          // lambda history slots, indexed by m mod kRing
constexpr double kReplayTol = 1e-4;      // Newton tolerance of the recomputed steps (WRMS units)
constexpr int kReplayIters = 8;

struct AdjDev {
  int n_cot;
  double run_tol;               // Newton tolerance of the recorded run
  int64_t lda;
  int *N, *K, *seg, *astat;     // [lda]: frozen steps, segments, current segment, status
  int* seg_q;                   // [kCkpt][lda]
  int* ring_q;                  // [kRing][lda]
  double* seg_y;                // [kCkpt][n][lda] recomputed states of the segment
  double* seg_h;                // [kCkpt][lda]
  double* seg_alpha;            // [kCkpt][QMAX+1][lda]
  double* ring_alpha;           // [kRing][QMAX+1][lda]
  double* lam;                  // [kRing][n_cot][n][lda]
  double* kc;                   // [Cc][n_r] rate coefficients, cell-major
  double* g;                    // [Cc][n_cot][n_r] gradient accumulators, cell-major
  double* slots;                // [kCkpt][Cc][lu_stride] factors of M_m
  const double* cot;            // [n_cot][n][ldu]
  int64_t ldu;
};

__device__ __forceinline__ double* slot_lu(const Dev& d, const AdjDev& a, int j, int64_t c) {
  return a.slots + ((int64_t)j * d.C + c) * d.lu_stride;
}

__global__ void adj_setup_kernel(Dev d, AdjDev a, const double* __restrict__ k, int64_t ldk) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int N = d.steps[c];
  const bool ok = d.status[c] == SM_CELL_OK && N >= 1 && N <= d.record;
  const int K = ok ? (N + kCkpt - 1) / kCkpt : 0;
  a.N[c] = ok ? N : 0;
  a.K[c] = K;
  a.astat[c] = ok ? 0 : 1;
  atomicMax(&d.counters[3], K);
  atomicMax(&d.counters[1], ok ? N : 0);
  for (int j = 0; j < d.n_r; ++j) a.kc[c * d.n_r + j] = k[(int64_t)j * ldk + c];
  for (int64_t i = 0; i < (int64_t)a.n_cot * d.n_r; ++i) a.g[c * a.n_cot * d.n_r + i] = 0.0;
  for (int i = 0; i < kRing; ++i) a.ring_q[(int64_t)i * a.lda + c] = 0;
}

// Restores the step history stored before segment K - 1 - rs (rs >= 0), or
// before segment 0 for every cell (rs < 0: a replay from the start).
__global__ void seg_restore_kernel(Dev d, AdjDev a, int rs) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int sg = a.astat[c] == 0 ? (rs >= 0 ? a.K[c] - 1 - rs : 0) : -1;
  a.seg[c] = sg;
  if (sg < 0) return;
  const int nh = d.ck_nh[(int64_t)sg * d.ld + c];
  const int64_t vs = (int64_t)d.n * d.ld;
  const double* src = d.ck_Y + (int64_t)sg * (QMAX + 1) * vs;
  for (int i = 0; i < nh; ++i) {
    for (int s = 0; s < d.n; ++s) Yh(d, i)[(int64_t)s * d.ld + c] = src[i * vs + (int64_t)s * d.ld + c];
    d.tn[(int64_t)i * d.ld + c] = d.ck_t[((int64_t)sg * (QMAX + 1) + i) * d.ld + c];
  }
  d.nh[c] = nh;
}

// Global index m of segment position j for cell c, 0 if the cell has none.
__device__ __forceinline__ int seg_step(const AdjDev& a, int64_t c, int j) {
  const int sg = a.seg[c];
  if (sg < 0) return 0;
  const int m = sg * kCkpt + 1 + j;
  return m <= a.N[c] ? m : 0;
}

// Predictor, BDF coefficients and Newton set-up of frozen step m; with
// `store` the step's h, q and alpha are kept for the backward pass.
__global__ void rpredict_kernel(Dev d, AdjDev a, int j, int store) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int m = seg_step(a, c, j);
  if (!m) {
    d.flags[c] = 0;
    return;
  }
  const double tnew = d.log_t[(int64_t)(m - 1) * d.ld + c];
  const double h = d.log_h[(int64_t)(m - 1) * d.ld + c];
  const int q = d.log_q[(int64_t)(m - 1) * d.ld + c];
  const int nh = d.nh[c];
  double T[QMAX + 1], wts[QMAX + 1], al[QMAX + 1];
  for (int i = 0; i < nh; ++i) T[i] = d.tn[(int64_t)i * d.ld + c];
  const bool lagr = nh > q;
  if (lagr) lagrange(T, q + 1, tnew, wts);
  bdf_alphas(tnew, T, q, h, al);
  d.h[c] = h;
  d.gam[c] = h / al[0];
  for (int i = 0; i <= QMAX; ++i) {
    const double v = i <= q ? al[i] : 0.0;
    d.alpha[(int64_t)i * d.ld + c] = v;
    if (store) a.seg_alpha[((int64_t)j * (QMAX + 1) + i) * a.lda + c] = v;
  }
  if (store) {
    a.seg_h[(int64_t)j * a.lda + c] = h;
    a.seg_q[(int64_t)j * a.lda + c] = q;
  }
  // the previous step's factors serve as Newton matrix unless gamma moved too
  // far from theirs (the integrator's own refresh rule); every kCkpt-th step
  // (each segment's first) starts from fresh factors at the predictor
  const bool fresh = j % kCkpt == 0 || fabs(h / al[0] / d.gam_J[c] - 1.0) > d.gamma_tol;
  d.flags[c] = F_NEWTON | (fresh ? F_REFRESH : 0);
  d.m_it[c] = 0;
  d.dprev[c] = 0.0;
  d.crate[c] = 1.0;
  for (int s = 0; s < d.n; ++s) {
    const int64_t o = (int64_t)s * d.ld + c;
    const double y0 = Yh(d, 0)[o];
    double yp;
    if (lagr) {
      yp = 0.0;
      for (int i = 0; i <= q; ++i) yp += wts[i] * Yh(d, i)[o];
    } else {
      yp = y0 + h * d.f0[o];
    }
    double ps = 0.0;
    for (int i = 1; i <= q; ++i) ps += al[i] * Yh(d, i - 1)[o];
    d.ypred[o] = yp;
    d.y[o] = yp;
    d.psi[o] = ps;
    d.w[o] = 1.0 / (d.rtol * fabs(y0) + d.atol);
  }
}

// Refresh list: the cells that take frozen step j (need_flag = 0), or those
// of them whose flags contain need_flag.
__global__ void adj_list_kernel(Dev d, AdjDev a, int j, int need_flag) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  if (seg_step(a, c, j) && (d.flags[c] & need_flag) == need_flag) d.list[atomicAdd(&d.counters[0], 1)] = (int)c;
}

// Second chance for cells whose Newton iteration did not converge: restart
// from the predictor with fresh factors (F_REFRESH); converged cells are
// taken out of the Newton set.
__global__ void rretry_kernel(Dev d, AdjDev a, int j) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  if (!seg_step(a, c, j)) return;
  if (d.flags[c] & F_CONV) {
    d.flags[c] = F_CONV;
    return;
  }
  d.flags[c] = F_NEWTON | F_REFRESH;
  d.m_it[c] = 0;
  d.dprev[c] = 0.0;
  d.crate[c] = 1.0;
  for (int s = 0; s < d.n; ++s) d.y[(int64_t)s * d.ld + c] = d.ypred[(int64_t)s * d.ld + c];
}

// Keeps the solved state for the backward pass and shifts the history; the
// state also becomes the point at which the next refresh evaluates J.
__global__ void rcommit_kernel(Dev d, AdjDev a, int j, int store) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int m = seg_step(a, c, j);
  if (!m) return;
  // iterations stopped short of the replay tolerance still count when the
  // last correction met the tolerance the recorded run was solved to
  if (!(d.flags[c] & F_CONV) && !(d.dprev[c] <= a.run_tol)) a.astat[c] = 2;
  const int nh = d.nh[c], nh_new = min(nh + 1, d.q_max + 1);
  for (int s = 0; s < d.n; ++s) {
    const int64_t o = (int64_t)s * d.ld + c;
    const double yv = d.y[o];
    if (store) {
      a.seg_y[((int64_t)j * d.n + s) * a.lda + c] = yv;
      d.ypred[o] = yv;
    }
    for (int i = nh_new - 1; i >= 1; --i) Yh(d, i)[o] = Yh(d, i - 1)[o];
    Yh(d, 0)[o] = yv;
  }
  for (int i = nh_new - 1; i >= 1; --i) d.tn[(int64_t)i * d.ld + c] = d.tn[(int64_t)(i - 1) * d.ld + c];
  d.tn[c] = d.log_t[(int64_t)(m - 1) * d.ld + c];
  d.nh[c] = nh_new;
}

// One backward step at segment position j: block = one cell, one warp per
// cotangent.  The slot holds the factors of M_m in elimination order (unit L,
// U with inverse pivots on the diagonal), so M_m^T = U^T L^T is solved as a
// forward sweep over the rows of U followed by a backward sweep over the rows
// of L, each row scattering its contribution.
__global__ void adj_step_kernel(Dev d, AdjDev a, int j) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t c = blockIdx.x;
  const int m = seg_step(a, c, j);
  if (!m) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int n = d.n, n_r = d.n_r, ldm = d.ldm;
  double* Rs = reinterpret_cast<double*>(smem_raw);  // [n_r] reaction rates at y_m
  double* xs = Rs + n_r + (size_t)warp * 2 * n;      // this warp's vector, elimination order
  double* ls = xs + n;                               // lambda_m in species order
  const double* ym = a.seg_y + (int64_t)j * n * a.lda;
  for (int r = tid; r < n_r; r += blockDim.x) {
    const int2 rc = __ldg(d.reac + r);
    double v = a.kc[c * n_r + r] * ym[(int64_t)rc.x * a.lda + c];
    if (rc.y >= 0) v *= ym[(int64_t)rc.y * a.lda + c];
    Rs[r] = v;
  }
  __syncthreads();
  const double h = a.seg_h[(int64_t)j * a.lda + c];
  const double inv_a0 = 1.0 / a.seg_alpha[((int64_t)j * (QMAX + 1)) * a.lda + c];
  const int N = a.N[c];
  const int slot = m % kRing;
  const double* A = slot_lu(d, a, j, c);
  for (int v = warp; v < a.n_cot; v += nwarps) {
    for (int s = lane; s < n; s += 32) {
      double b = m == N ? a.cot[((int64_t)v * n + s) * a.ldu + c] : 0.0;
      for (int dd = 1; dd <= QMAX && m + dd <= N; ++dd) {
        const int sl = (m + dd) % kRing;
        if (a.ring_q[(int64_t)sl * a.lda + c] >= dd)
          b -= a.ring_alpha[((int64_t)sl * (QMAX + 1) + dd) * a.lda + c] *
               a.lam[(((int64_t)sl * a.n_cot + v) * n + s) * a.lda + c];
      }
      xs[__ldg(d.iperm + s)] = b * inv_a0;
    }
    __syncwarp();
    // U^T: u_k = x_k / u_kk, then x_j -= u_kj u_k over row k of U
    for (int kk = 0; kk < n; ++kk) {
      const double uk = xs[kk] * A[(int64_t)kk * ldm + kk];
      __syncwarp();
      if (lane == 0) xs[kk] = uk;
      const double* Ak = A + (int64_t)kk * ldm;
      const int p1 = __ldg(d.uptr + kk + 1);
      for (int p = __ldg(d.uptr + kk) + lane; p < p1; p += 32) {
        const int jj = __ldg(d.uidx + p);
        xs[jj] -= Ak[jj] * uk;
      }
      __syncwarp();
    }
    // L^T (unit): v_i is final once the rows below it are done; x_k -= l_ik v_i
    for (int ii = n - 1; ii > 0; --ii) {
      const double vi = xs[ii];
      const double* Ai = A + (int64_t)ii * ldm;
      const int p1 = __ldg(d.lrptr + ii + 1);
      for (int p = __ldg(d.lrptr + ii) + lane; p < p1; p += 32) {
        const int kk = __ldg(d.lridx + p);
        xs[kk] -= Ai[kk] * vi;
      }
      __syncwarp();
    }
    for (int s = lane; s < n; s += 32) {
      const double lv = xs[__ldg(d.iperm + s)];
      ls[s] = lv;
      a.lam[(((int64_t)slot * a.n_cot + v) * n + s) * a.lda + c] = lv;
    }
    __syncwarp();
    double* gv = a.g + (c * a.n_cot + v) * n_r;
    for (int r = lane; r < n_r; r += 32) {
      double w = 0.0;
      const int p1 = __ldg(d.sc_ptr + r + 1);
      for (int p = __ldg(d.sc_ptr + r); p < p1; ++p) {
        const uint32_t e = __ldg(d.sc_ent + p);
        w = fma((double)(int8_t)(e >> 24), ls[e & 0xFFFFFFu], w);
      }
      gv[r] = fma(h * Rs[r], w, gv[r]);
    }
    __syncwarp();
  }
  __syncthreads();
  if (tid == 0) a.ring_q[(int64_t)slot * a.lda + c] = a.seg_q[(int64_t)j * a.lda + c];
  if (tid <= QMAX)
    a.ring_alpha[((int64_t)slot * (QMAX + 1) + tid) * a.lda + c] =
        a.seg_alpha[((int64_t)j * (QMAX + 1) + tid) * a.lda + c];
}

// Gradient out as [n_cot][n_r][ldg] (cells fastest), per-cell status, and the
// number of cells without a usable result in counters[2].
__global__ void adj_out_kernel(Dev d, AdjDev a, double* __restrict__ out, int64_t ldg, int* __restrict__ astat_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  for (int v = 0; v < a.n_cot; ++v)
    for (int r = 0; r < d.n_r; ++r)
      out[((int64_t)v * d.n_r + r) * ldg + c] = a.g[(c * a.n_cot + v) * d.n_r + r];
  const int s = a.astat[c];
  if (astat_out) astat_out[c] = s;
  if (s) atomicAdd(&d.counters[2], 1);
}

// dPhi/dy_0 = -sum_{m'} alpha_{m'}^{m'} lambda_{m'} over the first steps with
// q_{m'} >= m' (their lambdas are still in the ring once segment 0 is done),
// as out[n_cot][n][ldg]; 0 for cells without a usable result.
__global__ void adj_y0_kernel(Dev d, AdjDev a, double* __restrict__ out, int64_t ldg) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const bool ok = a.astat[c] == 0;
  const int N = a.N[c];
  for (int v = 0; v < a.n_cot; ++v)
    for (int s = 0; s < d.n; ++s) {
      double g = 0.0;
      for (int mp = 1; ok && mp <= QMAX && mp <= N; ++mp) {
        const int sl = mp % kRing;
        if (a.ring_q[(int64_t)sl * a.lda + c] >= mp)
          g -= a.ring_alpha[((int64_t)sl * (QMAX + 1) + mp) * a.lda + c] *
               a.lam[(((int64_t)sl * a.n_cot + v) * d.n + s) * a.lda + c];
      }
      out[((int64_t)v * d.n + s) * ldg + c] = g;
    }
}

// Replay result: y_N of replayed cells, NaN for the others.
__global__ void replay_out_kernel(Dev d, AdjDev a, double* __restrict__ yout, int64_t ldu,
                                  int* __restrict__ astat_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int s = a.astat[c];
  for (int i = 0; i < d.n; ++i) yout[(int64_t)i * ldu + c] = s == 0 ? Yh(d, 0)[(int64_t)i * d.ld + c] : NAN;
  if (astat_out) astat_out[c] = s;
  if (s) atomicAdd(&d.counters[2], 1);
}

}  // namespace

// Cell conditions of a thermal state (chi = 1 where none is given).
static __global__ void th_cells_kernel(Dev d, int64_t C, const double* __restrict__ nH, const double* __restrict__ Av,
                                const double* __restrict__ chi) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double* cond = const_cast<double*>(d.c_nH);
  cond[c] = nH[c];
  cond[d.ld + c] = Av[c];
  cond[2 * d.ld + c] = chi ? chi[c] : 1.0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sm_state {
  const sm_net* net = nullptr;
  sm_opts opts{};
  int64_t cap = 0, C = 0, ld = 0;
  double t_end = 0.0;
  Dev d{};
  DevArray scal_d, scal_i, vec, lu, lup, list, counters, scratch, rec_d, rec_i, kslot, cpt;
  DevArray th_par, th_cool, cond, bord;   // coupled temperature: parameters, coolants, cell conditions, border
  int64_t cells_set = 0;                  // cells whose conditions sm_state_set_cells copied
  size_t border_smem = 0;
  const double* kslot_src = nullptr;   // the caller's k the slot-ordered copy was taken from
  DevArray adj_d, adj_i, adj_lu;   // sm_adjoint workspace, grown on demand
  cudaStream_t s = nullptr, s2 = nullptr;          // s2: second half of the Newton rounds
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  int* h_counters = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  const double* graph_k = nullptr;
  int64_t graph_ldk = 0, graph_C = 0;
  double graph_t_end = 0.0;   // the captured kernels hold Dev by value, t_end included
  int refresh_ctas = 0;
  RefreshPlan plan{};
  // instrumentation
  int64_t launches = 0, timed = 0;
  double timed_ms = 0.0;
  std::vector<cudaEvent_t> ev_pool;   // pairs recorded by the current group
  size_t ev_used = 0;
  int64_t graph_launches_per_group = 0;
};

extern "C" void sm_opts_default(sm_opts* o) {
  if (!o) return;
  o->rtol = 1e-6;
  o->atol = 1e-20;
  o->gamma_tol = 0.3;
  o->newton_tol = 0.1;
  o->eta_max = 5.0;
  o->eta_keep = 1.5;
  o->q_max = 5;
  o->max_steps = 100000;
  o->j_age_max = 20;
  o->newton_max = 4;
  o->max_conv_fails = 10;
  o->precision = SM_PREC_FP64;
  o->use_graph = 1;
  o->attempts_per_sync = 8;
  o->timing_kind = SM_TIME_NONE;
  o->record_steps = 0;
  o->refresh_ctas_per_sm = 0;
}

namespace {

struct Scope {
  int prev = -1;
  bool ok = true;
  explicit Scope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~Scope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool opts_ok(const sm_opts& o) {
  return o.rtol >= 0.0 && o.atol > 0.0 && o.gamma_tol > 0.0 && o.newton_tol > 0.0 && o.eta_max >= 1.0 &&
         o.eta_keep >= 1.0 && o.q_max >= 1 && o.q_max <= QMAX && o.max_steps >= 1 && o.j_age_max >= 1 &&
         o.newton_max >= 1 && o.newton_max <= 8 && o.max_conv_fails >= 1 &&
         (o.precision == SM_PREC_FP64 || o.precision == SM_PREC_MIXED || o.precision == SM_PREC_TF32) &&
         o.attempts_per_sync >= 1 &&
         o.timing_kind >= SM_TIME_NONE && o.timing_kind <= SM_TIME_FINISH && o.record_steps >= 0 &&
         o.refresh_ctas_per_sm >= 0;
}

void free_state(sm_state* st) {
  if (st->graph) cudaGraphExecDestroy(st->graph);
  for (cudaEvent_t e : st->ev_pool) cudaEventDestroy(e);
  st->ev_pool.clear();
  st->scal_d.release();
  st->scal_i.release();
  st->vec.release();
  st->lu.release();
  st->lup.release();
  st->kslot.release();
  st->cpt.release();
  st->th_par.release();
  st->th_cool.release();
  st->cond.release();
  st->bord.release();
  st->list.release();
  st->counters.release();
  st->scratch.release();
  st->rec_d.release();
  st->rec_i.release();
  st->adj_d.release();
  st->adj_i.release();
  st->adj_lu.release();
  if (st->h_counters) cudaFreeHost(st->h_counters);
  if (st->ev_in) cudaEventDestroy(st->ev_in);
  if (st->ev_out) cudaEventDestroy(st->ev_out);
  if (st->ev_fork) cudaEventDestroy(st->ev_fork);
  if (st->ev_join) cudaEventDestroy(st->ev_join);
  if (st->s2) cudaStreamDestroy(st->s2);
  if (st->s) cudaStreamDestroy(st->s);
}

unsigned blocks(int64_t C, int t) { return (unsigned)((C + t - 1) / t); }

// Event pair around one launch of the timed kernel class (no-op otherwise).
sm_status time_mark(sm_state* st, int kind, bool begin, cudaStream_t s) {
  if (st->opts.timing_kind != kind || kind == SM_TIME_NONE) return SM_OK;
  if (begin && st->ev_used + 2 > st->ev_pool.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      SM_TRY_CUDA(cudaEventCreate(&e));
      st->ev_pool.push_back(e);
    }
  }
  const size_t slot = begin ? st->ev_used : st->ev_used + 1;
  // inside stream capture an external record node keeps the event usable for
  // cudaEventElapsedTime after each graph launch
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SM_TRY_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    SM_TRY_CUDA(cudaEventRecordWithFlags(st->ev_pool[slot], s, cudaEventRecordExternal));
  } else {
    SM_TRY_CUDA(cudaEventRecord(st->ev_pool[slot], s));
  }
  if (!begin) st->ev_used += 2;
  return SM_OK;
}

// Adds the durations of all recorded pairs (call after the stream synced).
void harvest_times(sm_state* st) {
  for (size_t i = 0; i + 1 < st->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, st->ev_pool[i], st->ev_pool[i + 1]) == cudaSuccess) {
      st->timed_ms += ms;
      st->timed += 1;
    } else {
      (void)cudaGetLastError();  // an untimed pair must not poison later calls
    }
  }
}

Dev shift_cells(const Dev& d0, int64_t c0, int64_t Cc);

constexpr int kLaunchesFixed = 3;  // predict, refresh, finish (+3 per Newton round and half)
constexpr int64_t kSplitMin = 2048; // smallest half worth a second stream

template <class T>
sm_status enqueue_attempt(sm_state* st, const double* k, int64_t ldk, cudaStream_t s) {
  Dev& d = st->d;
  const sm_net* net = st->net;
  sm_status r;
  SM_TRY_CUDA(cudaMemsetAsync(d.counters, 0, 2 * sizeof(int), s));
  if ((r = time_mark(st, SM_TIME_PREDICT, true, s)) != SM_OK) return r;
  predict_kernel<<<blocks(d.C, 32), 32 * kCoopWarps, 0, s>>>(d);
  if ((r = time_mark(st, SM_TIME_PREDICT, false, s)) != SM_OK) return r;
  if ((r = time_mark(st, SM_TIME_REFRESH, true, s)) != SM_OK) return r;
  if (d.kslot) {
    k = d.kslot;   // the rate coefficients in slot order
    ldk = d.ld;
  }
  const dim3 th_grid(blocks(d.C, 128), (unsigned)((d.n_r + kThRatesChunk - 1) / kThRatesChunk));
  if (d.therm) {
    // k'(T) at the predicted state, for the refresh and the first Newton round
    th_rates_kernel<<<th_grid, 128, 0, s>>>(d, d.ypred + (int64_t)d.t_idx * d.ld, 0);
    st->launches += 1;
  }
  refresh_kernel<T><<<st->refresh_ctas, kRefreshThreads, st->plan.bytes, s>>>(d, k, ldk, st->plan);
  if (d.therm) {
    const unsigned nb = (unsigned)std::min<int64_t>(blocks(d.C, kBorderWarps), 152LL * 16);
    th_border_kernel<T><<<nb, 32 * kBorderWarps, st->border_smem, s>>>(d);
    st->launches += 1;
  }
  if ((r = time_mark(st, SM_TIME_REFRESH, false, s)) != SM_OK) return r;
  const size_t smem = sizeof(T) * (size_t)kSolveWarps * ((d.n + 3) / 4 * 4);
  // Newton rounds.  Unless the RHS or solve class is being timed, the cells
  // are split into two halves whose rounds run on two streams: the RHS
  // (FP64-pipe bound) of one half overlaps the substitution (bandwidth
  // bound) of the other.
  // (not with compaction: the running cells are then all in the first half)
  const bool split = !d.compact && !d.therm && st->opts.timing_kind != SM_TIME_RHS &&
                     st->opts.timing_kind != SM_TIME_SOLVE && d.C >= 2 * kSplitMin;
  const int64_t ch = split ? (d.C / 2 + 31) / 32 * 32 : d.C;
  if (split) {
    SM_TRY_CUDA(cudaEventRecord(st->ev_fork, s));
    SM_TRY_CUDA(cudaStreamWaitEvent(st->s2, st->ev_fork, 0));
  }
  for (int half = 0; half < (split ? 2 : 1); ++half) {
    const int64_t c0 = half * ch, cn = split ? (half ? d.C - ch : ch) : d.C;
    cudaStream_t hs = half ? st->s2 : s;
    Dev dh = shift_cells(d, c0, cn);
    for (int m = 0; m < d.newton_max; ++m) {
      if ((r = time_mark(st, SM_TIME_RHS, true, hs)) != SM_OK) return r;
      if (d.therm && m > 0) {
        th_rates_kernel<<<dim3(blocks(cn, 128), th_grid.y), 128, 0, hs>>>(dh, dh.y + (int64_t)d.t_idx * d.ld, 0);
        st->launches += 1;
      }
      r = launch_rhs_masked(net, cn, k + c0, ldk, dh.y, dh.f, d.ld, st->scratch.as<double>() + c0, d.ld,
                            dh.flags, F_NEWTON, d.compact ? d.counters + kCAct : nullptr, hs);
      if (r != SM_OK) return r;
      if (d.therm) {
        th_energy_kernel<<<blocks(cn, 128), 128, 0, hs>>>(dh, dh.y, dh.f, 0);
        st->launches += 1;
      }
      if ((r = time_mark(st, SM_TIME_RHS, false, hs)) != SM_OK) return r;
      if ((r = time_mark(st, SM_TIME_SOLVE, true, hs)) != SM_OK) return r;
      solve_update_kernel<T><<<blocks(cn, kSolveWarps), 32 * kSolveWarps, smem, hs>>>(dh, F_NEWTON, F_NEWTON);
      if ((r = time_mark(st, SM_TIME_SOLVE, false, hs)) != SM_OK) return r;
    }
  }
  if (split) {
    SM_TRY_CUDA(cudaEventRecord(st->ev_join, st->s2));
    SM_TRY_CUDA(cudaStreamWaitEvent(s, st->ev_join, 0));
  }
  if ((r = time_mark(st, SM_TIME_FINISH, true, s)) != SM_OK) return r;
  finish_kernel<<<blocks(d.C, 32), 32 * kCoopWarps, 0, s>>>(d);
  if ((r = time_mark(st, SM_TIME_FINISH, false, s)) != SM_OK) return r;
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += kLaunchesFixed + 3 * d.newton_max * (split ? 2 : 1);
  return SM_OK;
}

sm_status enqueue_group(sm_state* st, const double* k, int64_t ldk, int attempts, cudaStream_t s) {
  if (!st->opts.use_graph) st->ev_used = 0;
  for (int a = 0; a < attempts; ++a) {
    sm_status r = st->opts.precision != SM_PREC_FP64 ? enqueue_attempt<float>(st, k, ldk, s)
                                                      : enqueue_attempt<double>(st, k, ldk, s);
    if (r != SM_OK) return r;
  }
  const Dev& d = st->d;
  if (d.compact && attempts > 0) {
    compact_count_kernel<<<blocks(d.C, 256), 256, 0, s>>>(d);
    compact_list_kernel<<<blocks(d.C, 256), 256, 0, s>>>(d);
    compact_swap_kernel<<<1024, 256, 0, s>>>(d);
    compact_commit_kernel<<<1, 32, 0, s>>>(d);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 4;
  }
  return SM_OK;
}

// Runs `attempts` attempts on the state's stream, through a cached CUDA graph
// when enabled (captured once per (k, ldk, C, t_end)).
sm_status run_attempts(sm_state* st, const double* k, int64_t ldk, int attempts) {
  if (!st->opts.use_graph) {
    sm_status r = enqueue_group(st, k, ldk, attempts, st->s);
    if (r == SM_OK && st->opts.timing_kind != SM_TIME_NONE) {
      SM_TRY_CUDA(cudaStreamSynchronize(st->s));
      harvest_times(st);
    }
    return r;
  }
  const int per = st->opts.attempts_per_sync;
  if (!st->graph || st->graph_k != k || st->graph_ldk != ldk || st->graph_C != st->d.C ||
      st->graph_t_end != st->d.t_end) {
    if (st->graph) {
      cudaGraphExecDestroy(st->graph);
      st->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    SM_TRY_CUDA(cudaStreamBeginCapture(st->s, cudaStreamCaptureModeThreadLocal));
    st->ev_used = 0;
    const int64_t before = st->launches;
    sm_status r = enqueue_group(st, k, ldk, per, st->s);
    st->graph_launches_per_group = st->launches - before;
    st->launches = before;
    cudaError_t e = cudaStreamEndCapture(st->s, &g);
    if (r != SM_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    SM_TRY_CUDA(e);
    e = cudaGraphInstantiate(&st->graph, g, 0);
    cudaGraphDestroy(g);
    SM_TRY_CUDA(e);
    st->graph_k = k;
    st->graph_ldk = ldk;
    st->graph_C = st->d.C;
    st->graph_t_end = st->d.t_end;
  }
  for (int done = 0; done < attempts; done += per) {
    if (attempts - done >= per) {
      SM_TRY_CUDA(cudaGraphLaunch(st->graph, st->s));
      st->launches += st->graph_launches_per_group;
    } else {
      // the remainder runs uncaptured; its events would collide with the
      // graph's pairs, so it is not timed
      const int kind = st->opts.timing_kind;
      st->opts.timing_kind = SM_TIME_NONE;
      sm_status r = enqueue_group(st, k, ldk, attempts - done, st->s);
      st->opts.timing_kind = kind;
      if (r != SM_OK) return r;
    }
    if (st->opts.timing_kind != SM_TIME_NONE) {
      SM_TRY_CUDA(cudaStreamSynchronize(st->s));
      harvest_times(st);
    }
  }
  return SM_OK;
}

sm_status running_count(sm_state* st, int64_t* out, int64_t* failed = nullptr) {
  SM_TRY_CUDA(cudaMemsetAsync(st->d.counters + 1, 0, 2 * sizeof(int), st->s));
  count_running_kernel<<<blocks(st->d.C, 256), 256, 0, st->s>>>(st->d);
  st->launches += 1;
  SM_TRY_CUDA(cudaMemcpyAsync(st->h_counters, st->d.counters, 3 * sizeof(int), cudaMemcpyDeviceToHost, st->s));
  SM_TRY_CUDA(cudaStreamSynchronize(st->s));
  *out = st->h_counters[1];
  if (failed) *failed = st->h_counters[2];
  return SM_OK;
}

sm_status join_in(sm_state* st, void* stream) {
  SM_TRY_CUDA(cudaEventRecord(st->ev_in, (cudaStream_t)stream));
  SM_TRY_CUDA(cudaStreamWaitEvent(st->s, st->ev_in, 0));
  return SM_OK;
}

sm_status join_out(sm_state* st, void* stream) {
  SM_TRY_CUDA(cudaEventRecord(st->ev_out, st->s));
  SM_TRY_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, st->ev_out, 0));
  return SM_OK;
}


// The per-cell views of cells [c0, c0 + Cc) as a state of Cc cells.
Dev shift_cells(const Dev& d0, int64_t c0, int64_t Cc) {
  Dev d = d0;
  d.C = Cc;
  auto sh = [c0](auto*& p) {
    if (p) p += c0;
  };
  sh(d.t); sh(d.h); sh(d.gam); sh(d.gam_J); sh(d.crate); sh(d.dprev); sh(d.tn); sh(d.alpha);
  sh(d.q); sh(d.nh); sh(d.n_at_q); sh(d.j_age); sh(d.flags); sh(d.crej); sh(d.ccf); sh(d.status);
  sh(d.m_it); sh(d.steps); sh(d.rejects); sh(d.conv_fails); sh(d.newton_iters); sh(d.jac_evals); sh(d.slot_cell);
  sh(d.Y); sh(d.ypred); sh(d.y); sh(d.psi); sh(d.f); sh(d.f0); sh(d.eprev); sh(d.w); sh(d.wf);
  sh(d.log_t); sh(d.log_h); sh(d.log_q); sh(d.ck_Y); sh(d.ck_t); sh(d.ck_nh);
  return d;
}

// Views of the pass [c0, c0 + Cp) for the reverse sweep and the replay: the
// state shifted to the pass, Newton set to the replay tolerance, and the
// adjoint workspace carved up.  Runs the per-cell set-up and returns the
// largest segment count and step count of the pass.
sm_status adj_prepare(sm_state* st, int64_t c0, int64_t Cp, int64_t lda, const double* k, int64_t ldk,
                      const double* cot, int n_cot, Dev* dd_out, AdjDev* a_out, int* Kmax, int* Nmax) {
  const int n = st->d.n, n_r = st->d.n_r;
  cudaStream_t s = st->s;
  Dev dd = shift_cells(st->d, c0, Cp);
  dd.lup = nullptr;   // the replay factorises into dense per-cell storage
  dd.lu_cta = 0;
  dd.mixed = 0;
  dd.newton_tol = kReplayTol;
  dd.newton_max = kReplayIters;
  double* ad = st->adj_d.as<double>();
  int* ai = st->adj_i.as<int>();
  dd.jac_evals = ai + (4 + kCkpt + kRing) * lda;   // replay counters stay out of the run's statistics
  dd.newton_iters = dd.jac_evals + lda;
  AdjDev a{};
  a.n_cot = n_cot;
  a.run_tol = st->d.newton_tol;
  a.lda = lda;
  a.N = ai; a.K = ai + lda; a.seg = ai + 2 * lda; a.astat = ai + 3 * lda;
  a.seg_q = ai + 4 * lda; a.ring_q = a.seg_q + kCkpt * lda;
  a.seg_y = ad;
  a.seg_h = a.seg_y + (int64_t)kCkpt * n * lda;
  a.seg_alpha = a.seg_h + kCkpt * lda;
  a.ring_alpha = a.seg_alpha + (int64_t)kCkpt * (QMAX + 1) * lda;
  a.lam = a.ring_alpha + (int64_t)kRing * (QMAX + 1) * lda;
  a.kc = a.lam + (int64_t)kRing * n_cot * n * lda;
  a.g = a.kc + Cp * n_r;
  a.slots = st->adj_lu.as<double>();
  a.cot = cot ? cot + c0 : nullptr;
  a.ldu = ldk;
  SM_TRY_CUDA(cudaMemsetAsync(dd.counters, 0, 4 * sizeof(int), s));
  adj_setup_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, k + c0, ldk);
  SM_TRY_CUDA(cudaGetLastError());
  SM_TRY_CUDA(cudaMemcpyAsync(st->h_counters, dd.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  SM_TRY_CUDA(cudaStreamSynchronize(s));
  st->launches += 1;
  *Kmax = st->h_counters[3];
  *Nmax = st->h_counters[1];
  *dd_out = dd;
  *a_out = a;
  return SM_OK;
}

// Number of cells without a usable result (counters[2], set by the output
// kernels), added to *bad.
sm_status adj_count_bad(sm_state* st, int64_t* bad) {
  SM_TRY_CUDA(cudaMemcpyAsync(st->h_counters, st->d.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, st->s));
  SM_TRY_CUDA(cudaStreamSynchronize(st->s));
  *bad += st->h_counters[2];
  return SM_OK;
}

// One pass of the reverse sweep over cells [c0, c0 + Cp); adds the number of
// cells without a usable result to *bad.
sm_status adjoint_pass(sm_state* st, int64_t c0, int64_t Cp, int64_t lda, const double* k, int64_t ldk,
                       const double* cot, int n_cot, double* grad, double* grad_y0, int32_t* astat, int warps,
                       size_t smem, int64_t* bad) {
  const sm_net* net = st->net;
  cudaStream_t s = st->s;
  Dev dd;
  AdjDev a;
  int Kmax = 0, Nmax = 0;
  sm_status r = adj_prepare(st, c0, Cp, lda, k, ldk, cot, n_cot, &dd, &a, &Kmax, &Nmax);
  if (r != SM_OK) return r;
  const double* kp = k + c0;
  double* scratch = st->scratch.as<double>() + c0;
  auto slot_dev = [&](int j) {
    Dev x = dd;
    x.lu = a.slots + (int64_t)j * Cp * dd.lu_stride;
    return x;
  };
  auto refresh_at = [&](int j, int need_flag) -> sm_status {
    SM_TRY_CUDA(cudaMemsetAsync(dd.counters, 0, sizeof(int), s));
    adj_list_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, need_flag);
    refresh_kernel<double><<<st->refresh_ctas, kRefreshThreads, st->plan.bytes, s>>>(slot_dev(j), kp, ldk, st->plan);
    st->launches += 2;
    return SM_OK;
  };
  const size_t solve_smem = sizeof(double) * (size_t)kSolveWarps * ((dd.n + 3) / 4 * 4);
  for (int rs = 0; rs < Kmax; ++rs) {
    seg_restore_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, rs);
    st->launches += 1;
    for (int j = 0; j < kCkpt; ++j) {
      rpredict_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, 1);
      st->launches += 1;
      // Newton matrix: the factors at y_{m-1} (slot j - 1), or, for the cells
      // flagged F_REFRESH, fresh ones at the predictor in slot j (replaced by
      // the factors at y_m once the step is solved)
      const Dev d_old = slot_dev(j > 0 ? j - 1 : 0), d_new = slot_dev(j);
      const int need = F_NEWTON | F_REFRESH;
      for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
          rretry_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j);
          st->launches += 1;
        }
        if ((r = refresh_at(j, need)) != SM_OK) return r;
        for (int it = 0; it < kReplayIters; ++it) {
          r = launch_rhs_masked(net, Cp, kp, ldk, dd.y, dd.f, dd.ld, scratch, dd.ld, dd.flags, F_NEWTON, nullptr, s);
          if (r != SM_OK) return r;
          if (j > 0 && attempt == 0) {
            solve_update_kernel<double><<<blocks(Cp, kSolveWarps), 32 * kSolveWarps, solve_smem, s>>>(d_old, need, F_NEWTON);
            st->launches += 1;
          }
          solve_update_kernel<double><<<blocks(Cp, kSolveWarps), 32 * kSolveWarps, solve_smem, s>>>(d_new, need, need);
          st->launches += 3;
        }
      }
      rcommit_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, 1);
      st->launches += 1;
      if ((r = refresh_at(j, 0)) != SM_OK) return r;
    }
    for (int j = kCkpt - 1; j >= 0; --j) {
      adj_step_kernel<<<(unsigned)Cp, 32 * warps, smem, s>>>(dd, a, j);
      st->launches += 1;
    }
    SM_TRY_CUDA(cudaGetLastError());
  }
  SM_TRY_CUDA(cudaMemsetAsync(dd.counters + 2, 0, sizeof(int), s));
  adj_out_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, grad + c0, ldk, astat ? astat + c0 : nullptr);
  st->launches += 1;
  if (grad_y0) {
    adj_y0_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, grad_y0 + c0, ldk);
    st->launches += 1;
  }
  SM_TRY_CUDA(cudaGetLastError());
  return adj_count_bad(st, bad);
}

// One pass of the frozen-step replay over cells [c0, c0 + Cp): the recorded
// steps re-solved from the recorded initial state with rate coefficients k,
// the Newton matrix refreshed by the gamma rule and every kCkpt steps, in the
// state's own factor storage.
sm_status replay_pass(sm_state* st, int64_t c0, int64_t Cp, int64_t lda, const double* k, int64_t ldk,
                      double* y, int32_t* astat, int64_t* bad) {
  const sm_net* net = st->net;
  cudaStream_t s = st->s;
  Dev dd;
  AdjDev a;
  int Kmax = 0, Nmax = 0;
  sm_status r = adj_prepare(st, c0, Cp, lda, k, ldk, nullptr, 0, &dd, &a, &Kmax, &Nmax);
  if (r != SM_OK) return r;
  const double* kp = k + c0;
  double* scratch = st->scratch.as<double>() + c0;
  const size_t solve_smem = sizeof(double) * (size_t)kSolveWarps * ((dd.n + 3) / 4 * 4);
  seg_restore_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, -1);
  st->launches += 1;
  for (int j = 0; j < Nmax; ++j) {
    rpredict_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, 0);
    st->launches += 1;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (attempt == 1) {
        rretry_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j);
        st->launches += 1;
      }
      SM_TRY_CUDA(cudaMemsetAsync(dd.counters, 0, sizeof(int), s));
      adj_list_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, F_NEWTON | F_REFRESH);
      refresh_kernel<double><<<st->refresh_ctas, kRefreshThreads, st->plan.bytes, s>>>(dd, kp, ldk, st->plan);
      st->launches += 2;
      for (int it = 0; it < kReplayIters; ++it) {
        r = launch_rhs_masked(net, Cp, kp, ldk, dd.y, dd.f, dd.ld, scratch, dd.ld, dd.flags, F_NEWTON, nullptr, s);
        if (r != SM_OK) return r;
        solve_update_kernel<double><<<blocks(Cp, kSolveWarps), 32 * kSolveWarps, solve_smem, s>>>(dd, F_NEWTON, F_NEWTON);
        st->launches += 3;
      }
    }
    rcommit_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, j, 0);
    st->launches += 1;
    SM_TRY_CUDA(cudaGetLastError());
  }
  SM_TRY_CUDA(cudaMemsetAsync(dd.counters + 2, 0, sizeof(int), s));
  replay_out_kernel<<<blocks(Cp, 128), 128, 0, s>>>(dd, a, y + c0, ldk, astat ? astat + c0 : nullptr);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 1;
  return adj_count_bad(st, bad);
}

// Workspace of the reverse sweep / replay for passes of Cc cells.
sm_status adj_workspace(sm_state* st, int64_t Cc, int64_t lda, int n_cot) {
  const int n = st->d.n, n_r = st->d.n_r;
  const size_t nd = (size_t)kCkpt * n * lda + (size_t)kCkpt * lda + (size_t)kCkpt * (QMAX + 1) * lda +
                    (size_t)kRing * (QMAX + 1) * lda + (size_t)kRing * n_cot * n * lda + (size_t)Cc * n_r +
                    (size_t)Cc * n_cot * n_r;
  const size_t ni = (size_t)(4 + kCkpt + kRing + 2) * lda;
  sm_status r;
  if ((r = st->adj_d.ensure(sizeof(double) * nd)) != SM_OK) return r;
  if ((r = st->adj_i.ensure(sizeof(int) * ni)) != SM_OK) return r;
  return SM_OK;
}

// Cells per pass: all (0), or the request rounded up to a multiple of 32 so
// that every pass starts on a 32-cell boundary.
int64_t pass_cells(int64_t C, int64_t cells_per_pass) {
  int64_t Cc = cells_per_pass > 0 ? std::min<int64_t>(cells_per_pass, C) : C;
  if (Cc < C) Cc = std::min<int64_t>(C, (Cc + 31) / 32 * 32);
  return Cc;
}

}  // namespace

extern "C" {

sm_status sm_state_create(const sm_net* net, int64_t C, const sm_opts* opts, sm_state** out) {
  if (!out) return SM_EINVAL;
  *out = nullptr;
  if (!net || net->device < 0 || C < 1) return SM_EINVAL;
  sm_opts o;
  sm_opts_default(&o);
  if (opts) o = *opts;
  if (!opts_ok(o)) return SM_EINVAL;
  Scope scope(net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_state* st = new (std::nothrow) sm_state();
  if (!st) return SM_ENOMEM;
  st->net = net;
  st->opts = o;
  st->cap = C;
  st->ld = (C + 31) / 32 * 32;
  const int64_t ld = st->ld;
  const int n = net->n_s;
  const LUSymbolic& lu = net->lu;
  Dev& d = st->d;
  d.n = n;
  d.n_r = net->n_r;
  d.nnz_j = (int)net->jp_col.size();
  d.mixed = o.precision != SM_PREC_FP64;
  d.tf32 = o.precision == SM_PREC_TF32;
  d.C = C;
  d.ld = ld;
  d.rtol = o.rtol;
  d.atol = o.atol;
  d.gamma_tol = o.gamma_tol;
  d.newton_tol = o.newton_tol;
  d.eta_max = o.eta_max;
  d.eta_keep = o.eta_keep;
  d.q_max = o.q_max;
  d.max_steps = o.max_steps;
  d.j_age_max = o.j_age_max;
  d.newton_max = o.newton_max;
  d.max_conv_fails = o.max_conv_fails;
  d.ldm = lu.ld;
  d.head = lu.head;
  sm_status r = SM_OK;
  auto fail = [&](sm_status e) {
    free_state(st);
    delete st;
    return e;
  };
  const int n_dscal = 6 + 2 * (QMAX + 1);   // t h gam gam_J crate dprev | tn[6] alpha[6]
  const int n_iscal = 15;                   // q nh n_at_q j_age flags crej ccf status m_it steps rejects
                                            // conv_fails newton_iters jac_evals slot_cell
  const int n_vec = (QMAX + 1) + 8;         // Y[6] ypred y psi f f0 eprev w wf
  if ((r = st->scal_d.ensure(sizeof(double) * n_dscal * ld)) != SM_OK) return fail(r);
  if ((r = st->scal_i.ensure(sizeof(int) * n_iscal * ld)) != SM_OK) return fail(r);
  if ((r = st->vec.ensure(sizeof(double) * (size_t)n_vec * n * ld)) != SM_OK) return fail(r);
  const size_t esz = d.mixed ? sizeof(float) : sizeof(double);
  d.lu_stride = (int64_t)n * lu.ld;
  d.lup_stride = lu.p_size;
  if ((r = st->lup.ensure(esz * (size_t)d.lup_stride * C)) != SM_OK) return fail(r);
  if ((r = st->list.ensure(sizeof(int) * ld)) != SM_OK) return fail(r);
  if ((r = st->counters.ensure(sizeof(int) * kCounters)) != SM_OK) return fail(r);
  // compaction of running cells in states that record no steps (the
  // adjoint's records are indexed by cell)
  d.compact = o.record_steps > 0 ? 0 : 1;
  // slot-ordered rate coefficients: with compaction, and always with a
  // coupled temperature (its k'(T) is rewritten before every right-hand side)
  if (d.compact || net->th_t >= 0) {
    if ((r = st->kslot.ensure(sizeof(double) * (size_t)net->n_r * ld)) != SM_OK) return fail(r);
  }
  if (d.compact) {
    if ((r = st->cpt.ensure(sizeof(int) * 2 * (size_t)ld)) != SM_OK) return fail(r);
  }
  if ((r = st->scratch.ensure(sizeof(double) * (size_t)net->n_r * ld)) != SM_OK) return fail(r);
  double* ds = st->scal_d.as<double>();
  d.t = ds; d.h = ds + ld; d.gam = ds + 2 * ld; d.gam_J = ds + 3 * ld; d.crate = ds + 4 * ld;
  d.dprev = ds + 5 * ld; d.tn = ds + 6 * ld; d.alpha = ds + (6 + QMAX + 1) * ld;
  int* is = st->scal_i.as<int>();
  d.q = is; d.nh = is + ld; d.n_at_q = is + 2 * ld; d.j_age = is + 3 * ld; d.flags = is + 4 * ld;
  d.crej = is + 5 * ld; d.ccf = is + 6 * ld; d.status = is + 7 * ld; d.m_it = is + 8 * ld;
  d.steps = is + 9 * ld; d.rejects = is + 10 * ld; d.conv_fails = is + 11 * ld;
  d.newton_iters = is + 12 * ld; d.jac_evals = is + 13 * ld; d.slot_cell = is + 14 * ld;
  double* v = st->vec.as<double>();
  const int64_t vs = (int64_t)n * ld;
  d.Y = v; d.ypred = v + (QMAX + 1) * vs; d.y = d.ypred + vs; d.psi = d.y + vs; d.f = d.psi + vs;
  d.f0 = d.f + vs; d.eprev = d.f0 + vs; d.w = d.eprev + vs; d.wf = d.w + vs;
  d.list = st->list.as<int>();
  d.counters = st->counters.as<int>();
  d.kslot = st->kslot.p ? st->kslot.as<double>() : nullptr;
  d.holes = d.compact ? st->cpt.as<int>() : nullptr;
  d.runners = d.compact ? st->cpt.as<int>() + ld : nullptr;
  d.lu = st->lu.p;
  d.lup = st->lup.p;
  d.p_l11 = lu.p_l11; d.p_u11 = lu.p_u11; d.p_dinv = lu.p_dinv; d.p_l21 = lu.p_l21; d.p_u12 = lu.p_u12;
  d.p_d = lu.p_d; d.ldd = lu.ldd;
  d.n_flev = (int)lu.flev_ptr.size() - 1; d.n_blev = (int)lu.blev_ptr.size() - 1;
  d.u11ptr = lu.d_u11ptr.as<int>(); d.flev_ptr = lu.d_flev_ptr.as<int>(); d.flev = lu.d_flev.as<int>();
  d.blev_ptr = lu.d_blev_ptr.as<int>(); d.blev = lu.d_blev.as<int>();
  d.hop_ptr = lu.d_hop_ptr.as<int>(); d.hop_piv = lu.d_hop_piv.as<int>(); d.hop = lu.d_hop.as<int4>();
  d.hterm = lu.d_hterm.as<int2>(); d.n_hlev = lu.n_hlev;
  d.perm = lu.d_perm.as<int>(); d.iperm = lu.d_iperm.as<int>();
  d.lptr = lu.d_lptr.as<int>(); d.lidx = lu.d_lidx.as<int>();
  d.uptr = lu.d_uptr.as<int>(); d.uidx = lu.d_uidx.as<int>();
  d.lrptr = lu.d_lrptr.as<int>(); d.lridx = lu.d_lridx.as<int>();
  d.ucptr = lu.d_ucptr.as<int>(); d.ucidx = lu.d_ucidx.as<int>();
  d.jrc = lu.d_jrc.as<int>(); d.uoff = lu.d_uoff.as<int>(); d.lrhead = lu.d_lrhead.as<int>();
  d.lrhoff = lu.d_lrhoff.as<int>();
  d.u12off = lu.d_u12off.as<int>();
  d.lrhk = lu.d_lrhk.as<int>();
  d.srow = lu.d_srow.as<int>();
  d.n_srow = (int)lu.srow.size();
  d.jt_slot = net->d_jt_slot.as<int2>(); d.reac = net->d_reac.as<int2>();
  d.sc_ptr = net->d_sc_ptr.as<int>(); d.sc_ent = net->d_sc_ent.as<uint32_t>();
  d.jdesc = net->d_jdesc.as<int4>(); d.jlong = net->d_jlong.as<int>(); d.n_jlong = (int)net->jlong.size();
  d.jp_ptr = net->d_jp_ptr.as<int>(); d.jt_ptr = net->d_jt_ptr.as<int>();
  d.jt_word = net->d_jt_word.as<int2>(); d.jpos = lu.d_jpos.as<int>();
  d.record = o.record_steps > 0 ? o.record_steps : 0;
  if (d.record) {
    const int64_t R = d.record, K = R / kCkpt + 1;
    if ((r = st->rec_d.ensure(sizeof(double) * (size_t)(2 * R * ld + K * (QMAX + 1) * (int64_t)n * ld +
                                                        K * (QMAX + 1) * ld))) != SM_OK)
      return fail(r);
    if ((r = st->rec_i.ensure(sizeof(int) * (size_t)(R * ld + K * ld))) != SM_OK) return fail(r);
    double* rd = st->rec_d.as<double>();
    d.log_t = rd;
    d.log_h = rd + R * ld;
    d.ck_Y = rd + 2 * R * ld;
    d.ck_t = d.ck_Y + K * (QMAX + 1) * (int64_t)n * ld;
    int* ri = st->rec_i.as<int>();
    d.log_q = ri;
    d.ck_nh = ri + R * ld;
  }
  if (cudaStreamCreateWithFlags(&st->s, cudaStreamNonBlocking) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaStreamCreateWithFlags(&st->s2, cudaStreamNonBlocking) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaMallocHost(&st->h_counters, kCounters * sizeof(int)) != cudaSuccess) return fail(SM_ENOMEM);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device);
  {
    // shared memory of the refresh kernel: the largest of its three phases
    RefreshPlan& pl = st->plan;
    const int nt = n - lu.head;
    // rows past the panel height: zero padding for 4-wide loads; both pitches
    // are 8 mod 32 words so that the tensor-core fragment loads (4 k-rows x 8
    // columns per instruction) fall in 32 distinct banks
    pl.pitch = round_up(nt + 4, 4);
    while (pl.pitch % 32 != 8) pl.pitch += 4;
    pl.n_panels = (nt + kNB - 1) / kNB;
    pl.upitch = round_up(std::max(nt - kNB, 4), 4);
    while (pl.upitch % 32 != 8) pl.upitch += 4;
    const size_t tail = esz * (size_t)kNB * (pl.pitch + pl.upitch);
    const size_t stage = sizeof(double) * (2 * (size_t)net->n_r + 256) + sizeof(float) * 2 * (size_t)n;
    // phases B and S: the packed head factors H after the Schur pass's U12
    // panel tiles (kPS panels of h x kNB)
    const size_t ut = esz * (size_t)lu.head * kNB * std::min(kPS, pl.n_panels);
    pl.hv_off = (int)((ut + 15) / 16 * 16);
    pl.n_l21 = lu.lrhoff.empty() ? 0 : lu.lrhoff.back();
    pl.n_u12 = lu.u12off.empty() ? 0 : lu.u12off.back();
    pl.ix_off = (int)((pl.hv_off + esz * (size_t)lu.p_d + 15) / 16 * 16);
    const size_t head_b = (size_t)pl.ix_off + 4 * (size_t)((pl.n_l21 + pl.n_u12 + 1) / 2) +
                          sizeof(int) * (size_t)lu.head * (pl.n_panels + 1);
    pl.head_smem = lu.head > 0 && head_b <= (size_t)smem_max && n - lu.head < 65536;
    pl.bytes = std::max(tail, stage);
    if (pl.head_smem) pl.bytes = std::max(pl.bytes, head_b);
  }
  const size_t rsm = st->plan.bytes;

  if ((int64_t)rsm > smem_max) return fail(SM_ENOTSUP);
  // the attribute is a per-kernel cap shared by every state: set it to the
  // device limit so that a later state with a smaller plan cannot lower it
  // below what an earlier state launches with
  if (d.mixed) {
    SM_TRY_CUDA(cudaFuncSetAttribute(refresh_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  } else {
    SM_TRY_CUDA(cudaFuncSetAttribute(refresh_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  }
  int per_sm = 0;
  if (d.mixed) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refresh_kernel<float>, kRefreshThreads, rsm);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refresh_kernel<double>, kRefreshThreads, rsm);
  }
  if (o.refresh_ctas_per_sm > 0) per_sm = std::min(per_sm, (int)o.refresh_ctas_per_sm);
  st->refresh_ctas = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  // dense working matrices of the refresh: one per refresh CTA, except in
  // recording states, whose replays keep dense factors per cell
  d.lu_cta = d.record ? 0 : 1;
  if ((r = st->lu.ensure(esz * (size_t)d.lu_stride * (d.lu_cta ? st->refresh_ctas : C))) != SM_OK) return fail(r);
  d.lu = st->lu.p;
  // coupled temperature: a copy of the network's setting
  d.therm = 0;
  d.t_idx = -1;
  if (net->th_t >= 0) {
    d.therm = 1;
    d.t_idx = net->th_t;
    d.th_heat = net->th_heat;
    d.th_lam = net->th_lam;
    d.th_Td = net->th_Td;
    d.th_zeta = net->th_zeta;
    d.rpar = net->d_rate.as<RatePar>();
    std::vector<double> par(2 * (size_t)n + net->n_r);
    std::vector<int> cool;
    for (int i = 0; i < n; ++i) {
      par[i] = net->th_L[i];
      par[n + i] = net->th_E[i];
      if (net->th_L[i] > 0.0) cool.push_back(i);
    }
    for (int j = 0; j < net->n_r; ++j) {   // sum_i S_ij: products minus reactants
      int dn = 0;
      for (int q = 0; q < 2; ++q) dn -= net->reac[2 * j + q] >= 0 ? 1 : 0;
      for (int q = 0; q < 4; ++q) dn += net->prod[4 * j + q] >= 0 ? 1 : 0;
      par[2 * n + j] = dn;
    }
    if ((r = st->th_par.upload(par.data(), par.size() * sizeof(double))) != SM_OK) return fail(r);
    d.th_L = st->th_par.as<double>();
    d.th_E = d.th_L + n;
    d.th_dn = d.th_L + 2 * n;
    d.n_cool = (int)cool.size();
    if (!cool.empty() && (r = st->th_cool.upload(cool.data(), cool.size() * sizeof(int))) != SM_OK) return fail(r);
    d.th_cool = st->th_cool.as<int>();
    if ((r = st->cond.ensure(sizeof(double) * 3 * (size_t)ld)) != SM_OK) return fail(r);
    d.c_nH = st->cond.as<double>();
    d.c_Av = d.c_nH + ld;
    d.c_chi = d.c_nH + 2 * ld;
    d.bpad = (n + 3) / 4 * 4;
    if ((r = st->bord.ensure(sizeof(double) * (2 * (size_t)d.bpad + 1) * ld)) != SM_OK) return fail(r);
    d.bz = st->bord.as<double>();
    d.bgv = d.bz + (int64_t)d.bpad * ld;
    d.bs = d.bgv + (int64_t)d.bpad * ld;
    const int xs = (n + 3) / 4 * 4;
    st->border_smem = (size_t)kBorderWarps * xs * (3 * sizeof(double) + esz);
    if (st->border_smem > 48 * 1024) {
      const cudaError_t e =
          d.mixed ? cudaFuncSetAttribute(th_border_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)st->border_smem)
                  : cudaFuncSetAttribute(th_border_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)st->border_smem);
      if (e != cudaSuccess) return fail(SM_ECUDA);
    }
  }
  SM_TRY_CUDA(cudaMemset(st->scal_i.p, 0, st->scal_i.bytes));
  *out = st;
  return SM_OK;
}

sm_status sm_state_free(sm_state* st) {
  if (!st) return SM_EINVAL;
  Scope scope(st->net->device);
  free_state(st);
  delete st;
  return SM_OK;
}

sm_status sm_state_bytes(const sm_state* st, size_t* bytes) {
  if (!st || !bytes) return SM_EINVAL;
  *bytes = st->th_par.bytes + st->th_cool.bytes + st->cond.bytes + st->bord.bytes +
           st->scal_d.bytes + st->scal_i.bytes + st->vec.bytes + st->lu.bytes + st->lup.bytes + st->kslot.bytes +
           st->cpt.bytes + st->list.bytes +
           st->counters.bytes + st->scratch.bytes + st->rec_d.bytes + st->rec_i.bytes + st->adj_d.bytes + st->adj_i.bytes +
           st->adj_lu.bytes;
  return SM_OK;
}

sm_status sm_state_init(sm_state* st, int64_t C, const double* d_k, const double* d_y, int64_t ld,
                        double t_end, void* stream) {
  const bool therm = st && st->d.therm;
  if (!st || C < 1 || C > st->cap || !ld_ok(C, ld) || (!d_k && !therm) || !d_y || !(t_end > 0.0)) return SM_EINVAL;
  if (therm && st->cells_set < C) return SM_EINVAL;   // sm_state_set_cells first
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  st->C = C;
  st->t_end = t_end;
  Dev& d = st->d;
  d.C = C;
  d.t_end = t_end;
  if (therm) d_k = nullptr;
  init_copy_kernel<<<blocks(C, 128), 128, 0, st->s>>>(d, d_y, ld, d_k, ld);
  SM_TRY_CUDA(cudaGetLastError());
  st->kslot_src = d_k;
  if (therm) {
    // every rate coefficient from the initial T (slot order = cell order here)
    th_rates_kernel<<<dim3(blocks(C, 128), (unsigned)((d.n_r + kThRatesChunk - 1) / kThRatesChunk)), 128, 0,
                      st->s>>>(d, d.Y + (int64_t)d.t_idx * d.ld, 1);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 1;
  }
  r = launch_rhs_masked(st->net, C, therm ? d.kslot : d_k, therm ? d.ld : ld, d.Y, d.f0, d.ld,
                        st->scratch.as<double>(), d.ld, d.flags, F_NEWTON, nullptr, st->s);
  if (r != SM_OK) return r;
  if (therm) {
    th_energy_kernel<<<blocks(C, 128), 128, 0, st->s>>>(d, d.Y, d.f0, 1);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 1;
  }
  init_finish_kernel<<<blocks(C, 128), 128, 0, st->s>>>(d);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 4;
  return join_out(st, stream);
}

sm_status sm_step_bdf(sm_state* st, const double* d_k, int64_t ld, int32_t attempts, void* stream) {
  if (!st || (!d_k && !st->d.therm) || st->C < 1 || (!st->d.therm && !ld_ok(st->C, ld)) || attempts < 0)
    return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  if (st->d.therm) {
    d_k = nullptr;   // k' comes from the state's temperatures
    ld = st->d.ld;
  } else if (st->d.kslot && st->kslot_src != d_k) {
    kslot_gather_kernel<<<blocks(st->C, 128), 128, 0, st->s>>>(st->d, d_k, ld);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 1;
    st->kslot_src = d_k;
  }
  if ((r = run_attempts(st, d_k, ld, attempts)) != SM_OK) return r;
  return join_out(st, stream);
}

sm_status sm_state_read(sm_state* st, double* d_y, int64_t ld, sm_cell_stats* d_stats,
                        int64_t* h_running, void* stream) {
  if (!st || st->C < 1 || (d_y && !ld_ok(st->C, ld))) return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  if (d_y || d_stats) {
    read_kernel<<<blocks(st->C, 128), 128, 0, st->s>>>(st->d, d_y, ld, d_stats);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 1;
  }
  if (h_running && (r = running_count(st, h_running)) != SM_OK) return r;
  return join_out(st, stream);
}

sm_status sm_state_set_cells(sm_state* st, int64_t C, const double* d_nH, const double* d_Av, const double* d_chi,
                             void* stream) {
  if (!st || C < 1 || C > st->cap || !d_nH || !d_Av) return SM_EINVAL;
  if (!st->d.therm) return SM_ENOTSUP;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  th_cells_kernel<<<blocks(C, 128), 128, 0, st->s>>>(st->d, C, d_nH, d_Av, d_chi);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 1;
  st->cells_set = C;
  return join_out(st, stream);
}

sm_status sm_integrate(sm_state* st, int64_t C, const double* d_k, double* d_y, int64_t ld,
                       double t_end, sm_cell_stats* d_stats, void* stream) {
  sm_status r = sm_state_init(st, C, d_k, d_y, ld, t_end, stream);
  if (r != SM_OK) return r;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  const int per = st->opts.attempts_per_sync;
  // every attempt either accepts a step, shrinks h or counts a failure, so
  // this cap is never the binding limit for a well-posed problem
  const int64_t max_attempts = 20LL * st->opts.max_steps + 1000;
  int64_t running = 1;
  for (int64_t a = 0; a < max_attempts && running > 0; a += per) {
    if ((r = run_attempts(st, d_k, ld, per)) != SM_OK) return r;
    if ((r = running_count(st, &running)) != SM_OK) return r;
  }
  read_kernel<<<blocks(C, 128), 128, 0, st->s>>>(st->d, d_y, ld, d_stats);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 1;
  int64_t failed = 0;
  if ((r = running_count(st, &running, &failed)) != SM_OK) return r;
  if ((r = join_out(st, stream)) != SM_OK) return r;
  // a cell that did not reach t_end makes the call partial
  return (running > 0 || failed > 0) ? SM_EPARTIAL : SM_OK;
}

sm_status sm_state_steps(sm_state* st, int32_t m_max, double* d_t, double* d_h, int32_t* d_q, int64_t ld,
                         void* stream) {
  if (!st || st->C < 1 || m_max < 1 || m_max > st->d.record || !ld_ok(st->C, ld) || !d_t || !d_h || !d_q)
    return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  const Dev& d = st->d;
  SM_TRY_CUDA(cudaMemcpy2DAsync(d_t, ld * sizeof(double), d.log_t, d.ld * sizeof(double), st->C * sizeof(double),
                                m_max, cudaMemcpyDeviceToDevice, st->s));
  SM_TRY_CUDA(cudaMemcpy2DAsync(d_h, ld * sizeof(double), d.log_h, d.ld * sizeof(double), st->C * sizeof(double),
                                m_max, cudaMemcpyDeviceToDevice, st->s));
  SM_TRY_CUDA(cudaMemcpy2DAsync(d_q, ld * sizeof(int32_t), d.log_q, d.ld * sizeof(int), st->C * sizeof(int32_t),
                                m_max, cudaMemcpyDeviceToDevice, st->s));
  return join_out(st, stream);
}

sm_status sm_adjoint(sm_state* st, const double* d_k, int64_t ld, const double* d_cot, int32_t n_cot,
                     double* d_grad, double* d_grad_y0, int32_t* d_astat, int64_t cells_per_pass,
                     void* stream) {
  if (st && st->d.therm) return SM_ENOTSUP;   // the coupled-temperature adjoint is not built
  if (!st || !d_k || !d_cot || !d_grad || n_cot < 1 || n_cot > SM_ADJ_MAX_COT || st->C < 1 ||
      !ld_ok(st->C, ld) || cells_per_pass < 0 || st->d.record < 1)
    return SM_EINVAL;
  if (st->d.mixed) return SM_ENOTSUP;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  const int64_t C = st->C;
  const int n = st->d.n, n_r = st->d.n_r;
  const int64_t Cc = pass_cells(C, cells_per_pass);
  const int64_t lda = (Cc + 31) / 32 * 32;
  if ((r = adj_workspace(st, Cc, lda, n_cot)) != SM_OK) return r;
  if ((r = st->adj_lu.ensure(sizeof(double) * (size_t)kCkpt * Cc * st->d.lu_stride)) != SM_OK) return r;
  const int warps = std::min(n_cot, 8);
  const size_t smem = sizeof(double) * ((size_t)n_r + (size_t)warps * 2 * n);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->net->device);
  if (smem > (size_t)smem_max) return SM_ENOTSUP;
  SM_TRY_CUDA(cudaFuncSetAttribute(adj_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  if ((r = join_in(st, stream)) != SM_OK) return r;
  int64_t bad = 0;
  for (int64_t c0 = 0; c0 < C; c0 += Cc) {
    const int64_t Cp = std::min(Cc, C - c0);
    r = adjoint_pass(st, c0, Cp, lda, d_k, ld, d_cot, n_cot, d_grad, d_grad_y0, d_astat, warps, smem, &bad);
    if (r != SM_OK) return r;
  }
  if ((r = join_out(st, stream)) != SM_OK) return r;
  return bad > 0 ? SM_EPARTIAL : SM_OK;
}

sm_status sm_replay(sm_state* st, const double* d_k, int64_t ld, double* d_y, int32_t* d_astat,
                    int64_t cells_per_pass, void* stream) {
  if (st && st->d.therm) return SM_ENOTSUP;
  if (!st || !d_k || !d_y || st->C < 1 || !ld_ok(st->C, ld) || cells_per_pass < 0 || st->d.record < 1)
    return SM_EINVAL;
  if (st->d.mixed) return SM_ENOTSUP;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  const int64_t C = st->C;
  const int64_t Cc = pass_cells(C, cells_per_pass);
  const int64_t lda = (Cc + 31) / 32 * 32;
  if ((r = adj_workspace(st, Cc, lda, 0)) != SM_OK) return r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  int64_t bad = 0;
  for (int64_t c0 = 0; c0 < C; c0 += Cc) {
    r = replay_pass(st, c0, std::min(Cc, C - c0), lda, d_k, ld, d_y, d_astat, &bad);
    if (r != SM_OK) return r;
  }
  if ((r = join_out(st, stream)) != SM_OK) return r;
  return bad > 0 ? SM_EPARTIAL : SM_OK;
}

}  // extern "C"

namespace {

// Image of a state: this header, then the raw bytes of the per-cell scalars,
// the history and working vectors, the step records, and (optionally) the
// Newton factors, in that order.
struct StateImage {
  uint64_t magic;
  int32_t version, n_s, n_r, precision;
  int64_t cap, ld, C, lu_stride;
  double t_end;
  int32_t record, with_factors;
  uint64_t bytes[5];   // scal_d, scal_i, vec, rec_d + rec_i, lu
};
constexpr uint64_t kImageMagic = 0x534D5354415445ull;   // "SMSTATE"

void image_sizes(const sm_state* st, int with_factors, uint64_t* b) {
  b[0] = st->scal_d.bytes;
  b[1] = st->scal_i.bytes;
  b[2] = st->vec.bytes;
  b[3] = st->rec_d.bytes + st->rec_i.bytes;
  // the packed factors, and in recording states the dense per-cell ones
  b[4] = with_factors ? st->lup.bytes + (st->d.lu_cta ? 0 : st->lu.bytes) : 0;
}

}  // namespace

extern "C" sm_status sm_state_save(sm_state* st, int32_t with_factors, void* host, size_t bytes,
                                   size_t* needed, void* stream) {
  if (!st || !needed) return SM_EINVAL;
  if (st->d.therm) return SM_ENOTSUP;
  uint64_t b[5];
  image_sizes(st, with_factors, b);
  const size_t total = sizeof(StateImage) + b[0] + b[1] + b[2] + b[3] + b[4];
  *needed = total;
  if (!host) return SM_OK;
  if (bytes < total || st->C < 1) return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  StateImage im{};
  im.magic = kImageMagic;
  im.version = 2;
  im.n_s = st->d.n;
  im.n_r = st->d.n_r;
  im.precision = st->opts.precision;
  im.cap = st->cap;
  im.ld = st->ld;
  im.C = st->C;
  im.lu_stride = st->d.lu_stride;
  im.t_end = st->t_end;
  im.record = st->d.record;
  im.with_factors = with_factors ? 1 : 0;
  for (int i = 0; i < 5; ++i) im.bytes[i] = b[i];
  std::memcpy(host, &im, sizeof im);
  char* dst = static_cast<char*>(host) + sizeof im;
  const DevArray* parts[3] = {&st->scal_d, &st->scal_i, &st->vec};
  for (int i = 0; i < 3; ++i) {
    SM_TRY_CUDA(cudaMemcpyAsync(dst, parts[i]->p, parts[i]->bytes, cudaMemcpyDeviceToHost, st->s));
    dst += parts[i]->bytes;
  }
  if (st->rec_d.bytes) {
    SM_TRY_CUDA(cudaMemcpyAsync(dst, st->rec_d.p, st->rec_d.bytes, cudaMemcpyDeviceToHost, st->s));
    dst += st->rec_d.bytes;
  }
  if (st->rec_i.bytes) {
    SM_TRY_CUDA(cudaMemcpyAsync(dst, st->rec_i.p, st->rec_i.bytes, cudaMemcpyDeviceToHost, st->s));
    dst += st->rec_i.bytes;
  }
  if (b[4]) {
    SM_TRY_CUDA(cudaMemcpyAsync(dst, st->lup.p, st->lup.bytes, cudaMemcpyDeviceToHost, st->s));
    if (b[4] > st->lup.bytes)
      SM_TRY_CUDA(cudaMemcpyAsync(dst + st->lup.bytes, st->lu.p, st->lu.bytes, cudaMemcpyDeviceToHost, st->s));
  }
  SM_TRY_CUDA(cudaStreamSynchronize(st->s));
  return join_out(st, stream);
}

extern "C" sm_status sm_state_load(sm_state* st, const void* host, size_t bytes, void* stream) {
  if (!st || !host || bytes < sizeof(StateImage)) return SM_EINVAL;
  if (st->d.therm) return SM_ENOTSUP;
  StateImage im;
  std::memcpy(&im, host, sizeof im);
  uint64_t b[5];
  image_sizes(st, im.with_factors, b);
  const size_t total = sizeof(StateImage) + b[0] + b[1] + b[2] + b[3] + b[4];
  // the image must come from a state of the same shape: network size,
  // capacity, precision and recording
  if (im.magic != kImageMagic || im.version != 2 || im.n_s != st->d.n || im.n_r != st->d.n_r ||
      im.precision != st->opts.precision || im.cap != st->cap || im.ld != st->ld ||
      im.lu_stride != st->d.lu_stride || im.record != st->d.record || im.C < 1 || im.C > st->cap ||
      bytes < total)
    return SM_EINVAL;
  for (int i = 0; i < 5; ++i)
    if (im.bytes[i] != b[i]) return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  const char* src = static_cast<const char*>(host) + sizeof im;
  const DevArray* parts[3] = {&st->scal_d, &st->scal_i, &st->vec};
  for (int i = 0; i < 3; ++i) {
    SM_TRY_CUDA(cudaMemcpyAsync(parts[i]->p, src, parts[i]->bytes, cudaMemcpyHostToDevice, st->s));
    src += parts[i]->bytes;
  }
  if (st->rec_d.bytes) {
    SM_TRY_CUDA(cudaMemcpyAsync(st->rec_d.p, src, st->rec_d.bytes, cudaMemcpyHostToDevice, st->s));
    src += st->rec_d.bytes;
  }
  if (st->rec_i.bytes) {
    SM_TRY_CUDA(cudaMemcpyAsync(st->rec_i.p, src, st->rec_i.bytes, cudaMemcpyHostToDevice, st->s));
    src += st->rec_i.bytes;
  }
  if (b[4]) {
    SM_TRY_CUDA(cudaMemcpyAsync(st->lup.p, src, st->lup.bytes, cudaMemcpyHostToDevice, st->s));
    if (b[4] > st->lup.bytes)
      SM_TRY_CUDA(cudaMemcpyAsync(st->lu.p, src + st->lup.bytes, st->lu.bytes, cudaMemcpyHostToDevice, st->s));
  }
  st->C = im.C;
  st->t_end = im.t_end;
  st->d.C = im.C;
  st->d.t_end = im.t_end;
  st->kslot_src = nullptr;   // regathered from the next sm_step_bdf's d_k
  set_active_kernel<<<1, 32, 0, st->s>>>(st->d);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 1;
  if (!im.with_factors) {
    need_j_kernel<<<blocks(im.C, 128), 128, 0, st->s>>>(st->d);
    SM_TRY_CUDA(cudaGetLastError());
    st->launches += 1;
  }
  // the host copies must be complete before the caller may free its buffer
  SM_TRY_CUDA(cudaStreamSynchronize(st->s));
  return join_out(st, stream);
}

extern "C" sm_status sm_state_timing(const sm_state* st, int64_t* launches, double* ms, int64_t* timed) {
  if (!st) return SM_EINVAL;
  if (launches) *launches = st->launches;
  if (ms) *ms = st->timed_ms;
  if (timed) *timed = st->timed;
  return SM_OK;
}

extern "C" sm_status sm_state_timing_reset(sm_state* st) {
  if (!st) return SM_EINVAL;
  st->launches = 0;
  st->timed = 0;
  st->timed_ms = 0.0;
  return SM_OK;
}

extern "C" sm_status sm_phase_cycles(int32_t device, double* h_out, int32_t reset) {
#ifdef SM_PHASE_CLOCKS
  if (!h_out || device < 0) return SM_EINVAL;
  Scope scope(device);
  if (!scope.ok) return SM_ECUDA;
  unsigned long long v[kPhaseSlots];
  SM_TRY_CUDA(cudaMemcpyFromSymbol(v, g_phase_cycles, sizeof(v)));
  for (int i = 0; i < kPhaseSlots; ++i) h_out[i] = (double)v[i];
  if (reset) {
    const unsigned long long z[kPhaseSlots] = {0};
    SM_TRY_CUDA(cudaMemcpyToSymbol(g_phase_cycles, z, sizeof(z)));
  }
  return SM_OK;
#else
  (void)device;
  (void)h_out;
  (void)reset;
  return SM_ENOTSUP;
#endif
}
