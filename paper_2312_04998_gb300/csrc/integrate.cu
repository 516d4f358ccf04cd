// Batched variable-order BDF integration with simplified Newton iterations
// (the stiff-solver role of DLSODES in Section 3), one independent state
// machine per cell.
//
// One "attempt" advances every unfinished cell by one trial step:
//   predict   thread per cell: Lagrange predictor, BDF coefficients, weights,
//             and the decision whether the Newton matrix must be refreshed;
//   refresh   one CTA per cell on the compacted refresh list: J at the
//             predicted state, M = I - gamma J (FP64, equilibrated and
//             rounded to FP32 in mixed precision), in-place LU without
//             pivoting in the minimum-degree order, inverse pivots kept;
//   newton    up to newton_max rounds of: reaction rates + CRS gather of
//             S R(y) (cells fast axis, masked to iterating cells), then one
//             warp per cell forming the FP64 residual, forward/backward
//             substitution and the WRMS convergence test;
//   finish    thread per cell: error test, order / step selection, history.
// The host enqueues attempts in groups (captured once in a CUDA graph) and
// reads back only the number of running cells between groups.
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

constexpr int QMAX = 5;  // highest BDF order; the history keeps QMAX + 1 points
enum : int {
  F_NEED_J = 1, F_REJECTED = 2, F_HAS_EPREV = 4, F_NEWTON = 8, F_CONV = 16,
  F_FINAL = 32, F_REFRESH = 64, F_FAILED = 128, F_ATTEMPT = 256
};

struct Dev {
  int n, n_r, nnz_j, mixed, head;
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
  void* lu;
  int64_t lu_stride;
  int ldm;
  const int *perm, *iperm, *lptr, *lidx, *uptr, *uidx, *lrptr, *lridx, *jp_ptr, *jt_ptr, *jpos;
  const int2* jt_word;
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
  for (int j = 0; j < d.n_r; ++j) ok = ok && isfinite(k[(int64_t)j * ldk + c]);
  d.status[c] = ok ? SM_CELL_RUNNING : SM_CELL_NAN;
  d.flags[c] = ok ? F_NEWTON : 0;  // F_NEWTON selects the cells for f0
  d.t[c] = 0.0;
  d.steps[c] = d.rejects[c] = d.conv_fails[c] = d.newton_iters[c] = d.jac_evals[c] = 0;
  d.q[c] = 1;
  d.h[c] = 0.0;
}

__global__ void init_finish_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
}

// ---------------------------------------------------------------------------
// predict
// ---------------------------------------------------------------------------
__global__ void predict_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  int fl = d.flags[c] & ~(F_CONV | F_FAILED | F_REFRESH | F_FINAL | F_NEWTON | F_ATTEMPT);
  if (d.status[c] != SM_CELL_RUNNING) {
    d.flags[c] = fl;
    return;
  }
  atomicAdd(&d.counters[1], 1);
  if (d.steps[c] >= d.max_steps) {
    d.status[c] = SM_CELL_MAXSTEPS;
    d.flags[c] = fl;
    return;
  }
  const double t = d.t[c];
  double h = d.h[c];
  const int q = d.q[c], nh = d.nh[c];
  const bool fin = t + h >= d.t_end;
  if (fin) h = d.t_end - t;
  const double tnew = fin ? d.t_end : t + h;
  if (tnew == t || !(h > 0.0)) {
    d.status[c] = SM_CELL_HMIN;
    d.flags[c] = fl;
    return;
  }
  double T[QMAX + 1], wts[QMAX + 1], al[QMAX + 1];
  for (int i = 0; i < nh; ++i) T[i] = d.tn[(int64_t)i * d.ld + c];
  if (nh > 1) lagrange(T, q + 1, tnew, wts);
  bdf_alphas(tnew, T, q, h, al);
  const double gamma = h / al[0];
  const bool refresh = (fl & F_NEED_J) || d.j_age[c] >= d.j_age_max ||
                       fabs(gamma / d.gam_J[c] - 1.0) > d.gamma_tol;
  d.h[c] = h;
  d.gam[c] = gamma;
  for (int i = 0; i <= q; ++i) d.alpha[(int64_t)i * d.ld + c] = al[i];
  d.flags[c] = fl | F_NEWTON | F_ATTEMPT | (fin ? F_FINAL : 0) | (refresh ? F_REFRESH : 0);
  d.m_it[c] = 0;
  d.dprev[c] = 0.0;
  if (refresh) d.list[atomicAdd(&d.counters[0], 1)] = (int)c;
  for (int s = 0; s < d.n; ++s) {
    const int64_t o = (int64_t)s * d.ld + c;
    const double y0 = Yh(d, 0)[o];
    double yp;
    if (nh == 1) {
      yp = y0 + h * d.f0[o];
    } else {
      yp = 0.0;
      for (int i = 0; i <= q; ++i) yp += wts[i] * Yh(d, i)[o];
    }
    double ps = 0.0;
    for (int i = 1; i <= q; ++i) ps += al[i] * Yh(d, i - 1)[o];
    d.ypred[o] = yp;
    d.y[o] = yp;
    d.psi[o] = ps;
    d.w[o] = 1.0 / (d.rtol * fabs(y0) + d.atol);
  }
}

// ---------------------------------------------------------------------------
// refresh: J, M = I - gamma J and its LU without pivoting, in place in dense
// per-cell storage (elimination order = minimum degree).  One CTA per cell on
// the compacted refresh list (grid-stride).  The first `head` pivots are
// sparse and follow the symbolic schedule; the trailing block from `head` on
// is >= 90 % dense and is factorised by a right-looking blocked algorithm:
// panels of kNB columns are factorised in shared memory, U12 is solved in
// shared memory, and the trailing update A22 -= L21 U12 runs as a register-
// tiled GEMM (kTM x kTN outputs per thread).  Inverse pivots replace the
// diagonal.
// ---------------------------------------------------------------------------
constexpr int kRefreshThreads = 256;
constexpr int kNB = 32;
constexpr int kTM = 4, kTN = 4;

size_t refresh_smem_bytes(int n, int head, size_t esz) {
  const size_t nt = (size_t)(n - head);
  return esz * (nt * (kNB + 1) + (size_t)kNB * nt);
}

template <class T>
__global__ void __launch_bounds__(kRefreshThreads) refresh_kernel(Dev d, const double* __restrict__ k,
                                                                 int64_t ldk) {
  extern __shared__ unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int n = d.n, ldm = d.ldm, h = d.head, nt = n - h;
  T* P = reinterpret_cast<T*>(smem_raw);            // panel, pitch kNB + 1
  T* U = P + (size_t)nt * (kNB + 1);                // U12 block, pitch r
  constexpr int PP = kNB + 1;
  const int count = d.counters[0];
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t c = d.list[e];
    T* A = static_cast<T*>(d.lu) + c * d.lu_stride;
    const double gamma = d.gam[c];
    // zero the dense trailing block and the head's pattern entries
    for (int64_t i = tid; i < (int64_t)nt * nt; i += nthr) {
      const int r = (int)(i / nt), q = (int)(i - (int64_t)r * nt);
      A[(int64_t)(h + r) * ldm + h + q] = T(0);
    }
    for (int kp = warp; kp < h; kp += nwarps) {
      for (int p = __ldg(d.lptr + kp) + lane; p < __ldg(d.lptr + kp + 1); p += 32)
        A[(int64_t)__ldg(d.lidx + p) * ldm + kp] = T(0);
      for (int p = __ldg(d.uptr + kp) + lane; p < __ldg(d.uptr + kp + 1); p += 32)
        A[(int64_t)kp * ldm + __ldg(d.uidx + p)] = T(0);
      if (lane == 0) A[(int64_t)kp * ldm + kp] = T(0);
    }
    if (d.mixed)
      for (int s = tid; s < n; s += nthr) V(d.wf, d, s, c) = V(d.w, d, s, c);
    __syncthreads();
    // M = I - gamma J at the pattern positions (J gathered in FP64)
    for (int p = tid; p < d.nnz_j; p += nthr) {
      double acc = 0.0;
      const int t1 = __ldg(d.jt_ptr + p + 1);
      for (int t = __ldg(d.jt_ptr + p); t < t1; ++t) {
        const int2 wd = __ldg(d.jt_word + t);
        double v = k[(int64_t)(wd.x & 0xFFFFFF) * ldk + c];
        if (wd.y >= 0) v *= d.ypred[(int64_t)wd.y * d.ld + c];
        acc = fma((double)(int8_t)((uint32_t)wd.x >> 24), v, acc);
      }
      const int pos = __ldg(d.jpos + p);
      const int pi = pos / ldm, pj = pos - pi * ldm;
      double m = (pi == pj ? 1.0 : 0.0) - gamma * acc;
      if (d.mixed) {
        // equilibrated W M W^-1 with the error weights of this step
        m *= V(d.w, d, __ldg(d.perm + pi), c) / V(d.w, d, __ldg(d.perm + pj), c);
      }
      A[pos] = T(m);
    }
    __syncthreads();
    // sparse head pivots
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
    // dense trailing block: blocked right-looking LU
    for (int p0 = h; p0 < n; p0 += kNB) {
      const int w = min(kNB, n - p0), m = n - p0, r = m - w;
      for (int i = tid; i < m * w; i += nthr) {
        const int a = i / w, b = i - a * w;
        P[a * PP + b] = A[(int64_t)(p0 + a) * ldm + p0 + b];
      }
      __syncthreads();
      for (int kk = 0; kk < w; ++kk) {
        const T inv = T(1) / P[kk * PP + kk];
        for (int i = kk + 1 + tid; i < m; i += nthr) P[i * PP + kk] *= inv;
        __syncthreads();
        const int cols = w - kk - 1;
        if (cols > 0)
          for (int i = tid; i < (m - kk - 1) * cols; i += nthr) {
            const int a = kk + 1 + i / cols, b = kk + 1 + i % cols;
            P[a * PP + b] -= P[a * PP + kk] * P[kk * PP + b];
          }
        if (tid == 0) P[kk * PP + kk] = inv;
        __syncthreads();
      }
      for (int i = tid; i < m * w; i += nthr) {
        const int a = i / w, b = i - a * w;
        A[(int64_t)(p0 + a) * ldm + p0 + b] = P[a * PP + b];
      }
      if (r > 0) {
        // U12 = L11^-1 A12, one thread per column
        for (int i = tid; i < w * r; i += nthr) {
          const int a = i / r, b = i - a * r;
          U[a * r + b] = A[(int64_t)(p0 + a) * ldm + p0 + w + b];
        }
        __syncthreads();
        for (int b = tid; b < r; b += nthr) {
          for (int kk = 0; kk < w; ++kk) {
            const T u = U[kk * r + b];
            for (int a = kk + 1; a < w; ++a) U[a * r + b] -= P[a * PP + kk] * u;
          }
          for (int a = 0; a < w; ++a) A[(int64_t)(p0 + a) * ldm + p0 + w + b] = U[a * r + b];
        }
        __syncthreads();
        // A22 -= L21 U12, tiles of (16 kTM) x (16 kTN)
        const int ty = tid / 16, tx = tid % 16;
        constexpr int BM = 16 * kTM, BN = 16 * kTN;
        for (int t0 = 0; t0 < r; t0 += BM)
          for (int u0 = 0; u0 < r; u0 += BN) {
            T acc[kTM][kTN];
            const int i0 = t0 + ty * kTM, j0 = u0 + tx * kTN;
#pragma unroll
            for (int a = 0; a < kTM; ++a)
#pragma unroll
              for (int b = 0; b < kTN; ++b)
                acc[a][b] = (i0 + a < r && j0 + b < r)
                                ? A[(int64_t)(p0 + w + i0 + a) * ldm + p0 + w + j0 + b] : T(0);
            for (int kk = 0; kk < w; ++kk) {
              T lv[kTM], uv[kTN];
#pragma unroll
              for (int a = 0; a < kTM; ++a) lv[a] = (i0 + a < r) ? P[(w + i0 + a) * PP + kk] : T(0);
#pragma unroll
              for (int b = 0; b < kTN; ++b) uv[b] = (j0 + b < r) ? U[kk * r + j0 + b] : T(0);
#pragma unroll
              for (int a = 0; a < kTM; ++a)
#pragma unroll
                for (int b = 0; b < kTN; ++b) acc[a][b] -= lv[a] * uv[b];
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
    }
    if (tid == 0) {
      d.gam_J[c] = gamma;
      d.j_age[c] = 0;
      d.crate[c] = 1.0;
      d.flags[c] &= ~F_NEED_J;
      d.jac_evals[c] += 1;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Newton: residual, substitution, update and convergence test (warp per cell)
// ---------------------------------------------------------------------------
constexpr int kSolveWarps = 4;

template <class T>
__global__ void __launch_bounds__(32 * kSolveWarps) solve_update_kernel(Dev d) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * kSolveWarps + wi;
  if (c >= d.C) return;
  if (!(d.flags[c] & F_NEWTON)) return;
  const int n = d.n, ldm = d.ldm;
  T* x = reinterpret_cast<T*>(smem_raw) + (int64_t)wi * n;
  const T* A = static_cast<const T*>(d.lu) + c * d.lu_stride;
  const double a0 = d.alpha[c], h = d.h[c];
  const double inv_a0 = 1.0 / a0;
  for (int s = lane; s < n; s += 32) {
    const int64_t o = (int64_t)s * d.ld + c;
    double b = -(a0 * d.y[o] + d.psi[o] - h * d.f[o]) * inv_a0;
    if (d.mixed) b *= d.wf[o];
    x[__ldg(d.iperm + s)] = T(b);
  }
  __syncwarp();
  // forward: unit lower triangle, row-oriented
  for (int i = 0; i < n; ++i) {
    const int p0 = __ldg(d.lrptr + i), p1 = __ldg(d.lrptr + i + 1);
    if (p1 == p0) continue;
    T s = T(0);
    const T* Ai = A + (int64_t)i * ldm;
    for (int p = p0 + lane; p < p1; p += 32) {
      const int kk = __ldg(d.lridx + p);
      s += Ai[kk] * x[kk];
    }
    s = warp_sum(s);
    if (lane == 0) x[i] -= s;
    __syncwarp();
  }
  // backward: upper triangle with inverse pivots on the diagonal
  for (int kp = n - 1; kp >= 0; --kp) {
    const int u0 = __ldg(d.uptr + kp), u1 = __ldg(d.uptr + kp + 1);
    const T* Ak = A + (int64_t)kp * ldm;
    T s = T(0);
    for (int p = u0 + lane; p < u1; p += 32) {
      const int j = __ldg(d.uidx + p);
      s += Ak[j] * x[j];
    }
    s = warp_sum(s);
    if (lane == 0) x[kp] = (x[kp] - s) * Ak[kp];
    __syncwarp();
  }
  const double gamma = d.gam[c], gJ = d.gam_J[c];
  const double scale = gamma != gJ ? 2.0 / (1.0 + gamma / gJ) : 1.0;
  double acc = 0.0;
  for (int s = lane; s < n; s += 32) {
    const int64_t o = (int64_t)s * d.ld + c;
    double del = (double)x[__ldg(d.iperm + s)];
    if (d.mixed) del /= d.wf[o];
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
// finish: error test, step / order selection, history update
// ---------------------------------------------------------------------------
__global__ void finish_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  int fl = d.flags[c];
  if (!(fl & F_ATTEMPT)) return;
  fl &= ~F_ATTEMPT;
  const int n = d.n;
  const int q = d.q[c], nh = d.nh[c];
  double h = d.h[c];
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
  const double t = d.t[c];
  const double tnew = (fl & F_FINAL) ? d.t_end : t + h;
  double T[QMAX + 1];
  for (int i = 0; i < nh; ++i) T[i] = d.tn[(int64_t)i * d.ld + c];
  double acc = 0.0;
  for (int s = 0; s < n; ++s) {
    const int64_t o = (int64_t)s * d.ld + c;
    const double v = (d.y[o] - d.ypred[o]) * d.w[o];
    acc += v * v;
  }
  const double Cq = nh >= q + 1 ? h / (tnew - T[q]) : 1.0 / (q + 1);
  const double err = Cq * sqrt(acc / n);
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
  // accepted: rate neighbouring orders on the old history
  const int naq = d.n_at_q[c] + 1;
  double best_eta = 0.9 * pow(fmax(err, 1e-10), -1.0 / (q + 1));
  int best_q = q;
  if (naq >= q + 1) {
    const bool lo = q > 1;
    const bool hi = q < d.q_max && (fl & F_HAS_EPREV) && nh + 1 >= q + 2;
    if (lo || hi) {
      double wl[QMAX + 1];
      if (lo) lagrange(T, q, tnew, wl);
      double acc_lo = 0.0, acc_hi = 0.0;
      for (int s = 0; s < n; ++s) {
        const int64_t o = (int64_t)s * d.ld + c;
        const double yv = d.y[o], wv = d.w[o];
        if (lo) {
          double p = 0.0;
          for (int i = 0; i < q; ++i) p += wl[i] * Yh(d, i)[o];
          const double v = (yv - p) * wv;
          acc_lo += v * v;
        }
        if (hi) {
          const double v = ((yv - d.ypred[o]) - d.eprev[o]) * wv;
          acc_hi += v * v;
        }
      }
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
    }
  }
  // commit: shift the history, newest first
  const int nh_new = min(nh + 1, d.q_max + 1);
  const bool keep_e = best_q == q;
  for (int s = 0; s < n; ++s) {
    const int64_t o = (int64_t)s * d.ld + c;
    for (int i = nh_new - 1; i >= 1; --i) Yh(d, i)[o] = Yh(d, i - 1)[o];
    const double yv = d.y[o];
    if (keep_e) d.eprev[o] = yv - d.ypred[o];
    Yh(d, 0)[o] = yv;
  }
  for (int i = nh_new - 1; i >= 1; --i) d.tn[(int64_t)i * d.ld + c] = T[i - 1];
  d.tn[c] = tnew;
  d.nh[c] = nh_new;
  d.t[c] = tnew;
  d.steps[c] += 1;
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
  if (yout)
    for (int s = 0; s < d.n; ++s) yout[(int64_t)s * ldu + c] = Yh(d, 0)[(int64_t)s * d.ld + c];
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
    st[c] = r;
  }
}

// counters[1] = cells still running, counters[2] = cells stopped short of t_end
__global__ void count_running_kernel(Dev d) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  const int s = d.status[c];
  if (s == SM_CELL_RUNNING) atomicAdd(&d.counters[1], 1);
  else if (s != SM_CELL_OK) atomicAdd(&d.counters[2], 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sm_state {
  const sm_net* net = nullptr;
  sm_opts opts{};
  int64_t cap = 0, C = 0, ld = 0;
  double t_end = 0.0;
  Dev d{};
  DevArray scal_d, scal_i, vec, lu, list, counters, scratch;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int* h_counters = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  const double* graph_k = nullptr;
  int64_t graph_ldk = 0, graph_C = 0;
  int refresh_ctas = 0;
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
         (o.precision == SM_PREC_FP64 || o.precision == SM_PREC_MIXED) && o.attempts_per_sync >= 1 &&
         o.timing_kind >= SM_TIME_NONE && o.timing_kind <= SM_TIME_FINISH;
}

void free_state(sm_state* st) {
  if (st->graph) cudaGraphExecDestroy(st->graph);
  for (cudaEvent_t e : st->ev_pool) cudaEventDestroy(e);
  st->ev_pool.clear();
  st->scal_d.release();
  st->scal_i.release();
  st->vec.release();
  st->lu.release();
  st->list.release();
  st->counters.release();
  st->scratch.release();
  if (st->h_counters) cudaFreeHost(st->h_counters);
  if (st->ev_in) cudaEventDestroy(st->ev_in);
  if (st->ev_out) cudaEventDestroy(st->ev_out);
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

constexpr int kLaunchesFixed = 3;  // predict, refresh, finish (+3 per Newton round)

template <class T>
sm_status enqueue_attempt(sm_state* st, const double* k, int64_t ldk, cudaStream_t s) {
  Dev& d = st->d;
  const sm_net* net = st->net;
  sm_status r;
  SM_TRY_CUDA(cudaMemsetAsync(d.counters, 0, 2 * sizeof(int), s));
  if ((r = time_mark(st, SM_TIME_PREDICT, true, s)) != SM_OK) return r;
  predict_kernel<<<blocks(d.C, 128), 128, 0, s>>>(d);
  if ((r = time_mark(st, SM_TIME_PREDICT, false, s)) != SM_OK) return r;
  if ((r = time_mark(st, SM_TIME_REFRESH, true, s)) != SM_OK) return r;
  refresh_kernel<T><<<st->refresh_ctas, kRefreshThreads, refresh_smem_bytes(d.n, d.head, sizeof(T)), s>>>(
      d, k, ldk);
  if ((r = time_mark(st, SM_TIME_REFRESH, false, s)) != SM_OK) return r;
  const size_t smem = sizeof(T) * (size_t)kSolveWarps * d.n;
  for (int m = 0; m < d.newton_max; ++m) {
    if ((r = time_mark(st, SM_TIME_RHS, true, s)) != SM_OK) return r;
    r = launch_rhs_masked(net, d.C, k, ldk, d.y, d.f, d.ld, st->scratch.as<double>(), d.ld, d.flags,
                          F_NEWTON, s);
    if (r != SM_OK) return r;
    if ((r = time_mark(st, SM_TIME_RHS, false, s)) != SM_OK) return r;
    if ((r = time_mark(st, SM_TIME_SOLVE, true, s)) != SM_OK) return r;
    solve_update_kernel<T><<<blocks(d.C, kSolveWarps), 32 * kSolveWarps, smem, s>>>(d);
    if ((r = time_mark(st, SM_TIME_SOLVE, false, s)) != SM_OK) return r;
  }
  if ((r = time_mark(st, SM_TIME_FINISH, true, s)) != SM_OK) return r;
  finish_kernel<<<blocks(d.C, 128), 128, 0, s>>>(d);
  if ((r = time_mark(st, SM_TIME_FINISH, false, s)) != SM_OK) return r;
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += kLaunchesFixed + 3 * d.newton_max;
  return SM_OK;
}

sm_status enqueue_group(sm_state* st, const double* k, int64_t ldk, int attempts, cudaStream_t s) {
  if (!st->opts.use_graph) st->ev_used = 0;
  for (int a = 0; a < attempts; ++a) {
    sm_status r = st->opts.precision == SM_PREC_MIXED ? enqueue_attempt<float>(st, k, ldk, s)
                                                      : enqueue_attempt<double>(st, k, ldk, s);
    if (r != SM_OK) return r;
  }
  return SM_OK;
}

// Runs `attempts` attempts on the state's stream, through a cached CUDA graph
// when enabled (captured once per (k, ldk, C)).
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
  if (!st->graph || st->graph_k != k || st->graph_ldk != ldk || st->graph_C != st->d.C) {
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
  d.mixed = o.precision == SM_PREC_MIXED;
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
  const int n_iscal = 14;
  const int n_vec = (QMAX + 1) + 8;         // Y[6] ypred y psi f f0 eprev w wf
  if ((r = st->scal_d.ensure(sizeof(double) * n_dscal * ld)) != SM_OK) return fail(r);
  if ((r = st->scal_i.ensure(sizeof(int) * n_iscal * ld)) != SM_OK) return fail(r);
  if ((r = st->vec.ensure(sizeof(double) * (size_t)n_vec * n * ld)) != SM_OK) return fail(r);
  const size_t esz = d.mixed ? sizeof(float) : sizeof(double);
  d.lu_stride = (int64_t)n * lu.ld;
  if ((r = st->lu.ensure(esz * (size_t)d.lu_stride * C)) != SM_OK) return fail(r);
  if ((r = st->list.ensure(sizeof(int) * ld)) != SM_OK) return fail(r);
  if ((r = st->counters.ensure(sizeof(int) * 4)) != SM_OK) return fail(r);
  if ((r = st->scratch.ensure(sizeof(double) * (size_t)net->n_r * ld)) != SM_OK) return fail(r);
  double* ds = st->scal_d.as<double>();
  d.t = ds; d.h = ds + ld; d.gam = ds + 2 * ld; d.gam_J = ds + 3 * ld; d.crate = ds + 4 * ld;
  d.dprev = ds + 5 * ld; d.tn = ds + 6 * ld; d.alpha = ds + (6 + QMAX + 1) * ld;
  int* is = st->scal_i.as<int>();
  d.q = is; d.nh = is + ld; d.n_at_q = is + 2 * ld; d.j_age = is + 3 * ld; d.flags = is + 4 * ld;
  d.crej = is + 5 * ld; d.ccf = is + 6 * ld; d.status = is + 7 * ld; d.m_it = is + 8 * ld;
  d.steps = is + 9 * ld; d.rejects = is + 10 * ld; d.conv_fails = is + 11 * ld;
  d.newton_iters = is + 12 * ld; d.jac_evals = is + 13 * ld;
  double* v = st->vec.as<double>();
  const int64_t vs = (int64_t)n * ld;
  d.Y = v; d.ypred = v + (QMAX + 1) * vs; d.y = d.ypred + vs; d.psi = d.y + vs; d.f = d.psi + vs;
  d.f0 = d.f + vs; d.eprev = d.f0 + vs; d.w = d.eprev + vs; d.wf = d.w + vs;
  d.list = st->list.as<int>();
  d.counters = st->counters.as<int>();
  d.lu = st->lu.p;
  d.perm = lu.d_perm.as<int>(); d.iperm = lu.d_iperm.as<int>();
  d.lptr = lu.d_lptr.as<int>(); d.lidx = lu.d_lidx.as<int>();
  d.uptr = lu.d_uptr.as<int>(); d.uidx = lu.d_uidx.as<int>();
  d.lrptr = lu.d_lrptr.as<int>(); d.lridx = lu.d_lridx.as<int>();
  d.jp_ptr = net->d_jp_ptr.as<int>(); d.jt_ptr = net->d_jt_ptr.as<int>();
  d.jt_word = net->d_jt_word.as<int2>(); d.jpos = lu.d_jpos.as<int>();
  if (cudaStreamCreateWithFlags(&st->s, cudaStreamNonBlocking) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(SM_ECUDA);
  if (cudaMallocHost(&st->h_counters, 4 * sizeof(int)) != cudaSuccess) return fail(SM_ENOMEM);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device);
  const size_t rsm = refresh_smem_bytes(n, lu.head, esz);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device);
  if ((int64_t)rsm > smem_max) return fail(SM_ENOTSUP);
  if (d.mixed) {
    SM_TRY_CUDA(cudaFuncSetAttribute(refresh_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
  } else {
    SM_TRY_CUDA(cudaFuncSetAttribute(refresh_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
  }
  int per_sm = 0;
  if (d.mixed) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refresh_kernel<float>, kRefreshThreads, rsm);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refresh_kernel<double>, kRefreshThreads, rsm);
  }
  st->refresh_ctas = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
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
  *bytes = st->scal_d.bytes + st->scal_i.bytes + st->vec.bytes + st->lu.bytes + st->list.bytes +
           st->counters.bytes + st->scratch.bytes;
  return SM_OK;
}

sm_status sm_state_init(sm_state* st, int64_t C, const double* d_k, const double* d_y, int64_t ld,
                        double t_end, void* stream) {
  if (!st || C < 1 || C > st->cap || !ld_ok(C, ld) || !d_k || !d_y || !(t_end > 0.0)) return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
  st->C = C;
  st->t_end = t_end;
  Dev& d = st->d;
  d.C = C;
  d.t_end = t_end;
  init_copy_kernel<<<blocks(C, 128), 128, 0, st->s>>>(d, d_y, ld, d_k, ld);
  SM_TRY_CUDA(cudaGetLastError());
  r = launch_rhs_masked(st->net, C, d_k, ld, d.Y, d.f0, d.ld, st->scratch.as<double>(), d.ld, d.flags,
                        F_NEWTON, st->s);
  if (r != SM_OK) return r;
  init_finish_kernel<<<blocks(C, 128), 128, 0, st->s>>>(d);
  SM_TRY_CUDA(cudaGetLastError());
  st->launches += 4;
  return join_out(st, stream);
}

sm_status sm_step_bdf(sm_state* st, const double* d_k, int64_t ld, int32_t attempts, void* stream) {
  if (!st || !d_k || st->C < 1 || !ld_ok(st->C, ld) || attempts < 0) return SM_EINVAL;
  Scope scope(st->net->device);
  if (!scope.ok) return SM_ECUDA;
  sm_status r;
  if ((r = join_in(st, stream)) != SM_OK) return r;
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

}  // extern "C"

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
