// Right-hand side f = S R(x) (Eq. 7), batched with cells as the fast axis.
//
// Four traversals of S, the GPU counterparts of the paper's Listings 1-4:
//  * CRS  (Listing 3): rows gathered; the nonzeros of S are cut into equal
//    chunks (one per half-warp) so the long hub rows (H: ~2000 nonzeros) are
//    shared; rows split across chunks are summed in chunk order through shared
//    memory, so results are deterministic.
//  * COO  (Listing 1): each nonzero adds coef * R_col into f_row (two indirect
//    indices, FP64 atomics in L2).
//  * CCS  (Listing 2): each reaction's rate is formed once in registers and
//    scattered to its (at most six) species (FP64 atomics in L2).
//  * SELL-C-sigma (Listing 4): one thread per (cell, row of a slice) walks
//    the slice column-major, pads included.
// In every traversal a lane owns one cell: index loads are warp-uniform
// broadcasts and abundance / rate loads are 128-byte coalesced rows.
#include <atomic>
#include <mutex>

#include "internal.h"

namespace {

__constant__ double c_coef[256];  // (double)(int8_t)i : coefficient decode table
constexpr int kCells = 16;        // cells per CTA (half a warp)
constexpr int kChunks = 32;       // CRS nonzero chunks per CTA (two per warp)
constexpr int kRThreads = 128;
constexpr int kRChunk = 64;

__device__ __forceinline__ int upper_bound_i32(const int* __restrict__ a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int lower_bound_i32(const int* __restrict__ a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double neg_if(double v, bool neg) {
  return neg ? __longlong_as_double(__double_as_longlong(v) ^ (1ll << 63)) : v;
}

// R_j = k'_j * x_a * x_b, multiplied left to right.
__global__ void __launch_bounds__(kRThreads)
reaction_rate_kernel(int n_r, int64_t C, const int2* __restrict__ reac, const double* __restrict__ k,
                     int64_t ldk, const double* __restrict__ y, int64_t ldy, double* __restrict__ r,
                     int64_t ldr, const int* __restrict__ mask, int bit, const int* __restrict__ cact) {
  if (cact && (int64_t)blockIdx.x * kRThreads >= *cact) return;   // no running cell in this block
  const int64_t c = (int64_t)blockIdx.x * kRThreads + threadIdx.x;
  const bool act = c < C && (!mask || (mask[c] & bit));
  if (mask && !__syncthreads_or(act)) return;
  if (!act) return;
  const int j1 = min(n_r, (int)(blockIdx.y + 1) * kRChunk);
#pragma unroll 4
  for (int j = blockIdx.y * kRChunk; j < j1; ++j) {
    const int2 a = __ldg(reac + j);
    double v = k[(int64_t)j * ldk + c] * y[(int64_t)a.x * ldy + c];
    if (a.y >= 0) v *= y[(int64_t)a.y * ldy + c];
    r[(int64_t)j * ldr + c] = v;
  }
}

// sum over entries [b, e) of coef * r[col]: four independent partial sums so
// that four rate loads are in flight per thread (the FP64 gather is bound by
// their latency, not by the FP64 pipe)
__device__ __forceinline__ double dot_range(const uint32_t* __restrict__ ent, int b, int e,
                                            const double* __restrict__ r, int64_t ldr, int64_t c) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int p = b;
  for (; p + 3 < e; p += 4) {
    const uint32_t w0 = __ldg(ent + p), w1 = __ldg(ent + p + 1), w2 = __ldg(ent + p + 2), w3 = __ldg(ent + p + 3);
    const double r0 = r[(int64_t)(w0 & 0xFFFFFFu) * ldr + c], r1 = r[(int64_t)(w1 & 0xFFFFFFu) * ldr + c];
    const double r2 = r[(int64_t)(w2 & 0xFFFFFFu) * ldr + c], r3 = r[(int64_t)(w3 & 0xFFFFFFu) * ldr + c];
    s0 = fma(c_coef[w0 >> 24], r0, s0);
    s1 = fma(c_coef[w1 >> 24], r1, s1);
    s2 = fma(c_coef[w2 >> 24], r2, s2);
    s3 = fma(c_coef[w3 >> 24], r3, s3);
  }
  for (; p < e; ++p) {
    const uint32_t w0 = __ldg(ent + p);
    s0 = fma(c_coef[w0 >> 24], r[(int64_t)(w0 & 0xFFFFFFu) * ldr + c], s0);
  }
  return (s0 + s1) + (s2 + s3);
}

// CRS gather of KC cells per block (cells as the fast axis) with KCH nonzero
// chunks of about equal size, KC x KCH = 512 threads; a warp covers 32 / KC
// chunks.  Rows split across chunks are summed in chunk order through shared
// memory, so results do not depend on scheduling.
template <int KC, int KCH>
__global__ void __launch_bounds__(KC * KCH)
rhs_crs_kernel(int n_s, int64_t C, const int* __restrict__ row_ptr, const uint32_t* __restrict__ ent,
               const int* __restrict__ row_id, const int* __restrict__ chunk_nz,
               const double* __restrict__ r, int64_t ldr, double* __restrict__ f, int64_t ld,
               const int* __restrict__ mask, int bit, const int* __restrict__ cact) {
  static_assert(KC * KCH == kCells * kChunks && 32 % KC == 0, "block shape");
  if (cact && (int64_t)blockIdx.x * KC >= *cact) return;      // no running cell in this block
  __shared__ double part[KCH][2][KC];
  __shared__ int carry_row[KCH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ch = warp * (32 / KC) + lane / KC, cl = lane % KC;
  const int64_t c0 = (int64_t)blockIdx.x * KC + cl;
  const bool live = c0 < C && (!mask || (mask[c0] & bit));
  if (mask && !__syncthreads_or(live)) return;
  const int64_t c = live ? c0 : 0;  // dead lanes read cell 0 and store nothing
  const int z0 = __ldg(chunk_nz + ch), z1 = __ldg(chunk_nz + ch + 1);
  // carry-in row: contains position z0 but starts before it
  const int rc = upper_bound_i32(row_ptr, n_s + 1, z0) - 1;
  double carry = 0.0;
  bool has_carry = false;
  if (z0 < z1 && rc < n_s && __ldg(row_ptr + rc) < z0) {
    has_carry = true;
    carry = dot_range(ent, z0, min(__ldg(row_ptr + rc + 1), z1), r, ldr, c);
  }
  // -2 marks an empty chunk (possible when nnz < KCH): fix-ups skip it
  if (cl == 0) carry_row[ch] = z0 == z1 ? -2 : (has_carry ? rc : -1);
  part[ch][0][cl] = carry;
  // rows owned by this chunk: row_ptr[row] in [z0, z1) (all rows for the last)
  const int r_first = lower_bound_i32(row_ptr, n_s, z0);
  const int r_end = (ch == KCH - 1) ? n_s : lower_bound_i32(row_ptr, n_s, z1);
  double tail = 0.0;
  int tail_row = -1;
  for (int row = r_first; row < r_end; ++row) {
    const int b = __ldg(row_ptr + row), e = __ldg(row_ptr + row + 1);
    const double s = dot_range(ent, b, min(e, z1), r, ldr, c);
    if (e <= z1) {
      if (live) f[(int64_t)__ldg(row_id + row) * ld + c] = s;
    } else {
      tail = s;
      tail_row = row;
    }
  }
  part[ch][1][cl] = tail;
  __syncthreads();
  if (tail_row >= 0) {
    double tot = part[ch][1][cl];
    for (int w = ch + 1; w < KCH; ++w) {
      if (carry_row[w] == -2) continue;
      if (carry_row[w] != tail_row) break;
      tot += part[w][0][cl];
    }
    if (live) f[(int64_t)__ldg(row_id + tail_row) * ld + c] = tot;
  }
}

// COO: nonzeros in column-major order; ent = row | coef, col[] = reaction.
__global__ void __launch_bounds__(kRThreads)
rhs_coo_kernel(int nnz, int64_t C, const uint32_t* __restrict__ ent, const int* __restrict__ col,
               const double* __restrict__ r, int64_t ldr, double* __restrict__ f, int64_t ld) {
  const int64_t c = (int64_t)blockIdx.x * kRThreads + threadIdx.x;
  if (c >= C) return;
  const int p1 = min(nnz, (int)(blockIdx.y + 1) * kRChunk);
  for (int p = blockIdx.y * kRChunk; p < p1; ++p) {
    const uint32_t w = __ldg(ent + p);
    const int cf = (int)(int8_t)(w >> 24);
    double v = r[(int64_t)__ldg(col + p) * ldr + c];
    if (cf != 1 && cf != -1) v *= (double)(cf < 0 ? -cf : cf);
    atomicAdd(f + (int64_t)(w & 0xFFFFFFu) * ld + c, neg_if(v, cf < 0));
  }
}

// CCS: per reaction, R formed in registers then scattered to its species.
__global__ void __launch_bounds__(kRThreads)
rhs_ccs_kernel(int n_r, int64_t C, const int* __restrict__ col_ptr, const uint32_t* __restrict__ ent,
               const int* __restrict__ col_id, const int2* __restrict__ reac,
               const double* __restrict__ k, const double* __restrict__ y, double* __restrict__ f,
               int64_t ld) {
  const int64_t c = (int64_t)blockIdx.x * kRThreads + threadIdx.x;
  if (c >= C) return;
  const int q1 = min(n_r, (int)(blockIdx.y + 1) * kRChunk);
  for (int q = blockIdx.y * kRChunk; q < q1; ++q) {
    const int j = __ldg(col_id + q);
    const int2 a = __ldg(reac + j);
    double v = k[(int64_t)j * ld + c] * y[(int64_t)a.x * ld + c];
    if (a.y >= 0) v *= y[(int64_t)a.y * ld + c];
    const int pe = __ldg(col_ptr + q + 1);
    for (int p = __ldg(col_ptr + q); p < pe; ++p) {
      const uint32_t w = __ldg(ent + p);
      const int cf = (int)(int8_t)(w >> 24);
      double u = v;
      if (cf != 1 && cf != -1) u *= (double)(cf < 0 ? -cf : cf);
      atomicAdd(f + (int64_t)(w & 0xFFFFFFu) * ld + c, neg_if(u, cf < 0));
    }
  }
}

// SELL-C-sigma: block = kCells cells x C slice rows, one slice per blockIdx.y.
__global__ void rhs_sell_kernel(int64_t C, int slice_h, const int* __restrict__ slice_ptr,
                                const uint32_t* __restrict__ ent, const int* __restrict__ row_id,
                                const double* __restrict__ r, int64_t ldr, double* __restrict__ f,
                                int64_t ld) {
  const int cl = threadIdx.x, rr = threadIdx.y, s = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * kCells + cl;
  if (c >= C) return;
  const int i = __ldg(row_id + (int64_t)s * slice_h + rr);
  const int b = __ldg(slice_ptr + s);
  const int L = (__ldg(slice_ptr + s + 1) - b) / slice_h;
  double acc = 0.0;
  for (int kk = 0; kk < L; ++kk) {
    const uint32_t w = __ldg(ent + b + kk * slice_h + rr);
    acc = fma(c_coef[w >> 24], r[(int64_t)(w & 0xFFFFFFu) * ldr + c], acc);
  }
  if (i >= 0) f[(int64_t)i * ld + c] = acc;
}

constexpr int kMaxDevices = 64;
std::atomic<bool> g_coef_ready[kMaxDevices];
std::mutex g_coef_mu;

}  // namespace

// Loads the coefficient decode table into `device`'s constant memory (the
// device must be current).  Called once per device when a network is built,
// so that the right-hand-side launches never issue this synchronous copy;
// thread-safe.
sm_status rhs_prepare_device(int device) {
  if (device < 0 || device >= kMaxDevices) return SM_EINVAL;
  if (g_coef_ready[device].load(std::memory_order_acquire)) return SM_OK;
  std::lock_guard<std::mutex> lock(g_coef_mu);
  if (g_coef_ready[device].load(std::memory_order_relaxed)) return SM_OK;
  double t[256];
  for (int i = 0; i < 256; ++i) t[i] = (double)(int8_t)i;
  SM_TRY_CUDA(cudaMemcpyToSymbol(c_coef, t, sizeof(t)));
  g_coef_ready[device].store(true, std::memory_order_release);
  return SM_OK;
}

namespace {

sm_status ensure_coef_table(int device) {
  if (device >= 0 && device < kMaxDevices && g_coef_ready[device].load(std::memory_order_acquire))
    return SM_OK;
  return rhs_prepare_device(device);
}

}  // namespace

sm_status launch_rhs(const sm_net* net, int64_t C, const double* k, const double* y, double* f,
                     int64_t ld, double* scratch, int64_t ldr, cudaStream_t s) {
  if (C == 0) return SM_OK;
  sm_status st = ensure_coef_table(net->device);
  if (st != SM_OK) return st;
  const Format& F = net->cur;
  const unsigned groups_r = (unsigned)((C + kRThreads - 1) / kRThreads);
  if (F.fmt == SM_FMT_CCS) {
    SM_TRY_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * (size_t)net->n_s * ld, s));
    dim3 grid(groups_r, (unsigned)((net->n_r + kRChunk - 1) / kRChunk));
    rhs_ccs_kernel<<<grid, kRThreads, 0, s>>>(net->n_r, C, F.d_ptr.as<int>(), F.d_packed.as<uint32_t>(),
                                              F.d_aux.as<int>(), net->d_reac.as<int2>(), k, y, f, ld);
    SM_TRY_CUDA(cudaGetLastError());
    return SM_OK;
  }
  {
    dim3 grid(groups_r, (unsigned)((net->n_r + kRChunk - 1) / kRChunk));
    reaction_rate_kernel<<<grid, kRThreads, 0, s>>>(net->n_r, C, net->d_reac.as<int2>(), k, ld, y, ld,
                                                    scratch, ldr, nullptr, 0, nullptr);
    SM_TRY_CUDA(cudaGetLastError());
  }
  const unsigned groups = (unsigned)((C + kCells - 1) / kCells);
  if (F.fmt == SM_FMT_CRS) {
    if ((int)F.chunk_nz.size() != kChunks + 1) return SM_EINVAL;
    rhs_crs_kernel<kCells, kChunks><<<groups, kCells * kChunks, 0, s>>>(net->n_s, C, F.d_ptr.as<int>(),
                                                       F.d_packed.as<uint32_t>(), F.d_aux.as<int>(),
                                                       F.d_chunk.as<int>(), scratch, ldr, f, ld,
                                                       nullptr, 0, nullptr);
  } else if (F.fmt == SM_FMT_COO) {
    SM_TRY_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * (size_t)net->n_s * ld, s));
    const int nnz = (int)F.idx.size();
    dim3 grid(groups_r, (unsigned)((nnz + kRChunk - 1) / kRChunk));
    rhs_coo_kernel<<<grid, kRThreads, 0, s>>>(nnz, C, F.d_packed.as<uint32_t>(), F.d_aux.as<int>(),
                                              scratch, ldr, f, ld);
  } else {
    dim3 block(kCells, F.C);
    dim3 grid(groups, (unsigned)F.len.size());
    rhs_sell_kernel<<<grid, block, 0, s>>>(C, F.C, F.d_ptr.as<int>(), F.d_packed.as<uint32_t>(),
                                           F.d_aux.as<int>(), scratch, ldr, f, ld);
  }
  SM_TRY_CUDA(cudaGetLastError());
  return SM_OK;
}

sm_status launch_rhs_masked(const sm_net* net, int64_t C, const double* k, int64_t ldk,
                            const double* y, double* f, int64_t ld, double* scratch, int64_t ldr,
                            const int* mask, int bit, const int* cact, cudaStream_t s) {
  if (C == 0) return SM_OK;
  sm_status st = ensure_coef_table(net->device);
  if (st != SM_OK) return st;
  const Format& F = net->integ_fmt[net->integ_order];
  if (F.packed.empty()) return SM_EINVAL;
  dim3 grid((unsigned)((C + kRThreads - 1) / kRThreads), (unsigned)((net->n_r + kRChunk - 1) / kRChunk));
  reaction_rate_kernel<<<grid, kRThreads, 0, s>>>(net->n_r, C, net->d_reac.as<int2>(), k, ldk, y, ld,
                                                  scratch, ldr, mask, bit, cact);
  SM_TRY_CUDA(cudaGetLastError());
  const int kc = net->integ_kc;
  const unsigned nb = (unsigned)((C + kc - 1) / kc);
  if (kc == 8) {
    rhs_crs_kernel<8, 64><<<nb, kCells * kChunks, 0, s>>>(net->n_s, C, F.d_ptr.as<int>(),
        F.d_packed.as<uint32_t>(), F.d_aux.as<int>(), F.d_chunk64.as<int>(), scratch, ldr, f, ld, mask, bit, cact);
  } else if (kc == 32) {
    rhs_crs_kernel<32, 16><<<nb, kCells * kChunks, 0, s>>>(net->n_s, C, F.d_ptr.as<int>(),
        F.d_packed.as<uint32_t>(), F.d_aux.as<int>(), F.d_chunk16.as<int>(), scratch, ldr, f, ld, mask, bit, cact);
  } else {
    rhs_crs_kernel<16, 32><<<nb, kCells * kChunks, 0, s>>>(net->n_s, C, F.d_ptr.as<int>(),
        F.d_packed.as<uint32_t>(), F.d_aux.as<int>(), F.d_chunk.as<int>(), scratch, ldr, f, ld, mask, bit, cact);
  }
  SM_TRY_CUDA(cudaGetLastError());
  return SM_OK;
}
