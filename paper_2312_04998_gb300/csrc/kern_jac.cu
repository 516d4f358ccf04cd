// Jacobian values J = S dR/dx on the static pattern, cells as the fast axis.
//
// J_il = sum over reactions j with S_ij != 0 and species l among their
// reactants of S_ij dR_j/dx_l, where dR_j/dx_l = k'_j times the other
// reactant's abundance (2 k'_j x_l for a squared reactant, k'_j for a one-body
// reaction).  The host lists those terms per pattern entry as
// (reaction | coefficient, partner); a half-warp walks a chunk of entries
// (chunks balanced by term count) for 16 cells.
#include "internal.h"

namespace {

constexpr int kCells = 16;
constexpr int kChunksPerCta = 16;  // 8 warps x 2 half-warps

__global__ void __launch_bounds__(kCells * kChunksPerCta)
jac_kernel(int n_chunks, int64_t C, const int* __restrict__ jchunk, const int* __restrict__ jt_ptr,
           const int2* __restrict__ word, const double* __restrict__ k, const double* __restrict__ y,
           double* __restrict__ J, int64_t ld) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ch = blockIdx.y * kChunksPerCta + warp * 2 + (lane >> 4);
  const int64_t c = (int64_t)blockIdx.x * kCells + (lane & 15);
  if (ch >= n_chunks || c >= C) return;
  const int e1 = __ldg(jchunk + ch + 1);
  for (int e = __ldg(jchunk + ch); e < e1; ++e) {
    double acc = 0.0;
    const int t1 = __ldg(jt_ptr + e + 1);
    for (int t = __ldg(jt_ptr + e); t < t1; ++t) {
      const int2 w = __ldg(word + t);
      const int j = w.x & 0xFFFFFF;
      const double cf = (double)(int8_t)((uint32_t)w.x >> 24);
      double d = k[(int64_t)j * ld + c];
      if (w.y >= 0) d *= y[(int64_t)w.y * ld + c];
      acc = fma(cf, d, acc);
    }
    J[(int64_t)e * ld + c] = acc;
  }
}

}  // namespace

sm_status launch_jac(const sm_net* net, int64_t C, const double* k, const double* y, double* J,
                     int64_t ld, cudaStream_t s) {
  if (C == 0) return SM_OK;
  const int n_chunks = (int)net->jchunk.size() - 1;
  dim3 grid((unsigned)((C + kCells - 1) / kCells), (unsigned)((n_chunks + kChunksPerCta - 1) / kChunksPerCta));
  jac_kernel<<<grid, kCells * kChunksPerCta, 0, s>>>(n_chunks, C, net->d_jchunk.as<int>(),
                                                     net->d_jt_ptr.as<int>(), net->d_jt_word.as<int2>(),
                                                     k, y, J, ld);
  SM_TRY_CUDA(cudaGetLastError());
  return SM_OK;
}
