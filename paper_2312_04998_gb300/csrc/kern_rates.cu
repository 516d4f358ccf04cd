// Rate coefficients k'[n_r][ld], cells as the fast axis.
//
// The paper precomputes the coefficients outside the stiff solver, once per
// hydro step (Section 3); here one thread owns one cell for a chunk of
// reactions, so log(T/300) and 1/T are formed once per chunk and every
// reaction costs one exp.  Reaction parameters are warp-uniform broadcasts.
#include "internal.h"

namespace {

constexpr int kRatesThreads = 128;
constexpr int kRatesChunk = 64;

__global__ void __launch_bounds__(kRatesThreads)
rates_kernel(int n_r, int64_t C, const RatePar* __restrict__ par, const double* __restrict__ T,
             const double* __restrict__ nH, const double* __restrict__ Av, const double* __restrict__ chi,
             double zeta, double* __restrict__ k, int64_t ld) {
  const int64_t c = (int64_t)blockIdx.x * kRatesThreads + threadIdx.x;
  if (c >= C) return;
  const int j0 = blockIdx.y * kRatesChunk;
  const int j1 = min(n_r, j0 + kRatesChunk);
  const double t = T[c], n = nH[c], av = Av[c];
  const double fuv = chi ? chi[c] : 1.0;   // FUV field on the photorates
  const double lt = log(t * (1.0 / 300.0));
  const double it = 1.0 / t;
  for (int j = j0; j < j1; ++j) {
    const RatePar p = par[j];  // (log alpha | alpha, beta, gamma, class)
    const int cls = (int)p.w;
    double v;
    if (cls == SM_TWO_BODY || cls == SM_DISS_RECOMB) {
      v = exp(fma(p.y, lt, p.x) - p.z * it) * n;
    } else if (cls == SM_COSMIC_RAY) {
      v = p.x * zeta;
    } else {
      v = fuv * p.x * exp(-p.z * av);
    }
    k[(int64_t)j * ld + c] = v;
  }
}

}  // namespace

sm_status launch_rates(const sm_net* net, int64_t C, const double* T, const double* nH,
                       const double* Av, const double* chi, double zeta, double* k, int64_t ld, cudaStream_t s) {
  if (C == 0) return SM_OK;
  dim3 grid((unsigned)((C + kRatesThreads - 1) / kRatesThreads),
            (unsigned)((net->n_r + kRatesChunk - 1) / kRatesChunk));
  rates_kernel<<<grid, kRatesThreads, 0, s>>>(net->n_r, C, net->d_rate.as<RatePar>(), T, nH, Av, chi,
                                               zeta, k, ld);
  SM_TRY_CUDA(cudaGetLastError());
  return SM_OK;
}
