// Arithmetic-throughput probe of the device's FP64 and FP32 FMA pipes.
//
// The chemistry kernels are bound by FP64 arithmetic (the right-hand side,
// the Jacobian and the Newton residual accumulate in FP64) or by FP32
// arithmetic (the reduced-precision factorisation), not by HBM.  Their
// roofline needs the rate those pipes actually sustain; this kernel measures
// it: every thread runs kChains independent FMA dependency chains, so the
// pipe, not the FMA latency, limits the issue rate, with several CTAs per SM
// on every SM.
#include <algorithm>

#include "internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;
constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T* __restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int u = 0; u < kChains; ++u) x[u] = T(1) + T(threadIdx.x + u) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kChains; ++u) x[u] = fma(x[u], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int u = 0; u < kChains; ++u) s += x[u];
  out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

template <class T>
sm_status probe(int sms, int iters, double* tflops) {
  const int ctas = sms * kProbeCtasPerSm;
  T* out = nullptr;
  SM_TRY_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)ctas * kProbeThreads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sm_status r = SM_OK;
  float best = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = SM_ECUDA;
  // x <- x a + b with a slightly below 1 stays near b / (1 - a): no overflow,
  // no subnormals
  const T a = T(0.999999), b = T(1e-6);
  for (int rep = 0; rep < 4 && r == SM_OK; ++rep) {
    if (cudaEventRecord(e0, 0) != cudaSuccess) { r = SM_ECUDA; break; }
    fma_probe_kernel<T><<<ctas, kProbeThreads>>>(out, iters, a, b);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, 0) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess) {
      r = SM_ECUDA;
      break;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { r = SM_ECUDA; break; }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // the first launch is a warm-up
  }
  if (r == SM_OK) {
    const double flops = 2.0 * kChains * (double)iters * ctas * kProbeThreads;
    *tflops = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return r;
}

}  // namespace

extern "C" sm_status sm_probe_fma(int32_t device, int32_t fp64, double* tflops) {
  if (!tflops || device < 0) return SM_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(device) != cudaSuccess) return SM_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  sms = std::max(sms, 1);
  // about 30 ms per launch at the expected rates (FP64 ~1.2, FP32 ~70 TFLOP/s)
  const sm_status r = fp64 ? probe<double>(sms, 1 << 13, tflops) : probe<float>(sms, 1 << 18, tflops);
  if (prev >= 0) cudaSetDevice(prev);
  return r;
}
