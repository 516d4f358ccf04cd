// sm_rhs_eval_static: the right-hand side with its per-reaction rate buffer
// in a fixed array compiled into the library, for callers that cannot let the
// library allocate device memory (codes that pre-reserve the device memory for
// their own pool, time-step loops that must not allocate).  The kernels are
// the same as sm_rhs_eval's; only the buffer differs.
#include <mutex>

#include "internal.h"

namespace {

// One fixed buffer per device that loads the library; 32 MiB.
static __device__ __align__(256) double g_rhs_scratch[SM_STATIC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_rhs_scratch on `device` (which must be current).  The
// host-side name of the array is only a stand-in; kernels need this address.
sm_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return SM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) {
      sm_set_last_cuda_error(e, "cudaGetSymbolAddress(g_rhs_scratch)");
      return SM_ECUDA;
    }
    g_addr[device] = static_cast<double*>(p);
  }
  *out = g_addr[device];
  return SM_OK;
}

struct CurrentDevice {
  int prev = -1;
  bool ok = true;
  explicit CurrentDevice(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device) ok = cudaSetDevice(device) == cudaSuccess;
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" sm_status sm_rhs_eval_static(const sm_net* net, int64_t C, const double* d_k,
                                        const double* d_y, double* d_f, int64_t ld, void* stream) {
  if (!net || net->device < 0 || !ld_ok(C, ld)) return SM_EINVAL;
  if (C > 0 && (!d_k || !d_y || !d_f)) return SM_EINVAL;
  if (C == 0) return SM_OK;
  const int64_t ldr = (C + 31) / 32 * 32;
  if ((int64_t)net->n_r * ldr > (int64_t)SM_STATIC_SCRATCH_DOUBLES) return SM_ETOOBIG;
  CurrentDevice cd(net->device);
  if (!cd.ok) return SM_ECUDA;
  double* scratch = nullptr;
  sm_status st = scratch_address(net->device, &scratch);
  if (st != SM_OK) return st;
  return launch_rhs(net, C, d_k, d_y, d_f, ld, scratch, ldr, (cudaStream_t)stream);
}
