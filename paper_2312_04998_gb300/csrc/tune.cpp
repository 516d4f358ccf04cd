// Autotuner of the stoichiometry traversal used by sm_rhs_eval.
//
// The paper compares COO, CCS, CRS and SELL storage of S with and without
// row reordering (Section 3) and finds the winner depends on the network and
// the machine.  Here the choice is measured: every candidate of a fixed grid
// (format x row order x SELL slice height C and sort window sigma) is built,
// sm_rhs_eval is run on the caller's inputs and timed with CUDA events on the
// caller's stream (one warm-up call, kTrials timed calls, median), and the
// fastest candidate is left selected.  The integrator's own gather (a rate
// pass and a masked CRS gather, run in every Newton iteration) is tuned in
// the same call: CRS in each row order x 8, 16 or 32 cells per CTA (the
// gather's block shape), timed the same way.  Results are cached for the process per (network
// content hash, device name, batch-size bucket = C rounded up to a power of
// two), so a later call with the same key selects the cached format without
// timing anything.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

constexpr int kTrials = 5;

struct Candidate {
  int32_t fmt, order, C, sigma;
};

std::vector<Candidate> candidate_grid(int32_t n_s) {
  std::vector<Candidate> g;
  for (int32_t o : {SM_ORDER_NONE, SM_ORDER_NNZ, SM_ORDER_RCM}) g.push_back({SM_FMT_CRS, o, 1, 1});
  for (int32_t o : {SM_ORDER_NONE, SM_ORDER_RCM}) {
    g.push_back({SM_FMT_COO, o, 1, 1});
    g.push_back({SM_FMT_CCS, o, 1, 1});
  }
  for (int32_t C : {4, 8, 32}) {
    if (C > n_s) continue;
    for (int32_t sigma : {1, std::min(8 * C, n_s), n_s})
      for (int32_t o : {SM_ORDER_NONE, SM_ORDER_RCM}) g.push_back({SM_FMT_SELL, o, C, sigma});
  }
  // drop repeats (a sort window equal to the slice height or the row count)
  std::vector<Candidate> out;
  for (const Candidate& c : g) {
    bool dup = false;
    for (const Candidate& e : out)
      dup = dup || (e.fmt == c.fmt && e.order == c.order && e.C == c.C && e.sigma == c.sigma);
    if (!dup) out.push_back(c);
  }
  return out;
}

// FNV-1a over the network's defining arrays.
uint64_t net_hash(const sm_net* net) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  mix(&net->n_s, sizeof net->n_s);
  mix(&net->n_r, sizeof net->n_r);
  mix(net->comp.data(), net->comp.size() * sizeof(int32_t));
  mix(net->reac.data(), net->reac.size() * sizeof(int32_t));
  mix(net->prod.data(), net->prod.size() * sizeof(int32_t));
  mix(net->cls.data(), net->cls.size());
  return h;
}

int64_t bucket(int64_t C) {
  int64_t b = 1;
  while (b < C) b <<= 1;
  return b;
}

using Key = std::tuple<uint64_t, std::string, int64_t>;
std::mutex g_mu;
std::map<Key, sm_tune_result>& cache() {
  static std::map<Key, sm_tune_result> m;
  return m;
}

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

// Median time (ms) of kTrials sm_rhs_eval calls with the selected format.
sm_status time_rhs(sm_net* net, int64_t C, const double* k, const double* y, double* f, int64_t ld,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* ms_out) {
  sm_status st = sm_rhs_eval(net, C, k, y, f, ld, s);   // warm-up (grows scratch, loads code)
  if (st != SM_OK) return st;
  std::vector<float> t(kTrials);
  for (int i = 0; i < kTrials; ++i) {
    SM_TRY_CUDA(cudaEventRecord(e0, s));
    if ((st = sm_rhs_eval(net, C, k, y, f, ld, s)) != SM_OK) return st;
    SM_TRY_CUDA(cudaEventRecord(e1, s));
    SM_TRY_CUDA(cudaEventSynchronize(e1));
    SM_TRY_CUDA(cudaEventElapsedTime(&t[i], e0, e1));
  }
  std::sort(t.begin(), t.end());
  *ms_out = t[kTrials / 2];
  return SM_OK;
}

// Median time (ms) of kTrials integrator gathers (rate pass + masked CRS
// gather, no mask) with the network's current integrator choice.
sm_status time_integ(sm_net* net, int64_t C, const double* k, const double* y, double* f, int64_t ld,
                     double* scratch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* ms_out) {
  sm_status st = launch_rhs_masked(net, C, k, ld, y, f, ld, scratch, ld, nullptr, 0, nullptr, s);
  if (st != SM_OK) return st;
  std::vector<float> t(kTrials);
  for (int i = 0; i < kTrials; ++i) {
    SM_TRY_CUDA(cudaEventRecord(e0, s));
    if ((st = launch_rhs_masked(net, C, k, ld, y, f, ld, scratch, ld, nullptr, 0, nullptr, s)) != SM_OK) return st;
    SM_TRY_CUDA(cudaEventRecord(e1, s));
    SM_TRY_CUDA(cudaEventSynchronize(e1));
    SM_TRY_CUDA(cudaEventElapsedTime(&t[i], e0, e1));
  }
  std::sort(t.begin(), t.end());
  *ms_out = t[kTrials / 2];
  return SM_OK;
}

// The integrator's gather: CRS in each row order x 8 / 16 / 32 cells per CTA;
// leaves the fastest selected and reports it in *out.
sm_status tune_integ(sm_net* net, int64_t C, const double* k, const double* y, double* f, int64_t ld,
                     cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, sm_tune_result* out) {
  const int64_t ldr = (C + 31) / 32 * 32;
  sm_status st = net->d_scratch.ensure(sizeof(double) * (size_t)net->n_r * (size_t)ldr);
  if (st != SM_OK) return st;
  const int32_t prev_order = net->integ_order, prev_kc = net->integ_kc;
  double best = -1.0;
  for (int32_t o : {SM_ORDER_NONE, SM_ORDER_NNZ, SM_ORDER_RCM}) {
    if ((st = integ_format(net, o)) != SM_OK) break;
    for (int32_t kc : {8, 16, 32}) {
      net->integ_order = o;
      net->integ_kc = kc;
      double ms = 0.0;
      if ((st = time_integ(net, C, k, y, f, ld, net->d_scratch.as<double>(), s, e0, e1, &ms)) != SM_OK) break;
      if (best < 0.0 || ms < best) {
        best = ms;
        out->integ_order = o;
        out->integ_cells_per_cta = kc;
        out->integ_us = ms * 1e3;
      }
    }
    if (st != SM_OK) break;
  }
  if (st != SM_OK) {
    net->integ_order = prev_order;
    net->integ_kc = prev_kc;
    return st;
  }
  net->integ_order = out->integ_order;
  net->integ_kc = out->integ_cells_per_cta;
  return SM_OK;
}

}  // namespace

extern "C" sm_status sm_net_autotune(sm_net* net, int64_t C, const double* d_k, const double* d_y, double* d_f,
                                     int64_t ld, int32_t force, void* stream, sm_tune_result* out) {
  if (!net || net->device < 0 || C < 1 || !ld_ok(C, ld) || !d_k || !d_y || !d_f || !out) return SM_EINVAL;
  Scope scope(net->device);
  if (!scope.ok) return SM_ECUDA;
  cudaDeviceProp prop;
  SM_TRY_CUDA(cudaGetDeviceProperties(&prop, net->device));
  const Key key{net_hash(net), std::string(prop.name), bucket(C)};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = cache().find(key);
    if (!force && it != cache().end()) {
      sm_tune_result r = it->second;
      sm_status st = net_select_format(net, r.fmt, r.order, r.sell_C, r.sell_sigma);
      if (st != SM_OK) return st;
      if ((st = integ_format(net, r.integ_order)) != SM_OK) return st;
      net->integ_order = r.integ_order;
      net->integ_kc = r.integ_cells_per_cta;
      r.cached = 1;
      r.candidates = 0;   // nothing was timed by this call
      *out = r;
      return SM_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Format& cur = net->cur;
  const Candidate prev{cur.fmt, cur.order, cur.C, cur.sigma};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SM_TRY_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SM_ECUDA;
  }
  sm_tune_result best{};
  best.us = -1.0;
  sm_status st = SM_OK;
  const std::vector<Candidate> grid = candidate_grid(net->n_s);
  for (const Candidate& c : grid) {
    if ((st = net_select_format(net, c.fmt, c.order, c.C, c.sigma)) != SM_OK) break;
    double ms = 0.0;
    if ((st = time_rhs(net, C, d_k, d_y, d_f, ld, s, e0, e1, &ms)) != SM_OK) break;
    if (best.us < 0.0 || ms * 1e3 < best.us) {
      best.fmt = c.fmt;
      best.order = c.order;
      best.sell_C = c.C;
      best.sell_sigma = c.sigma;
      best.us = ms * 1e3;
    }
  }
  if (st == SM_OK) st = tune_integ(net, C, d_k, d_y, d_f, ld, s, e0, e1, &best);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SM_OK) {
    // leave the caller's traversal selected, not the failing candidate's
    net_select_format(net, prev.fmt, prev.order, prev.C, prev.sigma);
    return st;
  }
  best.candidates = (int32_t)grid.size() + 9;
  best.cached = 0;
  if ((st = net_select_format(net, best.fmt, best.order, best.sell_C, best.sell_sigma)) != SM_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    cache()[key] = best;
  }
  *out = best;
  return SM_OK;
}
