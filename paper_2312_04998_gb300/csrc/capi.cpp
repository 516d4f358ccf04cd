// extern "C" entry points of stoich.h: argument checks, device selection and
// dispatch to the host builders and kernel launchers.  No entry point aborts,
// traps or exits; failures come back as sm_status codes.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <new>

#include "internal.h"

namespace {

thread_local char g_last_cuda[256] = {0};

// Makes `device` current for the scope of a call and restores the caller's.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device) ok = cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

void sm_set_last_cuda_error(cudaError_t e, const char* what) {
  std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorString(e), what);
}

sm_status DevArray::upload(const void* h, size_t n) {
  if (n > bytes || !p) {
    release();
    if (n == 0) return SM_OK;
    SM_TRY_CUDA(cudaMalloc(&p, n));
    bytes = n;
  }
  if (n) SM_TRY_CUDA(cudaMemcpy(p, h, n, cudaMemcpyHostToDevice));
  return SM_OK;
}

sm_status DevArray::ensure(size_t n) {
  if (n <= bytes && p) return SM_OK;
  release();
  SM_TRY_CUDA(cudaMalloc(&p, n));
  bytes = n;
  return SM_OK;
}

void DevArray::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

namespace {

void release_all(sm_net* net) {
  if (net->device < 0) return;
  DeviceScope ds(net->device);
  Format& f = net->cur;
  f.d_ptr.release();
  f.d_packed.release();
  f.d_aux.release();
  f.d_chunk.release();
  f.d_chunk64.release();
  f.d_chunk16.release();
  for (Format& g : net->integ_fmt) {
    g.d_ptr.release();
    g.d_packed.release();
    g.d_aux.release();
    g.d_chunk.release();
    g.d_chunk64.release();
    g.d_chunk16.release();
  }
  LUSymbolic& lu = net->lu;
  lu.d_lrptr.release();
  lu.d_lridx.release();
  lu.d_ucptr.release();
  lu.d_ucidx.release();
  lu.d_jrc.release();
  lu.d_uoff.release();
  lu.d_lrhead.release();
  lu.d_lrhoff.release();
  lu.d_u12off.release();
  lu.d_lrhk.release();
  lu.d_srow.release();
  lu.d_u11ptr.release();
  lu.d_hop_ptr.release();
  lu.d_hop.release();
  lu.d_hop_piv.release();
  lu.d_hterm.release();
  lu.d_flev_ptr.release();
  lu.d_flev.release();
  lu.d_blev_ptr.release();
  lu.d_blev.release();
  net->d_jt_slot.release();
  net->d_jdesc.release();
  net->d_jlong.release();
  net->d_sc_ptr.release();
  net->d_sc_ent.release();
  lu.d_lptr.release();
  lu.d_lidx.release();
  lu.d_uptr.release();
  lu.d_uidx.release();
  lu.d_jpos.release();
  lu.d_perm.release();
  lu.d_iperm.release();
  net->d_reac.release();
  net->d_rate.release();
  net->d_jp_ptr.release();
  net->d_jt_ptr.release();
  net->d_jt_word.release();
  net->d_jchunk.release();
  net->d_status.release();
  net->d_scratch.release();
}

bool device_ready(const sm_net* net) { return net && net->device >= 0; }

}  // namespace

extern "C" {

const char* sm_status_str(sm_status s) {
  switch (s) {
    case SM_OK: return "ok";
    case SM_EINVAL: return "invalid argument";
    case SM_ENOMEM: return "out of memory";
    case SM_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case SM_ENOTCONS: return "network does not conserve elements or charge (E.S != 0)";
    case SM_ETIMEOUT: return "a bounded device wait ran out";
    case SM_EPARTIAL: return "some cells failed; see their status";
    case SM_ENOTSUP: return "not supported";
    case SM_ETOOBIG: return "request exceeds the fixed-size internal buffer (see SM_STATIC_SCRATCH_DOUBLES)";
    default: return "unknown status";
  }
}

sm_status sm_net_build(const sm_net_desc* d, int32_t device, sm_net** out) {
  if (!out) return SM_EINVAL;
  *out = nullptr;
  sm_net* net = new (std::nothrow) sm_net();
  if (!net) return SM_ENOMEM;
  net->device = device;
  sm_status st = net_build_host(d, net);
  if (st == SM_OK && device >= 0) {
    DeviceScope ds(device);
    if (!ds.ok) st = SM_ECUDA;
    if (st == SM_OK) st = net_upload(net);
    if (st == SM_OK) st = net_select_format(net, SM_FMT_CRS, SM_ORDER_NONE, 1, 1);
  } else if (st == SM_OK) {
    st = net_select_format(net, SM_FMT_CRS, SM_ORDER_NONE, 1, 1);
  }
  if (st != SM_OK) {
    release_all(net);
    delete net;
    return st;
  }
  *out = net;
  return SM_OK;
}

sm_status sm_net_free(sm_net* net) {
  if (!net) return SM_EINVAL;
  release_all(net);
  delete net;
  return SM_OK;
}

sm_status sm_net_set_format(sm_net* net, int32_t fmt, int32_t order, int32_t sell_C,
                            int32_t sell_sigma) {
  if (!net) return SM_EINVAL;
  if (net->device >= 0) {
    DeviceScope ds(net->device);
    if (!ds.ok) return SM_ECUDA;
    return net_select_format(net, fmt, order, sell_C, sell_sigma);
  }
  return net_select_format(net, fmt, order, sell_C, sell_sigma);
}

sm_status sm_net_set_thermal(sm_net* net, const sm_thermal* th) {
  if (!net) return SM_EINVAL;
  if (!th) {
    net->th_t = -1;
    net->th_L.clear();
    net->th_E.clear();
    return SM_OK;
  }
  const int32_t t = th->t_index, n = net->n_s, ne = net->n_elem + 1;
  if (t < 0 || t >= n || !th->L || !th->E) return SM_EINVAL;
  auto ok = [](double v) { return std::isfinite(v) && v >= 0.0; };
  if (!ok(th->heat) || !ok(th->lam) || !ok(th->T_dust) || !ok(th->zeta)) return SM_EINVAL;
  for (int32_t e = 0; e < ne; ++e)
    if (net->comp[(size_t)t * ne + e] != 0) return SM_EINVAL;   // no atoms, no charge
  for (int32_t v : net->reac)
    if (v == t) return SM_EINVAL;                                // in no reaction
  for (int32_t v : net->prod)
    if (v == t) return SM_EINVAL;
  for (int32_t i = 0; i < n; ++i) {
    if (!ok(th->L[i])) return SM_EINVAL;
    if (th->L[i] > 0.0 && !(std::isfinite(th->E[i]) && th->E[i] > 0.0)) return SM_EINVAL;
  }
  net->th_L.assign(th->L, th->L + n);
  net->th_E.assign(th->E, th->E + n);
  net->th_L[t] = 0.0;
  for (int32_t i = 0; i < n; ++i)
    if (net->th_L[i] == 0.0) net->th_E[i] = 1.0;
  net->th_heat = th->heat;
  net->th_lam = th->lam;
  net->th_Td = th->T_dust;
  net->th_zeta = th->zeta;
  net->th_t = t;
  return SM_OK;
}

sm_status sm_net_set_integ(sm_net* net, int32_t order, int32_t cells_per_cta) {
  if (!net || order < SM_ORDER_NONE || order > SM_ORDER_RCM ||
      (cells_per_cta != 8 && cells_per_cta != 16 && cells_per_cta != 32))
    return SM_EINVAL;
  sm_status st;
  if (net->device >= 0) {
    DeviceScope ds(net->device);
    if (!ds.ok) return SM_ECUDA;
    st = integ_format(net, order);
  } else {
    st = integ_format(net, order);
  }
  if (st != SM_OK) return st;
  net->integ_order = order;
  net->integ_kc = cells_per_cta;
  return SM_OK;
}

sm_status sm_net_get_info(const sm_net* net, sm_net_info* info) {
  if (!net || !info) return SM_EINVAL;
  *info = net->info;
  return SM_OK;
}

static sm_status export_view(const sm_net* net, int32_t what, const void** src, size_t* bytes) {
  const Format& f = net->cur;
  const bool crs = f.fmt == SM_FMT_CRS, ccs = f.fmt == SM_FMT_CCS, coo = f.fmt == SM_FMT_COO,
             sell = f.fmt == SM_FMT_SELL;
  auto v32 = [&](const std::vector<int32_t>& v) {
    *src = v.data();
    *bytes = v.size() * 4;
    return SM_OK;
  };
  switch (what) {
    case SM_X_ROW_ORDER: return v32(net->row_order[f.order]);
    case SM_X_COL_ORDER: return v32(net->col_order[f.order]);
    case SM_X_FMT_PTR:
      if (coo) return SM_EINVAL;
      return v32(f.ptr);
    case SM_X_FMT_IDX: return v32(f.idx);
    case SM_X_FMT_IDX2:
      if (!(coo || sell)) return SM_EINVAL;
      return v32(f.idx2);
    case SM_X_FMT_VAL:
      *src = f.val.data();
      *bytes = f.val.size() * 8;
      return SM_OK;
    case SM_X_FMT_LEN:
      if (!sell) return SM_EINVAL;
      return v32(f.len);
    case SM_X_JPAT_PTR: return v32(net->jp_ptr);
    case SM_X_JPAT_COL: return v32(net->jp_col);
    case SM_X_LU_PERM: return v32(net->lu.perm);
    default: (void)crs; (void)ccs; return SM_EINVAL;
  }
}

sm_status sm_net_export_size(const sm_net* net, int32_t what, size_t* bytes) {
  if (!net || !bytes) return SM_EINVAL;
  const void* src = nullptr;
  return export_view(net, what, &src, bytes);
}

sm_status sm_net_export(const sm_net* net, int32_t what, void* h_buf, size_t bytes) {
  if (!net || (!h_buf && bytes)) return SM_EINVAL;
  const void* src = nullptr;
  size_t n = 0;
  sm_status st = export_view(net, what, &src, &n);
  if (st != SM_OK) return st;
  if (bytes < n) return SM_EINVAL;
  if (n) std::memcpy(h_buf, src, n);
  return SM_OK;
}

sm_status sm_rates_eval(const sm_net* net, int64_t C, const double* d_T, const double* d_nH,
                        const double* d_Av, double zeta, double* d_k, int64_t ld, void* stream) {
  if (!device_ready(net) || !ld_ok(C, ld)) return SM_EINVAL;
  if (C > 0 && (!d_T || !d_nH || !d_Av || !d_k)) return SM_EINVAL;
  DeviceScope ds(net->device);
  if (!ds.ok) return SM_ECUDA;
  return launch_rates(net, C, d_T, d_nH, d_Av, nullptr, zeta, d_k, ld, (cudaStream_t)stream);
}

sm_status sm_rates_eval_chi(const sm_net* net, int64_t C, const double* d_T, const double* d_nH,
                            const double* d_Av, const double* d_chi, double zeta, double* d_k, int64_t ld,
                            void* stream) {
  if (!device_ready(net) || !ld_ok(C, ld)) return SM_EINVAL;
  if (C > 0 && (!d_T || !d_nH || !d_Av || !d_k)) return SM_EINVAL;
  DeviceScope ds(net->device);
  if (!ds.ok) return SM_ECUDA;
  return launch_rates(net, C, d_T, d_nH, d_Av, d_chi, zeta, d_k, ld, (cudaStream_t)stream);
}

sm_status sm_rhs_eval(const sm_net* net, int64_t C, const double* d_k, const double* d_y,
                      double* d_f, int64_t ld, void* stream) {
  if (!device_ready(net) || !ld_ok(C, ld)) return SM_EINVAL;
  if (C > 0 && (!d_k || !d_y || !d_f)) return SM_EINVAL;
  if (C == 0) return SM_OK;
  DeviceScope ds(net->device);
  if (!ds.ok) return SM_ECUDA;
  sm_net* m = const_cast<sm_net*>(net);  // the rate scratch is library-owned workspace
  const int64_t ldr = (C + 31) / 32 * 32;
  sm_status st = m->d_scratch.ensure(sizeof(double) * (size_t)net->n_r * (size_t)ldr);
  if (st != SM_OK) return st;
  return launch_rhs(net, C, d_k, d_y, d_f, ld, m->d_scratch.as<double>(), ldr, (cudaStream_t)stream);
}

sm_status sm_jac_eval(const sm_net* net, int64_t C, const double* d_k, const double* d_y,
                      double* d_J, int64_t ld, void* stream) {
  if (!device_ready(net) || !ld_ok(C, ld)) return SM_EINVAL;
  if (C > 0 && (!d_k || !d_y || !d_J)) return SM_EINVAL;
  DeviceScope ds(net->device);
  if (!ds.ok) return SM_ECUDA;
  return launch_jac(net, C, d_k, d_y, d_J, ld, (cudaStream_t)stream);
}

sm_status sm_sync(const sm_net* net, void* stream) {
  if (!device_ready(net)) return SM_EINVAL;
  DeviceScope ds(net->device);
  if (!ds.ok) return SM_ECUDA;
  SM_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int32_t word = 0;
  SM_TRY_CUDA(cudaMemcpy(&word, net->d_status.p, 4, cudaMemcpyDeviceToHost));
  if (word != DEV_ERR_NONE) {
    int32_t zero = 0;
    SM_TRY_CUDA(cudaMemcpy(net->d_status.p, &zero, 4, cudaMemcpyHostToDevice));
    return (word & DEV_ERR_TIMEOUT) ? SM_ETIMEOUT : SM_EINVAL;
  }
  return SM_OK;
}

}  // extern "C"
