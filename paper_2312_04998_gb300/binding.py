"""Thin ctypes binding of libstoich.so (include/stoich.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream; batched
arrays are [n][ld] tensors (cells fastest, ld a multiple of 32) of which the
first C columns are used.  If the library is missing the import fails loudly;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstoich.so")
# libstoich_phases.so (the phase-clock profiling build) when STOICH_PHASES=1
if os.environ.get("STOICH_PHASES") == "1":
    LIB_PATH = os.path.join(_PKG, "libstoich_phases.so")

SM_OK, SM_EINVAL, SM_ENOMEM, SM_ECUDA, SM_ENOTCONS, SM_ETIMEOUT, SM_EPARTIAL, SM_ENOTSUP, SM_ETOOBIG = range(9)
STATIC_SCRATCH_DOUBLES = 4194304
FMT = {"crs": 0, "coo": 1, "ccs": 2, "sell": 3}
ORDER = {"none": 0, "nnz": 1, "rcm": 2}
X_ROW_ORDER, X_COL_ORDER, X_FMT_PTR, X_FMT_IDX, X_FMT_IDX2, X_FMT_VAL, X_FMT_LEN, \
    X_JPAT_PTR, X_JPAT_COL, X_LU_PERM = range(10)


class StoichError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {status_str(code)} (status {code})")
        self.code = code


class NetDesc_c(ct.Structure):
    _fields_ = [("n_s", ct.c_int32), ("n_r", ct.c_int32), ("n_elem", ct.c_int32),
                ("comp", ct.POINTER(ct.c_int32)), ("reactants", ct.POINTER(ct.c_int32)),
                ("products", ct.POINTER(ct.c_int32)), ("rclass", ct.POINTER(ct.c_int8)),
                ("alpha", ct.POINTER(ct.c_double)), ("beta", ct.POINTER(ct.c_double)),
                ("gamma", ct.POINTER(ct.c_double))]


class NetInfo_c(ct.Structure):
    _fields_ = [("n_s", ct.c_int32), ("n_r", ct.c_int32), ("nnz_S", ct.c_int64),
                ("nnz_J", ct.c_int64), ("n_jac_terms", ct.c_int64), ("nnz_LU", ct.c_int64),
                ("lu_flops", ct.c_int64), ("lu_head", ct.c_int32), ("max_row_nnz", ct.c_int32),
                ("fmt", ct.c_int32), ("order", ct.c_int32), ("sell_C", ct.c_int32),
                ("sell_sigma", ct.c_int32), ("fmt_entries", ct.c_int64), ("rhs_bytes", ct.c_double),
                ("rhs_flops", ct.c_double), ("jac_bytes", ct.c_double), ("jac_flops", ct.c_double),
                ("lu_packed", ct.c_int64)]


class TuneResult_c(ct.Structure):
    _fields_ = [("fmt", ct.c_int32), ("order", ct.c_int32), ("sell_C", ct.c_int32), ("sell_sigma", ct.c_int32),
                ("us", ct.c_double), ("candidates", ct.c_int32), ("cached", ct.c_int32),
                ("integ_order", ct.c_int32), ("integ_cells_per_cta", ct.c_int32), ("integ_us", ct.c_double)]


class Thermal_c(ct.Structure):
    _fields_ = [("t_index", ct.c_int32), ("heat", ct.c_double), ("lam", ct.c_double), ("T_dust", ct.c_double),
                ("zeta", ct.c_double), ("L", ct.c_void_p), ("E", ct.c_void_p)]


class Opts_c(ct.Structure):
    _fields_ = [("rtol", ct.c_double), ("atol", ct.c_double), ("gamma_tol", ct.c_double),
                ("newton_tol", ct.c_double), ("eta_max", ct.c_double), ("eta_keep", ct.c_double),
                ("q_max", ct.c_int32), ("max_steps", ct.c_int32), ("j_age_max", ct.c_int32),
                ("newton_max", ct.c_int32), ("max_conv_fails", ct.c_int32), ("precision", ct.c_int32),
                ("use_graph", ct.c_int32), ("attempts_per_sync", ct.c_int32),
                ("timing_kind", ct.c_int32), ("record_steps", ct.c_int32), ("refresh_ctas_per_sm", ct.c_int32)]


CELL_STATS_DTYPE = np.dtype([("status", np.int32), ("steps", np.int32), ("rejects", np.int32),
                             ("conv_fails", np.int32), ("newton_iters", np.int32),
                             ("jac_evals", np.int32), ("q_last", np.int32), ("pad", np.int32),
                             ("t", np.float64), ("h", np.float64)])
PREC = {"fp64": 0, "mixed": 1, "tf32": 2}
TIME = {"none": 0, "refresh": 1, "rhs": 2, "solve": 3, "predict": 4, "finish": 5}
CELL_OK, CELL_MAXSTEPS, CELL_HMIN, CELL_CONV, CELL_NAN, CELL_RUNNING = range(6)

_lib = None

# (name, restype, argtypes) of every exported entry point.
_SIGS = [
    ("sm_status_str", ct.c_char_p, [ct.c_int32]),
    ("sm_net_build", ct.c_int32, [ct.POINTER(NetDesc_c), ct.c_int32, ct.POINTER(ct.c_void_p)]),
    ("sm_net_free", ct.c_int32, [ct.c_void_p]),
    ("sm_synth_network", ct.c_int32, [ct.c_uint64, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                      ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    ("sm_net_build_synthetic", ct.c_int32, [ct.c_uint64, ct.c_int32, ct.c_int32, ct.c_int32,
                                            ct.POINTER(ct.c_void_p)]),
    ("sm_net_set_format", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32]),
    ("sm_net_get_info", ct.c_int32, [ct.c_void_p, ct.POINTER(NetInfo_c)]),
    ("sm_net_set_integ", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.c_int32]),
    ("sm_net_set_thermal", ct.c_int32, [ct.c_void_p, ct.POINTER(Thermal_c)]),
    ("sm_state_set_cells", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                        ct.c_void_p]),
    ("sm_net_autotune", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                     ct.c_int64, ct.c_int32, ct.c_void_p, ct.POINTER(TuneResult_c)]),
    ("sm_net_export_size", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_size_t)]),
    ("sm_net_export", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_size_t]),
    ("sm_rates_eval", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                   ct.c_double, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    ("sm_rates_eval_chi", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                       ct.c_void_p, ct.c_double, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    ("sm_rhs_eval", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                 ct.c_int64, ct.c_void_p]),
    ("sm_rhs_eval_static", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                        ct.c_int64, ct.c_void_p]),
    ("sm_jac_eval", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                 ct.c_int64, ct.c_void_p]),
    ("sm_sync", ct.c_int32, [ct.c_void_p, ct.c_void_p]),
    ("sm_probe_fma", ct.c_int32, [ct.c_int32, ct.c_int32, ct.POINTER(ct.c_double)]),
    ("sm_phase_cycles", ct.c_int32, [ct.c_int32, ct.c_void_p, ct.c_int32]),
    ("sm_opts_default", None, [ct.POINTER(Opts_c)]),
    ("sm_state_create", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.POINTER(Opts_c), ct.POINTER(ct.c_void_p)]),
    ("sm_state_free", ct.c_int32, [ct.c_void_p]),
    ("sm_state_bytes", ct.c_int32, [ct.c_void_p, ct.POINTER(ct.c_size_t)]),
    ("sm_integrate", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_int64,
                                  ct.c_double, ct.c_void_p, ct.c_void_p]),
    ("sm_state_init", ct.c_int32, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_int64,
                                   ct.c_double, ct.c_void_p]),
    ("sm_state_timing", ct.c_int32, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double),
                                     ct.POINTER(ct.c_int64)]),
    ("sm_state_timing_reset", ct.c_int32, [ct.c_void_p]),
    ("sm_step_bdf", ct.c_int32, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_void_p]),
    ("sm_state_read", ct.c_int32, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p,
                                   ct.POINTER(ct.c_int64), ct.c_void_p]),
    ("sm_state_save", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_size_t, ct.POINTER(ct.c_size_t),
                                   ct.c_void_p]),
    ("sm_state_load", ct.c_int32, [ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    ("sm_state_steps", ct.c_int32, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                    ct.c_int64, ct.c_void_p]),
    ("sm_adjoint", ct.c_int32, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int32,
                                ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    ("sm_replay", ct.c_int32, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p,
                               ct.c_int64, ct.c_void_p]),
]
ADJ_MAX_COT = 64
CHECKPOINT_EVERY = 16


def lib():
    """Load libstoich.so once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ct.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().sm_status_str(int(code)).decode()


def _check(code, what):
    if code != SM_OK:
        raise StoichError(code, what)


def _ptr(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


def _dptr(t):
    return ct.c_void_p(t.data_ptr())


def _stream(device):
    import torch
    return ct.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def pad_ld(C: int) -> int:
    return max(32, (int(C) + 31) // 32 * 32)


class Network:
    """An uploaded network (sm_net).  device=-1 builds host structures only
    (formats, orders, Jacobian pattern) for inspection without a GPU."""

    def __init__(self, desc, device: int = 0):
        L = lib()
        self._keep = dict(
            comp=np.ascontiguousarray(desc.comp, dtype=np.int32),
            reac=np.ascontiguousarray(desc.reactants, dtype=np.int32),
            prod=np.ascontiguousarray(desc.products, dtype=np.int32),
            cls=np.ascontiguousarray(desc.rclass, dtype=np.int8),
            alpha=np.ascontiguousarray(desc.alpha, dtype=np.float64),
            beta=np.ascontiguousarray(desc.beta, dtype=np.float64),
            gamma=np.ascontiguousarray(desc.gamma, dtype=np.float64))
        k = self._keep
        n_s, n_r = k["comp"].shape[0], k["reac"].shape[0]
        d = NetDesc_c(n_s, n_r, k["comp"].shape[1] - 1, _ptr(k["comp"], ct.c_int32),
                      _ptr(k["reac"], ct.c_int32), _ptr(k["prod"], ct.c_int32),
                      _ptr(k["cls"], ct.c_int8), _ptr(k["alpha"], ct.c_double),
                      _ptr(k["beta"], ct.c_double), _ptr(k["gamma"], ct.c_double))
        h = ct.c_void_p()
        _check(L.sm_net_build(ct.byref(d), int(device), ct.byref(h)), "sm_net_build")
        self.h = h
        self.device = device
        self.n_s, self.n_r = n_s, n_r

    @classmethod
    def synthetic(cls, seed: int, n_s: int, n_r: int, device: int = 0):
        """A network drawn and built inside the library (sm_net_build_synthetic)."""
        self = cls.__new__(cls)
        h = ct.c_void_p()
        _check(lib().sm_net_build_synthetic(int(seed), int(n_s), int(n_r), int(device), ct.byref(h)),
               "sm_net_build_synthetic")
        self.h, self.device, self.n_s, self.n_r, self._keep = h, device, n_s, n_r, {}
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().sm_net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_format(self, fmt="crs", order="none", C=1, sigma=1):
        _check(lib().sm_net_set_format(self.h, FMT[fmt], ORDER[order], int(C), int(sigma)),
               "sm_net_set_format")

    def info(self) -> dict:
        inf = NetInfo_c()
        _check(lib().sm_net_get_info(self.h, ct.byref(inf)), "sm_net_get_info")
        return {name: getattr(inf, name) for name, _ in NetInfo_c._fields_}

    def export(self, what: int, dtype=np.int32) -> np.ndarray:
        n = ct.c_size_t()
        _check(lib().sm_net_export_size(self.h, what, ct.byref(n)), "sm_net_export_size")
        out = np.empty(n.value // np.dtype(dtype).itemsize, dtype=dtype)
        _check(lib().sm_net_export(self.h, what, out.ctypes.data_as(ct.c_void_p), n.value),
               "sm_net_export")
        return out

    # ---- batched device calls: torch tensors [n][ld], first C columns used ----

    def _ld(self, *tensors):
        ld = tensors[0].stride(0)
        for t in tensors:
            if t.stride(0) != ld or t.stride(-1) != 1:
                raise ValueError("batched tensors must share the row stride ld with unit column stride")
        return ld

    def rates_eval_chi(self, T, nH, Av, chi, k, C=None, zeta=1.3e-17):
        """sm_rates_eval_chi: photorates scaled by the per-cell FUV field chi
        (device tensor, or None for 1)."""
        C = T.shape[0] if C is None else C
        _check(lib().sm_rates_eval_chi(self.h, int(C), _dptr(T), _dptr(nH), _dptr(Av),
                                       _dptr(chi) if chi is not None else None, float(zeta),
                                       _dptr(k), int(self._ld(k)), _stream(k.device)), "sm_rates_eval_chi")

    def rates_eval(self, T, nH, Av, k, C=None, zeta=1.3e-17):
        C = T.shape[0] if C is None else C
        _check(lib().sm_rates_eval(self.h, int(C), _dptr(T), _dptr(nH), _dptr(Av), float(zeta),
                                   _dptr(k), int(self._ld(k)), _stream(k.device)), "sm_rates_eval")
        return k

    def autotune(self, k, y, f, C, force=False):
        """Times sm_rhs_eval over the candidate traversals on these device
        arrays and leaves the fastest selected; returns the choice as a dict."""
        r = TuneResult_c()
        _check(lib().sm_net_autotune(self.h, int(C), _dptr(k), _dptr(y), _dptr(f), int(self._ld(k, y, f)),
                                     int(bool(force)), _stream(y.device), ct.byref(r)), "sm_net_autotune")
        inv_f = {v: k_ for k_, v in FMT.items()}
        inv_o = {v: k_ for k_, v in ORDER.items()}
        return {"fmt": inv_f[r.fmt], "order": inv_o[r.order], "sell_C": r.sell_C, "sell_sigma": r.sell_sigma,
                "us": r.us, "candidates": r.candidates, "cached": bool(r.cached),
                "integ_order": inv_o[r.integ_order], "integ_cells_per_cta": r.integ_cells_per_cta,
                "integ_us": r.integ_us}

    def set_integ(self, order="none", cells_per_cta=16):
        """The integrator's gather: CRS row order and cells per CTA (8, 16, 32)."""
        _check(lib().sm_net_set_integ(self.h, ORDER[order], int(cells_per_cta)), "sm_net_set_integ")

    def set_thermal(self, th):
        """Couple the gas temperature (sm_net_set_thermal); th has t_index, L,
        E, heat, lam, T_dust and zeta (None turns it off)."""
        if th is None:
            _check(lib().sm_net_set_thermal(self.h, None), "sm_net_set_thermal")
            return
        L = np.ascontiguousarray(th.L, dtype=np.float64)
        E = np.ascontiguousarray(th.E, dtype=np.float64)
        c = Thermal_c(int(th.t_index), float(th.heat), float(th.lam), float(th.T_dust), float(th.zeta),
                      L.ctypes.data, E.ctypes.data)
        _check(lib().sm_net_set_thermal(self.h, ct.byref(c)), "sm_net_set_thermal")

    def rhs_eval(self, k, y, f, C):
        ld = self._ld(k, y, f)
        _check(lib().sm_rhs_eval(self.h, int(C), _dptr(k), _dptr(y), _dptr(f), int(ld),
                                 _stream(f.device)), "sm_rhs_eval")
        return f

    def rhs_eval_static(self, k, y, f, C):
        """sm_rhs_eval_static: same result as rhs_eval, no device allocation."""
        ld = self._ld(k, y, f)
        _check(lib().sm_rhs_eval_static(self.h, int(C), _dptr(k), _dptr(y), _dptr(f), int(ld),
                                        _stream(f.device)), "sm_rhs_eval_static")
        return f

    def jac_eval(self, k, y, J, C):
        ld = self._ld(k, y, J)
        _check(lib().sm_jac_eval(self.h, int(C), _dptr(k), _dptr(y), _dptr(J), int(ld),
                                 _stream(J.device)), "sm_jac_eval")
        return J

    def sync(self):
        import torch
        _check(lib().sm_sync(self.h, _stream(torch.device("cuda", self.device))), "sm_sync")


def synth_network(seed: int, n_s: int, n_r: int) -> dict:
    """The library's seeded synthetic network arrays (sm_synth_network)."""
    comp = np.zeros((n_s, 4), dtype=np.int32)
    reac = np.zeros((n_r, 2), dtype=np.int32)
    prod = np.zeros((n_r, 4), dtype=np.int32)
    cls = np.zeros(n_r, dtype=np.int8)
    alpha, beta, gamma = np.zeros(n_r), np.zeros(n_r), np.zeros(n_r)
    _check(lib().sm_synth_network(int(seed), int(n_s), int(n_r), comp.ctypes.data, reac.ctypes.data,
                                  prod.ctypes.data, cls.ctypes.data, alpha.ctypes.data, beta.ctypes.data,
                                  gamma.ctypes.data), "sm_synth_network")
    return {"comp": comp, "reactants": reac, "products": prod, "rclass": cls, "alpha": alpha, "beta": beta,
            "gamma": gamma}


def default_opts(**kw) -> Opts_c:
    o = Opts_c()
    lib().sm_opts_default(ct.byref(o))
    for key, v in kw.items():
        if key == "precision" and isinstance(v, str):
            v = PREC[v]
        if key == "timing_kind" and isinstance(v, str):
            v = TIME[v]
        setattr(o, key, v)
    return o


class State:
    """Integrator workspace (sm_state) for up to `cells` cells of `net`."""

    def __init__(self, net: Network, cells: int, **opts):
        self.net = net
        self.opts = default_opts(**opts)
        h = ct.c_void_p()
        _check(lib().sm_state_create(net.h, int(cells), ct.byref(self.opts), ct.byref(h)),
               "sm_state_create")
        self.h = h
        self.cells = cells
        self.generation = 0   # counts integrations (autograd checks its record is current)

    def close(self):
        if getattr(self, "h", None):
            lib().sm_state_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def timing(self):
        """(kernel launches so far, summed ms of the timed class, timed launches)."""
        n, ms, t = ct.c_int64(), ct.c_double(), ct.c_int64()
        _check(lib().sm_state_timing(self.h, ct.byref(n), ct.byref(ms), ct.byref(t)), "sm_state_timing")
        return n.value, ms.value, t.value

    def timing_reset(self):
        _check(lib().sm_state_timing_reset(self.h), "sm_state_timing_reset")

    def nbytes(self) -> int:
        n = ct.c_size_t()
        _check(lib().sm_state_bytes(self.h, ct.byref(n)), "sm_state_bytes")
        return n.value

    def set_cells(self, nH, Av, chi=None, C=None):
        """Cell conditions of a thermal state (device FP64 arrays of >= C)."""
        C = nH.shape[0] if C is None else C
        _check(lib().sm_state_set_cells(self.h, int(C), _dptr(nH), _dptr(Av),
                                        _dptr(chi) if chi is not None else None, _stream(nH.device)),
               "sm_state_set_cells")

    def integrate(self, k, y, t_end, C=None, stats=None, allow_partial=True):
        """Integrate C cells from t = 0 to t_end; y (device [n_s][ld]) is
        overwritten.  stats: optional device uint8 tensor of C*48 bytes.
        k may be None for a thermal state.  Returns the status code (SM_OK
        or SM_EPARTIAL)."""
        C = y.shape[1] if C is None else C
        ld = self.net._ld(k, y) if k is not None else self.net._ld(y)
        self.generation += 1
        code = lib().sm_integrate(self.h, int(C), _dptr(k) if k is not None else None, _dptr(y), int(ld),
                                  float(t_end),
                                  _dptr(stats) if stats is not None else None, _stream(y.device))
        if code == SM_EPARTIAL and allow_partial:
            return code
        _check(code, "sm_integrate")
        return code

    def init(self, k, y, t_end, C=None):
        C = y.shape[1] if C is None else C
        self.generation += 1
        ld = self.net._ld(k, y) if k is not None else self.net._ld(y)
        _check(lib().sm_state_init(self.h, int(C), _dptr(k) if k is not None else None, _dptr(y), int(ld),
                                   float(t_end), _stream(y.device)), "sm_state_init")

    def step(self, k, attempts, device=None):
        """attempts BDF attempts; k may be None for a thermal state (then
        device, default the network's, selects the stream)."""
        import torch
        dev = k.device if k is not None else torch.device("cuda", self.net.device if device is None else device)
        _check(lib().sm_step_bdf(self.h, _dptr(k) if k is not None else None,
                                 int(k.stride(0)) if k is not None else 32, int(attempts), _stream(dev)),
               "sm_step_bdf")

    def read(self, y=None, stats=None):
        running = ct.c_int64()
        import torch
        dev = y.device if y is not None else torch.device("cuda", self.net.device)
        _check(lib().sm_state_read(self.h, _dptr(y) if y is not None else None,
                                   int(y.stride(0)) if y is not None else 32,
                                   _dptr(stats) if stats is not None else None, ct.byref(running),
                                   _stream(dev)), "sm_state_read")
        return running.value


    def save(self, with_factors=True):
        """Host image of the state (numpy uint8 array), see sm_state_save."""
        import torch
        n = ct.c_size_t()
        _check(lib().sm_state_save(self.h, int(bool(with_factors)), None, 0, ct.byref(n), None), "sm_state_save")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().sm_state_save(self.h, int(bool(with_factors)), buf.ctypes.data, buf.nbytes, ct.byref(n),
                                   _stream(torch.device("cuda", self.net.device))), "sm_state_save")
        return buf

    def load(self, image):
        import torch
        image = np.ascontiguousarray(image, dtype=np.uint8)
        _check(lib().sm_state_load(self.h, image.ctypes.data, image.nbytes,
                                   _stream(torch.device("cuda", self.net.device))), "sm_state_load")
        self.generation += 1

    def steps_log(self, m_max, C=None):
        """Recorded accepted steps: device tensors t, h (float64) and q (int32),
        each [m_max][ld]; row m is step m + 1 of every cell."""
        import torch
        C = self.cells if C is None else C
        ld = pad_ld(C)
        dev = torch.device("cuda", self.net.device)
        t = torch.zeros((m_max, ld), dtype=torch.float64, device=dev)
        h = torch.zeros((m_max, ld), dtype=torch.float64, device=dev)
        q = torch.zeros((m_max, ld), dtype=torch.int32, device=dev)
        _check(lib().sm_state_steps(self.h, int(m_max), _dptr(t), _dptr(h), _dptr(q), int(ld), _stream(dev)),
               "sm_state_steps")
        return t, h, q

    def adjoint(self, k, cot, grad, astat=None, cells_per_pass=0, allow_partial=True, grad_y0=None):
        """Reverse sweep of the last recorded run: cot [n_cot][n_s][ld] ->
        grad [n_cot][n_r][ld] = dPhi/dlog k per cell and, if given, grad_y0
        [n_cot][n_s][ld] = dPhi/dy_0 (device float64 tensors, same ld as k).
        astat: optional device int32 tensor of C entries.
        Returns SM_OK or SM_EPARTIAL."""
        ld = int(k.stride(0))
        assert cot.dim() == 3 and cot.stride(1) == ld and grad.stride(1) == ld
        assert grad_y0 is None or grad_y0.stride(1) == ld
        code = lib().sm_adjoint(self.h, _dptr(k), ld, _dptr(cot), int(cot.shape[0]), _dptr(grad),
                                _dptr(grad_y0) if grad_y0 is not None else None,
                                _dptr(astat) if astat is not None else None, int(cells_per_pass),
                                _stream(k.device))
        if code == SM_EPARTIAL and allow_partial:
            return code
        _check(code, "sm_adjoint")
        return code

    def replay(self, k, y, astat=None, cells_per_pass=0, allow_partial=True):
        """Frozen-step replay of the last recorded run with rate coefficients k;
        y [n_s][ld] receives y_N.  Returns SM_OK or SM_EPARTIAL."""
        ld = int(k.stride(0))
        assert y.stride(0) == ld
        code = lib().sm_replay(self.h, _dptr(k), ld, _dptr(y), _dptr(astat) if astat is not None else None,
                               int(cells_per_pass), _stream(k.device))
        if code == SM_EPARTIAL and allow_partial:
            return code
        _check(code, "sm_replay")
        return code


def probe_fma(device: int, fp64: bool) -> float:
    """Measured FMA throughput of the FP64 (fp64=True) or FP32 pipe, TFLOP/s."""
    v = ct.c_double()
    _check(lib().sm_probe_fma(int(device), int(bool(fp64)), ct.byref(v)), "sm_probe_fma")
    return v.value


PHASE_NAMES = ["zero + dR + weights", "Jacobian gather + M", "sparse head (A11, L21, U12)",
               "head Schur complement", "head packing", "panel loads", "panel LU", "U block load",
               "U block solve", "trailing update", "epilogue"]


def use_phase_build():
    """Switch this process to libstoich_phases.so (the phase-clock build made
    by build.build(phase_clocks=True)); call before creating any handle."""
    global _lib, LIB_PATH
    LIB_PATH = os.path.join(_PKG, "libstoich_phases.so")
    _lib = None
    lib()


def phase_cycles(device: int, reset: bool = False) -> np.ndarray:
    """Refresh-kernel cycles per phase (16 slots, see sm_phase_cycles);
    needs the phase-clock build (STOICH_PHASES=1)."""
    out = np.zeros(16)
    _check(lib().sm_phase_cycles(int(device), out.ctypes.data, int(bool(reset))), "sm_phase_cycles")
    return out


def stats_tensor(C, device):
    import torch
    return torch.zeros(C * CELL_STATS_DTYPE.itemsize, dtype=torch.uint8, device=device)


def stats_to_numpy(t):
    return np.frombuffer(t.cpu().numpy().tobytes(), dtype=CELL_STATS_DTYPE)
