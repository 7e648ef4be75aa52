"""Thin ctypes binding of the uotk C ABI (include/uotk.h).

Argument marshalling only: every step of every operation runs in the CUDA
library ``_lib/libuotk.so``.  Tensors are torch CUDA tensors (PyTorch provides
device memory and the current stream); nothing here computes.  If the library
is missing, ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libuotk.so")

UOTK_OK = 0
UOTK_ERR_NOT_CONVERGED = 6
DIRECT, NFFT, DIRECT_BF16, DIRECT_BF16X3, AUTO = 0, 1, 2, 3, 4
REF_PRODUCT, REF_COUNTING = 0, 1
WARM_START = 1
LOG_DOMAIN = 2
CSTAR_INIT = 4

_lib = None
_lock = threading.Lock()


class UotkError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"uotk status {status}: {message}")
        self.status = status


class SumOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("bandwidth", ctypes.c_int32), ("cutoff", ctypes.c_int32),
                ("period", ctypes.c_double), ("target_err", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("reg_degree", ctypes.c_int32)]


KERNELS = {"gauss": 0, "laplace": 1, "imq": 2, "energy": 3}


class NfftPlan(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("bandwidth", ctypes.c_int32), ("cutoff", ctypes.c_int32),
                ("center", ctypes.c_float * 3), ("inv_h", ctypes.c_float),
                ("h", ctypes.c_double), ("eps", ctypes.c_double)]

    def as_dict(self):
        return {"d": self.d, "grid": self.grid, "bandwidth": self.bandwidth,
                "cutoff": self.cutoff, "center": list(self.center), "inv_h": self.inv_h,
                "h": self.h, "eps": self.eps}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    """Load the CUDA library; raise if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"uotk CUDA library not built: {LIB_PATH} missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.uotk_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
        L.uotk_destroy.argtypes = [_P]
        L.uotk_last_error.argtypes = [_P]
        L.uotk_last_error.restype = ctypes.c_char_p
        L.uotk_status_string.restype = ctypes.c_char_p
        L.uotk_launch_count.argtypes = [_P]
        L.uotk_launch_count.restype = _I64
        L.uotk_set_profiling.argtypes = [_P, ctypes.c_int]
        L.uotk_set_profiling.restype = ctypes.c_int
        L.uotk_set_workspace_limit.argtypes = [_P, _I64]
        L.uotk_set_wait_timeout_test.argtypes = [_P, _I64]
        L.uotk_profile_read.argtypes = [_P, ctypes.c_char_p, ctypes.c_int,
                                        ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.c_int]
        L.uotk_profile_read.restype = ctypes.c_int
        L.uotk_profile_reset.argtypes = [_P]
        opts = ctypes.POINTER(SumOpts)
        plan = ctypes.POINTER(NfftPlan)
        L.uotk_kernel_sum.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D, opts]
        L.uotk_kernel_sum_noalloc.argtypes = [_P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D]
        L.uotk_autotune_sum.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _D, opts,
                                        opts, ctypes.POINTER(_D)]
        L.uotk_kernel_sum_noalloc.restype = ctypes.c_int
        L.uotk_uot_sinkhorn.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D, _D,
                                        _D, ctypes.c_int, _D, ctypes.c_int, ctypes.c_uint, _P, _P,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_D), opts]
        L.uotk_sinkhorn_divergence.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P,
                                               _D, _D, ctypes.c_int, _D, ctypes.POINTER(_D),
                                               ctypes.POINTER(_D), opts]
        L.uotk_mmd2.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D,
                                ctypes.POINTER(_D), ctypes.POINTER(_D), opts]
        L.uotk_uot_sinkhorn_scaled.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P,
                                               _P, ctypes.c_int, _D, _D, ctypes.c_int, _D,
                                               ctypes.c_int, ctypes.c_uint, _P, _P, _P,
                                               ctypes.POINTER(_D), opts]
        L.uotk_uot_sinkhorn_batch.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                              _P, _P, _P, _P, _P, _P, ctypes.c_int, _D,
                                              ctypes.c_int, _P, _P, _P, _P, opts]
        L.uotk_batch_forms.argtypes = [_P, ctypes.c_int, _P]
        L.uotk_mean_cost.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P,
                                     ctypes.c_int, ctypes.POINTER(_D), opts]
        L.uotk_cstar.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D, _D, _D,
                                 ctypes.c_int, ctypes.POINTER(_D), opts]
        L.uotk_measure_unit_rates.argtypes = [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]
        L.uotk_mmd2_grad.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64, _P, _D,
                                     ctypes.POINTER(_D), _P, _P, _P, _P, opts]
        L.uotk_sinkhorn_divergence_grad.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _P, _I64,
                                                    _P, _D, _D, ctypes.c_int, _D,
                                                    ctypes.POINTER(_D), ctypes.POINTER(_D), _P,
                                                    _P, _P, _P, opts]
        L.uotk_nfft_plan.argtypes = [_P, _P, ctypes.c_int, _P, _I64, _P, _I64, _D, opts, plan]
        L.uotk_nfft_cells.argtypes = [_P, _P, plan, _P, _I64, _P]
        L.uotk_nfft_spread.argtypes = [_P, _P, plan, _P, _I64, _P, _P]
        L.uotk_nfft_convolve.argtypes = [_P, _P, plan, _P, _P]
        L.uotk_nfft_gather.argtypes = [_P, _P, plan, _P, _P, _I64, _P]
        for name in ("uotk_create", "uotk_kernel_sum", "uotk_uot_sinkhorn",
                     "uotk_sinkhorn_divergence", "uotk_mmd2", "uotk_mmd2_grad",
                     "uotk_sinkhorn_divergence_grad", "uotk_measure_unit_rates",
                     "uotk_uot_sinkhorn_batch", "uotk_batch_forms", "uotk_uot_sinkhorn_scaled",
            "uotk_mean_cost",
                     "uotk_cstar", "uotk_nfft_plan",
                     "uotk_nfft_cells", "uotk_nfft_spread", "uotk_nfft_convolve",
                     "uotk_nfft_gather"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


class Context:
    """One uotk_ctx (device workspace, flags) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = _P()
        st = lib().uotk_create(ctypes.byref(h), int(device))
        if st != UOTK_OK:
            raise UotkError(st, f"uotk_create(device={device}) failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().uotk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(lib().uotk_launch_count(self.handle))

    def set_profiling(self, on: bool):
        self.check(lib().uotk_set_profiling(self.handle, int(bool(on))))

    def set_workspace_limit(self, nbytes: int):
        """Largest device workspace of this context (0: no limit)."""
        self.check(lib().uotk_set_workspace_limit(self.handle, int(nbytes)))

    def set_wait_timeout_test(self, cycles: int):
        """cycles > 0: the first bounded device wait per CTA of the NFFT spread
        and gather waits on a barrier nothing completes and runs out after that
        many cycles (calls then return UOTK_ERR_TIMEOUT); 0 turns it off."""
        self.check(lib().uotk_set_wait_timeout_test(self.handle, int(cycles)))

    def profile(self) -> dict:
        """{stage: (launches, total device ms)} since the last reset."""
        names = ctypes.create_string_buffer(4096)
        counts = (_I64 * 32)()
        ms = (_D * 32)()
        k = lib().uotk_profile_read(self.handle, names, 4096, counts, ms, 32)
        labels = names.value.decode().split(";") if k else []
        return {labels[i]: (int(counts[i]), float(ms[i])) for i in range(k)}

    def profile_reset(self):
        lib().uotk_profile_reset(self.handle)

    def check(self, st, ok=(UOTK_OK,)):
        if st not in ok:
            msg = lib().uotk_last_error(self.handle).decode()
            raise UotkError(st, msg)
        return st


_contexts = {}


def default_context(device=None) -> Context:
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _contexts:
        _contexts[dev] = Context(dev)
    return _contexts[dev]


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _f32(t, name, ndim=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    return t.contiguous()


def _pts(t, name):
    t = _f32(t, name)
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    if t.dim() != 2:
        raise ValueError(f"{name} must be (n, d)")
    return t


def _opts(method="direct", grid=0, bandwidth=0, cutoff=0, period=0.0, target_err=0.0,
          kernel="gauss", reg_degree=0):
    """uotk_sum_opts; kernel is one of Table tab:0 (gauss, laplace, imq, energy);
    reg_degree: the NFFT regularisation degree p of the non-Gaussian kernels."""
    m = {"direct": DIRECT, "nfft": NFFT, "direct_bf16": DIRECT_BF16,
         "direct_bf16x3": DIRECT_BF16X3, "auto": AUTO}.get(method, method)
    k = KERNELS.get(kernel, kernel)
    return SumOpts(int(m), int(grid), int(bandwidth), int(cutoff), float(period),
                   float(target_err), int(k), int(reg_degree))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def kernel_sum(src, w, tgt, eps, method="direct", out=None, ctx=None, **nfft):
    """out_j = sum_i w_i exp(-||src_i - tgt_j||^2/eps) (uotk_kernel_sum); with
    kernel="laplace" / "imq" / "energy" the kernel of Table tab:0 with p = eps."""
    src, tgt, w = _pts(src, "src"), _pts(tgt, "tgt"), _f32(w, "w").reshape(-1)
    ctx = ctx or default_context()
    if out is None:
        out = torch.empty(tgt.shape[0], device=tgt.device, dtype=torch.float32)
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_kernel_sum(ctx.handle, _stream(), src.shape[1], _ptr(src), src.shape[0],
                                    _ptr(w), _ptr(tgt), tgt.shape[0], _ptr(out), float(eps),
                                    ctypes.byref(o)))
    return out


METHOD_NAMES = {DIRECT: "direct", NFFT: "nfft", DIRECT_BF16: "direct_bf16",
                DIRECT_BF16X3: "direct_bf16x3"}


def autotune_sum(src, w, tgt, eps, target_err=0.0, grid=0, cutoff=0, ctx=None):
    """uotk_autotune_sum: the fastest summation form for src -> tgt within
    target_err (max error / sum|w|; 0: 1e-5), measured on this GPU and cached
    in the context.  Returns (options dict, report dict)."""
    src, tgt, w = _pts(src, "src"), _pts(tgt, "tgt"), _f32(w, "w").reshape(-1)
    ctx = ctx or default_context()
    o = _opts("direct", grid=grid, cutoff=cutoff, target_err=target_err)
    chosen = SumOpts()
    rep = (_D * 8)()
    ctx.check(lib().uotk_autotune_sum(ctx.handle, _stream(), src.shape[1], _ptr(src),
                                      src.shape[0], _ptr(w), _ptr(tgt), tgt.shape[0],
                                      float(eps), ctypes.byref(o), ctypes.byref(chosen), rep))
    opts = {"method": METHOD_NAMES.get(chosen.method, chosen.method), "grid": chosen.grid,
            "bandwidth": chosen.bandwidth, "cutoff": chosen.cutoff,
            "target_err": chosen.target_err}
    report = dict(zip(["ms", "err", "direct_ms", "forms", "grid", "cutoff", "samples",
                       "target"], list(rep)))
    return opts, report


def kernel_sum_noalloc(src, w, tgt, eps, out):
    """Direct kernel sum through uotk_kernel_sum_noalloc: no context, no
    allocation inside the library; `out` must be provided by the caller.
    Returns the status code (0 on success)."""
    src, tgt, w = _pts(src, "src"), _pts(tgt, "tgt"), _f32(w, "w").reshape(-1)
    return int(lib().uotk_kernel_sum_noalloc(_stream(), src.shape[1], _ptr(src), src.shape[0],
                                             _ptr(w), _ptr(tgt), tgt.shape[0], _ptr(out),
                                             float(eps)))


def uot_sinkhorn(x, a, y, b, eps, rho1, rho2=None, max_sweeps=100, tol=0.0, ref="product",
                 gamma0=None, method="direct", ctx=None, beta=None, gamma=None,
                 log_domain=False, cstar_init=False, **nfft):
    """KL-penalised entropic UOT by Sinkhorn (uotk_uot_sinkhorn).

    log_domain: per-row log-sum-exp half-steps (UOTK_LOG_DOMAIN; direct form).
    cstar_init: gamma^0 = c* 1, c* of Eq. (561) (UOTK_CSTAR_INIT).
    Returns (beta, gamma, sweeps_done, value, converged)."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    rho2 = rho1 if rho2 is None else rho2
    ctx = ctx or default_context()
    dev = x.device
    beta = torch.empty(x.shape[0], device=dev, dtype=torch.float64) if beta is None else beta
    flags = 0
    if gamma0 is not None:
        gamma = gamma0.to(device=dev, dtype=torch.float64).contiguous().clone()
        flags |= WARM_START
    elif gamma is None:
        gamma = torch.empty(y.shape[0], device=dev, dtype=torch.float64)
    if log_domain:
        flags |= LOG_DOMAIN
    if cstar_init:
        flags |= CSTAR_INIT
    refc = {"product": REF_PRODUCT, "counting": REF_COUNTING}.get(ref, ref)
    sweeps = ctypes.c_int(0)
    value = _D(0.0)
    o = _opts(method, **nfft)
    st = ctx.check(lib().uotk_uot_sinkhorn(
        ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a), _ptr(y), y.shape[0],
        _ptr(b), float(eps), float(rho1), float(rho2), int(max_sweeps), float(tol), int(refc),
        flags, _ptr(beta), _ptr(gamma), ctypes.byref(sweeps), ctypes.byref(value),
        ctypes.byref(o)), ok=(UOTK_OK, UOTK_ERR_NOT_CONVERGED))
    return beta, gamma, sweeps.value, value.value, st == UOTK_OK


def mean_cost(x, a, y, b, r=2, method="direct", ctx=None, **nfft):
    """<mu (x) nu|d^r> for r = 2 (moments) or r = 1 (energy kernel, direct or
    NFFT) with the masses (uotk_mean_cost): returns (cost, mu(X), nu(X))."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    out = (_D * 3)()
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_mean_cost(ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0],
                                   _ptr(a), _ptr(y), y.shape[0], _ptr(b), int(r), out,
                                   ctypes.byref(o)))
    return tuple(out)


def cstar(x, a, y, b, eps, rho1, rho2=None, r=2, method="direct", ctx=None, **nfft):
    """c* of Eq. (561) for the cost |x - y|^r (uotk_cstar): returns (c*, Eq. (W4)
    objective at c* mu (x) nu, <mu (x) nu|d^r>)."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    rho2 = rho1 if rho2 is None else rho2
    ctx = ctx or default_context()
    out = (_D * 3)()
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_cstar(ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a),
                               _ptr(y), y.shape[0], _ptr(b), float(eps), float(rho1),
                               float(rho2), int(r), out, ctypes.byref(o)))
    return tuple(out)


def uot_sinkhorn_scaled(x, a, y, b, eps_schedule, rho1, rho2=None, max_sweeps=1000, tol=1e-6,
                        ref="product", method="direct", log_domain=False, ctx=None, **nfft):
    """lambda-scaling (uotk_uot_sinkhorn_scaled): stages eps_schedule[0], ... each
    warm-started from the previous gamma.  Returns (beta, gamma, sweeps per stage,
    value of the last stage, converged)."""
    import numpy as np
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    rho2 = rho1 if rho2 is None else rho2
    ctx = ctx or default_context()
    sched = np.ascontiguousarray(np.asarray(eps_schedule, dtype=np.float64))
    beta = torch.empty(x.shape[0], device=x.device, dtype=torch.float64)
    gamma = torch.empty(y.shape[0], device=x.device, dtype=torch.float64)
    sweeps = np.zeros(sched.size, dtype=np.int32)
    value = _D(0.0)
    refc = {"product": REF_PRODUCT, "counting": REF_COUNTING}.get(ref, ref)
    o = _opts(method, **nfft)
    st = ctx.check(lib().uotk_uot_sinkhorn_scaled(
        ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a), _ptr(y), y.shape[0],
        _ptr(b), sched.ctypes.data, sched.size, float(rho1), float(rho2), int(max_sweeps),
        float(tol), int(refc), LOG_DOMAIN if log_domain else 0, _ptr(beta), _ptr(gamma),
        sweeps.ctypes.data, ctypes.byref(value), ctypes.byref(o)),
        ok=(UOTK_OK, UOTK_ERR_NOT_CONVERGED))
    return beta, gamma, sweeps, value.value, st == UOTK_OK


def uot_sinkhorn_batch(x, a, x_off, y, b, y_off, eps, rho1, rho2=None, max_sweeps=100, tol=0.0,
                       ref="product", method="direct", target_err=0.0, ctx=None):
    """Many independent problems at once (uotk_uot_sinkhorn_batch).

    x, a, y, b: concatenated CUDA tensors; x_off, y_off: host sequences of
    npairs + 1 offsets; eps, rho1, rho2: per-pair sequences (or scalars).
    method "direct" (all pairs in the grouped direct batch) or "auto" (each
    large pair's form measured; see batch_forms).
    Returns (beta, gamma, sweeps_done[npairs], values[npairs], converged)."""
    import numpy as np
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    xo = np.ascontiguousarray(np.asarray(x_off, dtype=np.int64))
    yo = np.ascontiguousarray(np.asarray(y_off, dtype=np.int64))
    npairs = xo.size - 1
    def per_pair(v):
        return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (npairs,)))
    e, r1 = per_pair(eps), per_pair(rho1)
    r2 = per_pair(rho1 if rho2 is None else rho2)
    beta = torch.empty(x.shape[0], device=x.device, dtype=torch.float64)
    gamma = torch.empty(y.shape[0], device=x.device, dtype=torch.float64)
    sweeps = np.zeros(npairs, dtype=np.int32)
    values = np.zeros(npairs, dtype=np.float64)
    refc = {"product": REF_PRODUCT, "counting": REF_COUNTING}.get(ref, ref)
    o = _opts(method, target_err=target_err)
    st = ctx.check(lib().uotk_uot_sinkhorn_batch(
        ctx.handle, _stream(), x.shape[1], npairs, xo.ctypes.data, _ptr(x), _ptr(a),
        yo.ctypes.data, _ptr(y), _ptr(b), e.ctypes.data, r1.ctypes.data, r2.ctypes.data,
        int(max_sweeps), float(tol), int(refc), _ptr(beta), _ptr(gamma), sweeps.ctypes.data,
        values.ctypes.data, ctypes.byref(o)), ok=(UOTK_OK, UOTK_ERR_NOT_CONVERGED))
    return beta, gamma, sweeps, values, st == UOTK_OK


def batch_forms(npairs, ctx=None):
    """The form (DIRECT or NFFT) each pair of the last uot_sinkhorn_batch call on
    ctx was solved with (uotk_batch_forms)."""
    import numpy as np
    ctx = ctx or default_context()
    forms = np.zeros(npairs, dtype=np.int32)
    ctx.check(lib().uotk_batch_forms(ctx.handle, int(npairs), forms.ctypes.data))
    return forms


def sinkhorn_divergence(x, a, y, b, eps, rho, max_sweeps=100, tol=0.0, method="direct",
                        ctx=None, **nfft):
    """Unbalanced Sinkhorn divergence of Eq. (586); returns (sd, [UOT_xy, UOT_xx, UOT_yy])."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    sd = _D(0.0)
    parts = (_D * 3)()
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_sinkhorn_divergence(
        ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a), _ptr(y), y.shape[0],
        _ptr(b), float(eps), float(rho), int(max_sweeps), float(tol), ctypes.byref(sd), parts,
        ctypes.byref(o)), ok=(UOTK_OK, UOTK_ERR_NOT_CONVERGED))
    return sd.value, list(parts)


def mmd2(x, a, y, b, ell, method="direct", ctx=None, **nfft):
    """MMD^2 of Eq. (1205), Gaussian kernel exp(-d^2/ell^2), or with kernel=
    "laplace" / "imq" / "energy" the kernel of Table tab:0 with p = ell;
    returns (value, [A, B, C])."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    v = _D(0.0)
    parts = (_D * 3)()
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_mmd2(ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a),
                              _ptr(y), y.shape[0], _ptr(b), float(ell), ctypes.byref(v), parts,
                              ctypes.byref(o)))
    return v.value, list(parts)


def measure_unit_rates(ctx=None):
    """(ex2 ops, FP32 FMA ops) per clock per SM of this GPU (uotk_measure_unit_rates)."""
    ctx = ctx or default_context()
    e, f = _D(0.0), _D(0.0)
    ctx.check(lib().uotk_measure_unit_rates(ctx.handle, _stream(), ctypes.byref(e),
                                            ctypes.byref(f)))
    return e.value, f.value


def _grad_outputs(x, y, need):
    """FP64 device gradient buffers (a, x, b, y); None where not needed."""
    n, d = x.shape
    m = y.shape[0]
    shapes = ((n,), (n, d), (m,), (m, d))
    return [torch.empty(sh, device=x.device, dtype=torch.float64) if k else None
            for sh, k in zip(shapes, need)]


def mmd2_grad(x, a, y, b, ell, method="direct", need=(True, True, True, True), ctx=None,
              **nfft):
    """MMD^2 (Eq. 1205) and its gradients (uotk_mmd2_grad).

    Returns (value, grad_a, grad_x, grad_b, grad_y): FP64 device tensors in the
    caller's order, None where `need` is False."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    g = _grad_outputs(x, y, need)
    v = _D(0.0)
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_mmd2_grad(ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0],
                                   _ptr(a), _ptr(y), y.shape[0], _ptr(b), float(ell),
                                   ctypes.byref(v), *[_ptr(t) for t in g], ctypes.byref(o)))
    return (v.value, *g)


def sinkhorn_divergence_grad(x, a, y, b, eps, rho, max_sweeps=100, tol=0.0, method="direct",
                             need=(True, True, True, True), ctx=None, **nfft):
    """Sinkhorn divergence (Eq. 586) and its envelope-theorem gradients
    (uotk_sinkhorn_divergence_grad).

    Returns (sd, parts, grad_a, grad_x, grad_b, grad_y), gradients as FP64
    device tensors in the caller's order, None where `need` is False."""
    x, y = _pts(x, "x"), _pts(y, "y")
    a, b = _f32(a, "a").reshape(-1), _f32(b, "b").reshape(-1)
    ctx = ctx or default_context()
    g = _grad_outputs(x, y, need)
    sd = _D(0.0)
    parts = (_D * 3)()
    o = _opts(method, **nfft)
    ctx.check(lib().uotk_sinkhorn_divergence_grad(
        ctx.handle, _stream(), x.shape[1], _ptr(x), x.shape[0], _ptr(a), _ptr(y), y.shape[0],
        _ptr(b), float(eps), float(rho), int(max_sweeps), float(tol), ctypes.byref(sd), parts,
        *[_ptr(t) for t in g], ctypes.byref(o)), ok=(UOTK_OK, UOTK_ERR_NOT_CONVERGED))
    return (sd.value, list(parts), *g)


class _LossFn(torch.autograd.Function):
    """Scalar loss with gradients from one library call in forward; backward
    scales the stored gradients by the incoming grad_output."""

    @staticmethod
    def forward(ctx_, call, x, a, y, b):
        nig = ctx_.needs_input_grad  # (call, x, a, y, b)
        value, *grads = call(x, a, y, b, (nig[2], nig[1], nig[4], nig[3]))
        ctx_.save_for_backward(*[g if g is not None else torch.empty(0) for g in grads])
        ctx_.has = [g is not None for g in grads]
        ctx_.dtypes = (a.dtype, x.dtype, b.dtype, y.dtype)
        ctx_.shapes = (a.shape, x.shape, b.shape, y.shape)
        return torch.tensor(value, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx_, gout):
        out = []
        for g, has, dt, sh in zip(ctx_.saved_tensors, ctx_.has, ctx_.dtypes, ctx_.shapes):
            out.append((gout * g).to(dt).reshape(sh) if has else None)
        ga, gx, gb, gy = out
        return None, gx, ga, gy, gb


def mmd2_loss(x, a, y, b, ell, method="direct", ctx=None, **nfft):
    """MMD^2 as a differentiable scalar (FP64 0-dim tensor) in x, a, y, b."""
    def call(x_, a_, y_, b_, need):
        return mmd2_grad(x_.detach(), a_.detach(), y_.detach(), b_.detach(), ell, method,
                         need, ctx, **nfft)
    return _LossFn.apply(call, x, a, y, b)


def sinkhorn_divergence_loss(x, a, y, b, eps, rho, max_sweeps=100, tol=0.0, method="direct",
                             ctx=None, **nfft):
    """Sinkhorn divergence as a differentiable scalar (FP64 0-dim tensor); the
    gradient is the envelope-theorem gradient at the final duals."""
    def call(x_, a_, y_, b_, need):
        sd, _, *g = sinkhorn_divergence_grad(x_.detach(), a_.detach(), y_.detach(),
                                             b_.detach(), eps, rho, max_sweeps, tol, method,
                                             need, ctx, **nfft)
        return (sd, *g)
    return _LossFn.apply(call, x, a, y, b)


def nfft_plan(src, tgt, eps, ctx=None, **nfft):
    src, tgt = _pts(src, "src"), _pts(tgt, "tgt")
    ctx = ctx or default_context()
    p = NfftPlan()
    o = _opts("nfft", **nfft)
    ctx.check(lib().uotk_nfft_plan(ctx.handle, _stream(), src.shape[1], _ptr(src), src.shape[0],
                                   _ptr(tgt), tgt.shape[0], float(eps), ctypes.byref(o),
                                   ctypes.byref(p)))
    return p


def nfft_cells(plan, pts, ctx=None):
    pts = _pts(pts, "pts")
    ctx = ctx or default_context()
    cells = torch.empty((pts.shape[0], 3), device=pts.device, dtype=torch.int32)
    ctx.check(lib().uotk_nfft_cells(ctx.handle, _stream(), ctypes.byref(plan), _ptr(pts),
                                    pts.shape[0], _ptr(cells)))
    return cells


def nfft_spread(plan, pts, w, ctx=None):
    pts, w = _pts(pts, "pts"), _f32(w, "w").reshape(-1)
    ctx = ctx or default_context()
    g = plan.grid
    grid = torch.empty((g, g, g), device=pts.device, dtype=torch.float32)
    ctx.check(lib().uotk_nfft_spread(ctx.handle, _stream(), ctypes.byref(plan), _ptr(pts),
                                     pts.shape[0], _ptr(w), _ptr(grid)))
    return grid


def nfft_convolve(plan, grid_in, grid_out=None, ctx=None):
    grid_in = _f32(grid_in, "grid_in")
    ctx = ctx or default_context()
    grid_out = torch.empty_like(grid_in) if grid_out is None else grid_out
    ctx.check(lib().uotk_nfft_convolve(ctx.handle, _stream(), ctypes.byref(plan), _ptr(grid_in),
                                       _ptr(grid_out)))
    return grid_out


def nfft_gather(plan, grid, pts, ctx=None):
    grid, pts = _f32(grid, "grid"), _pts(pts, "pts")
    ctx = ctx or default_context()
    out = torch.empty(pts.shape[0], device=pts.device, dtype=torch.float32)
    ctx.check(lib().uotk_nfft_gather(ctx.handle, _stream(), ctypes.byref(plan), _ptr(grid),
                                     _ptr(pts), pts.shape[0], _ptr(out)))
    return out


EXPORTED = ["uotk_create", "uotk_destroy", "uotk_last_error", "uotk_status_string",
            "uotk_launch_count", "uotk_set_profiling", "uotk_profile_read", "uotk_profile_reset",
            "uotk_set_workspace_limit", "uotk_set_wait_timeout_test",
            "uotk_kernel_sum", "uotk_kernel_sum_noalloc", "uotk_autotune_sum", "uotk_uot_sinkhorn",
            "uotk_sinkhorn_divergence", "uotk_mmd2", "uotk_mmd2_grad",
            "uotk_sinkhorn_divergence_grad", "uotk_measure_unit_rates",
            "uotk_uot_sinkhorn_batch", "uotk_batch_forms", "uotk_uot_sinkhorn_scaled",
            "uotk_mean_cost",
            "uotk_cstar", "uotk_nfft_plan", "uotk_nfft_cells",
            "uotk_nfft_spread", "uotk_nfft_convolve", "uotk_nfft_gather"]
