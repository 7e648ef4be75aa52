"""FP64 CPU oracle for the UOT / MMD kernel-summation path (arXiv 2306.13618).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library ``paper_2306_13618_gb300`` and never calls it.

The dense parts (kernel sums, Alg. 1, the dual and primal objectives, MMD^2,
the Sinkhorn divergence, balanced Sinkhorn) are plain C in ``uot_oracle.c``,
compiled with gcc and loaded with ctypes.  The NFFT fast-summation steps of
Sec. 4 are plain numpy in ``oracle.nfft``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, an invariant, brute force or a library routine
(tests/test_oracle_*.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uot_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile uot_oracle.c into oracle/_lib/liboracle.so (gcc, OpenMP, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.orc_ksum.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, ctypes.c_double, _D]
    lib.orc_uot_sinkhorn.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                     ctypes.c_double]
    lib.orc_dual_value.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   _D, _D, ctypes.c_int, ctypes.c_double]
    lib.orc_dual_value.restype = ctypes.c_double
    lib.orc_primal_value.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D,
                                     ctypes.c_double]
    lib.orc_primal_value.restype = ctypes.c_double
    lib.orc_plan.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D, ctypes.c_double,
                             _D, _D, ctypes.c_int, _D, ctypes.c_double]
    lib.orc_mmd2.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D, ctypes.c_double, _D]
    lib.orc_mmd2.restype = ctypes.c_double
    lib.orc_sinkhorn_divergence.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int, _D,
                                            ctypes.c_double]
    lib.orc_sinkhorn_divergence.restype = ctypes.c_double
    lib.orc_balanced_sinkhorn.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                          ctypes.c_double, ctypes.c_int, _D, _D]
    lib.orc_ksum_kernel.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _I64, _D,
                                    _D, _I64, _D]
    lib.orc_mmd2_kernel.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _I64, _D,
                                    _D, _I64, _D, _D]
    lib.orc_mmd2_kernel.restype = ctypes.c_double
    lib.orc_mmd2_grad.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D, ctypes.c_double,
                                  _D, _D, _D, _D]
    lib.orc_mmd2_grad_rows.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                       ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), _I64, _D, _D]
    lib.orc_dual_grad.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D, _D]
    lib.orc_sinkhorn_divergence_grad.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 _D, _D, _D, _D]
    lib.orc_sinkhorn_divergence_grad.restype = ctypes.c_double
    lib.orc_mean_cost.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _I64, _D, ctypes.c_double]
    lib.orc_mean_cost.restype = ctypes.c_double
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _pts(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return a


def _vec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _p(a):
    return a.ctypes.data_as(_D)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(k: int) -> None:
    _load().orc_set_num_threads(int(k))


def ksum(src, w, tgt, eps):
    """out_j = sum_i w_i exp(-||src_i - tgt_j||^2 / eps)  (Eq. fast_sum, Gaussian)."""
    src, tgt, w = _pts(src), _pts(tgt), _vec(w)
    d = src.shape[1]
    assert tgt.shape[1] == d and w.shape[0] == src.shape[0]
    out = np.empty(tgt.shape[0])
    _load().orc_ksum(d, _p(src), src.shape[0], _p(w), _p(tgt), tgt.shape[0], float(eps), _p(out))
    return out


def uot_sinkhorn(x, mu, y, nu, eps, eta1, eta2=None, sweeps=100, ref=0,
                 logdomain=False, gamma0=None, r=2):
    """Alg. 1 for `sweeps` sweeps (beta then gamma) from gamma0 (default 0).

    lambda = 1/eps.  ref 0: product reference (paper); ref 1: counting reference.
    r: the cost |x - y|^r (2: Gaussian Gibbs kernel, 1: Laplacian).
    Returns (beta, gamma) as float64 arrays."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    eta2 = eta1 if eta2 is None else eta2
    beta = np.zeros(x.shape[0])
    gamma = np.zeros(y.shape[0]) if gamma0 is None else _vec(gamma0).copy()
    _load().orc_uot_sinkhorn(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0], _p(nu),
                             1.0 / eps, float(eta1), float(eta2), int(sweeps), int(ref),
                             int(bool(logdomain)), _p(beta), _p(gamma), float(r))
    return beta, gamma


def dual_value(x, mu, y, nu, eps, eta1, eta2, beta, gamma, ref=0, r=2):
    """D(beta, gamma) of Eq. (dual_euot) with the cost |x - y|^r."""
    x, y, mu, nu, beta, gamma = _pts(x), _pts(y), _vec(mu), _vec(nu), _vec(beta), _vec(gamma)
    return _load().orc_dual_value(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0],
                                  _p(nu), 1.0 / eps, float(eta1), float(eta2),
                                  _p(beta), _p(gamma), int(ref), float(r))


def primal_value(x, mu, y, nu, eps, eta1, eta2, beta, gamma, r=2):
    """Discrete primal objective of Eq. (W4) at the plan of the duals (product reference)."""
    x, y, mu, nu, beta, gamma = _pts(x), _pts(y), _vec(mu), _vec(nu), _vec(beta), _vec(gamma)
    return _load().orc_primal_value(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0],
                                    _p(nu), 1.0 / eps, float(eta1), float(eta2),
                                    _p(beta), _p(gamma), float(r))


def plan(x, mu, y, nu, eps, beta, gamma, ref=0, r=2):
    """pi_ij = mu_i nu_j e^{lambda(beta_i+gamma_j)} k_ij (ref 0), n x m dense."""
    x, y, mu, nu, beta, gamma = _pts(x), _pts(y), _vec(mu), _vec(nu), _vec(beta), _vec(gamma)
    pi = np.empty((x.shape[0], y.shape[0]))
    _load().orc_plan(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0], _p(nu),
                     1.0 / eps, _p(beta), _p(gamma), int(ref), _p(pi), float(r))
    return pi


def mmd2(x, mu, y, nu, ell, return_parts=False):
    """MMD^2 of Eq. (1205), Gaussian kernel exp(-||.||^2/ell^2) (Table tab:0)."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    parts = np.empty(3)
    v = _load().orc_mmd2(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0], _p(nu),
                         float(ell), _p(parts))
    return (v, parts) if return_parts else v


def sinkhorn_divergence(x, mu, y, nu, eps, eta, sweeps=100, return_parts=False, r=2):
    """Unbalanced Sinkhorn divergence of Eq. (586) (product reference), cost |x - y|^r."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    parts = np.empty(3)
    v = _load().orc_sinkhorn_divergence(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y),
                                        y.shape[0], _p(nu), 1.0 / eps, float(eta),
                                        int(sweeps), _p(parts), float(r))
    return (v, parts) if return_parts else v


def balanced_sinkhorn(x, P, y, Q, eps, iters):
    """Textbook balanced entropic OT Sinkhorn (reference P (x) Q); returns (f, g)."""
    x, y, P, Q = _pts(x), _pts(y), _vec(P), _vec(Q)
    f = np.zeros(x.shape[0])
    g = np.zeros(y.shape[0])
    _load().orc_balanced_sinkhorn(x.shape[1], _p(x), x.shape[0], _p(P), _p(y), y.shape[0],
                                  _p(Q), 1.0 / eps, int(iters), _p(f), _p(g))
    return f, g


def _grad_bufs(x, y):
    n, d = x.shape
    m = y.shape[0]
    return np.empty(n), np.empty((n, d)), np.empty(m), np.empty((m, d))


def mmd2_grad(x, mu, y, nu, ell):
    """Derivatives of MMD^2 (Eq. 1205) in (mu, x, nu, y): returns (gmu, gx, gnu, gy)."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    ga, gx, gb, gy = _grad_bufs(x, y)
    _load().orc_mmd2_grad(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0], _p(nu),
                          float(ell), _p(ga), _p(gx), _p(gb), _p(gy))
    return ga, gx, gb, gy


def mmd2_grad_rows(x, mu, y, nu, ell, side, rows):
    """mmd2_grad at selected rows of one side (0: mu/x, 1: nu/y): returns (gw, gp)."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    gw, gp = np.empty(rows.size), np.empty((rows.size, x.shape[1]))
    _load().orc_mmd2_grad_rows(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0],
                               _p(nu), float(ell), int(side),
                               rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size,
                               _p(gw), _p(gp))
    return gw, gp


def dual_grad(x, mu, y, nu, eps, eta1, eta2, beta, gamma):
    """Partial derivatives of D(beta, gamma) (Eq. dual_euot, product reference) in
    (mu, x, nu, y) at fixed duals: returns (gmu, gx, gnu, gy)."""
    x, y, mu, nu, beta, gamma = _pts(x), _pts(y), _vec(mu), _vec(nu), _vec(beta), _vec(gamma)
    ga, gx, gb, gy = _grad_bufs(x, y)
    _load().orc_dual_grad(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0], _p(nu),
                          1.0 / eps, float(eta1), float(eta2), _p(beta), _p(gamma),
                          _p(ga), _p(gx), _p(gb), _p(gy))
    return ga, gx, gb, gy


def sinkhorn_divergence_grad(x, mu, y, nu, eps, eta, sweeps=100):
    """Sinkhorn divergence (Eq. 586) and its envelope-theorem gradient at the
    duals after `sweeps` sweeps: returns (sd, gmu, gx, gnu, gy)."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    ga, gx, gb, gy = _grad_bufs(x, y)
    v = _load().orc_sinkhorn_divergence_grad(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y),
                                             y.shape[0], _p(nu), 1.0 / eps, float(eta),
                                             int(sweeps), _p(ga), _p(gx), _p(gb), _p(gy))
    return v, ga, gx, gb, gy


KERNELS = {"gauss": 0, "laplace": 1, "imq": 2, "energy": 3}


def ksum_kernel(kind, p, src, w, tgt):
    """out_j = sum_i w_i k(src_i, tgt_j), k one of the kernels of Table tab:0:
    gauss exp(-r^2/p^2), laplace exp(-r/p), imq 1/sqrt(r^2 + p^2), energy -r."""
    src, tgt, w = _pts(src), _pts(tgt), _vec(w)
    out = np.empty(tgt.shape[0])
    _load().orc_ksum_kernel(KERNELS[kind], float(p), src.shape[1], _p(src), src.shape[0], _p(w),
                            _p(tgt), tgt.shape[0], _p(out))
    return out


def mmd2_kernel(kind, p, x, mu, y, nu, return_parts=False):
    """MMD^2 of Eq. (1205) with a kernel of Table tab:0 (see ksum_kernel)."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    parts = np.empty(3)
    v = _load().orc_mmd2_kernel(KERNELS[kind], float(p), x.shape[1], _p(x), x.shape[0], _p(mu),
                                _p(y), y.shape[0], _p(nu), _p(parts))
    return (v, parts) if return_parts else v


def mean_cost(x, mu, y, nu, r=2):
    """<mu (x) nu | d^r> = sum_ij mu_i nu_j ||x_i - y_j||^r, the double sum."""
    x, y, mu, nu = _pts(x), _pts(y), _vec(mu), _vec(nu)
    return _load().orc_mean_cost(x.shape[1], _p(x), x.shape[0], _p(mu), _p(y), y.shape[0],
                                 _p(nu), float(r))


def independent_objective(c, cost, m1, m2, eps, eta1, eta2):
    """Objective of Eq. (W4) at the plan c mu (x) nu, lambda = 1/eps:
        c <mu (x) nu|d^2> + (1/lambda) m1 m2 (c log c - c + 1)
        + eta1 m1 (c m2 log(c m2) - c m2 + 1) + eta2 m2 (c m1 log(c m1) - c m1 + 1),
    the marginals of c mu (x) nu being c m2 mu and c m1 nu (m1 = mu(X), m2 = nu(X))."""
    return (c * cost + eps * m1 * m2 * (c * np.log(c) - c + 1.0)
            + eta1 * m1 * (c * m2 * np.log(c * m2) - c * m2 + 1.0)
            + eta2 * m2 * (c * m1 * np.log(c * m1) - c * m1 + 1.0))


def cstar(x, mu, y, nu, eps, eta1, eta2, r=2):
    """c*_{r;eta;lambda} of Eq. (561) (Prop. prop:536), lambda = 1/eps:
        c* = exp(-<mu (x) nu|d^r> / (m1 m2 (eta1 + eta2 + 1/lambda)))
             m1^{-eta2/(eta1+eta2+1/lambda)} m2^{-eta1/(eta1+eta2+1/lambda)}.
    Returns (c*, objective of Eq. (W4) at c* mu (x) nu, <mu (x) nu|d^r>)."""
    mu, nu = _vec(mu), _vec(nu)
    m1, m2 = float(np.sum(mu)), float(np.sum(nu))
    cost = mean_cost(x, mu, y, nu, r)
    den = eta1 + eta2 + eps
    c = np.exp(-cost / (m1 * m2 * den)) * m1 ** (-eta2 / den) * m2 ** (-eta1 / den)
    return c, independent_objective(c, cost, m1, m2, eps, eta1, eta2), cost
