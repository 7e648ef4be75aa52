"""Fast summation for the non-smooth radial kernels of Table tab:0 (Laplace,
inverse multiquadric, energy), plain numpy FP64 (Sec. 4.2 of arXiv 2306.13618).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Shares no code with the
CUDA library.

The kernel is not smooth at r = 0 and not periodic, so its Fourier series
converges slowly.  Sec. 4.2 embeds it into a smooth 1-periodic function with
polynomial pieces that match its derivatives (the construction of the NFFT
fast-summation literature it cites).  In torus units rbar = r/h, with
Kh(rbar) = K(h rbar):

    K_R(rbar) = T_I(rbar)      rbar <  eps_I           (inner regularisation)
              = Kh(rbar)       eps_I <= rbar <= 1/2 - eps_B
              = T_B(rbar)      1/2 - eps_B < rbar <= 1/2   (boundary, the K_B of Sec. 4.2)
              = K_B            rbar > 1/2              (corners of the cube, d > 1)

T_I has degree 2p - 1 and matches Kh and its first p - 1 derivatives at eps_I
and, mirrored (K_R is even), at -eps_I.  T_B has degree 2p - 1, matches Kh and
its first p - 1 derivatives at 1/2 - eps_B, and at 1/2 takes the constant value
K_B with derivatives 1..p-1 zero, so that K_R, constant beyond the sphere
rbar = 1/2, is C^{p-1} on the whole torus (its periodic continuation across the
faces of the cube stays inside the constant region or is mirror symmetric).
K_B is the value at 1/2 of the polynomial that matches Kh at 1/2 - eps_B and
its mirror image Kh(1 - rbar) at 1/2 + eps_B.  Both pieces are two-point Taylor
interpolants.

The sum then splits into a smooth part and a near field:

    s_i = sum_j w_j K_R((x_i - y_j)/h)                     (Fourier series, Eq. 1724)
        + sum_{|x_i - y_j| < eps_I h} w_j (K(|x_i - y_j|) - T_I(|x_i - y_j|/h)),

exact whenever every difference satisfies |x_i - y_j| <= (1/2 - eps_B) h.
b_k is the discrete Fourier transform of K_R sampled on the N^d grid:

    b_k = N^{-d} sum_{l in I_N^d} K_R(||l||/N) e^{-2 pi i k.l/N}.
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np

from . import nfft as _nfft

KINDS = ("laplace", "imq", "energy", "gauss")


def taylor_coeffs(kind: str, p: float, r0: float, order: int) -> np.ndarray:
    """c_j = K^{(j)}(r0)/j!, j < order, of the radial kernel K of Table tab:0:
    laplace exp(-r/p), imq 1/sqrt(r^2 + p^2), energy -r, gauss exp(-r^2/p^2)."""
    c = np.zeros(order)
    if kind == "laplace":
        for j in range(order):
            c[j] = (-1.0 / p) ** j * np.exp(-r0 / p) / factorial(j)
    elif kind == "energy":
        c[0] = -r0
        if order > 1:
            c[1] = -1.0
    elif kind == "imq":
        # f = g^{-1/2}, g = r^2 + p^2: (r^2 + p^2) f' + r f = 0; at r = r0 + t the
        # coefficients of t^n give
        # (r0^2+p^2)(n+1) c_{n+1} + (2n+1) r0 c_n + n c_{n-1} = 0
        g0 = r0 * r0 + p * p
        c[0] = 1.0 / np.sqrt(g0)
        for n in range(order - 1):
            prev = c[n - 1] if n >= 1 else 0.0
            c[n + 1] = -((2 * n + 1) * r0 * c[n] + n * prev) / ((n + 1) * g0)
    elif kind == "gauss":
        # f' = -(2 r / p^2) f:  (n+1) c_{n+1} = -(2/p^2) (r0 c_n + c_{n-1})
        c[0] = np.exp(-r0 * r0 / (p * p))
        for n in range(order - 1):
            prev = c[n - 1] if n >= 1 else 0.0
            c[n + 1] = -2.0 / (p * p) * (r0 * c[n] + prev) / (n + 1)
    else:
        raise ValueError(kind)
    return c


def kernel(kind: str, p: float, r):
    r = np.asarray(r, dtype=np.float64)
    if kind == "laplace":
        return np.exp(-r / p)
    if kind == "imq":
        return 1.0 / np.sqrt(r * r + p * p)
    if kind == "energy":
        return -r
    if kind == "gauss":
        return np.exp(-r * r / (p * p))
    raise ValueError(kind)


def two_point_taylor(a: float, b: float, ca, cb, x):
    """The polynomial T of degree 2P - 1 (P = len(ca)) with T^{(j)}(a)/j! = ca[j]
    and T^{(j)}(b)/j! = cb[j] for j < P, evaluated at x:
        T(x) = (1-s)^P sum_j ca_j (x-a)^j sum_{k < P-j} C(P-1+k, k) s^k
             + s^P     sum_j cb_j (x-b)^j sum_{k < P-j} C(P-1+k, k) (1-s)^k,
    s = (x - a)/(b - a).  Each bracket is the Taylor polynomial at its end
    point times 1 + O(s^{P-j}) (the truncated series of (1-s)^{-P}), so the
    derivatives of order < P at a and at b are those prescribed."""
    x = np.asarray(x, dtype=np.float64)
    P = len(ca)
    s = (x - a) / (b - a)
    ta = np.zeros_like(x)
    tb = np.zeros_like(x)
    for j in range(P):
        sa = sum(comb(P - 1 + k, k) * s ** k for k in range(P - j))
        sb = sum(comb(P - 1 + k, k) * (1.0 - s) ** k for k in range(P - j))
        ta = ta + ca[j] * (x - a) ** j * sa
        tb = tb + cb[j] * (x - b) ** j * sb
    return (1.0 - s) ** P * ta + s ** P * tb


class RegKernel:
    """K_R of the module docstring for kernel `kind` with parameter `par`,
    torus period h, smoothness p (derivatives 0..p-1 matched), eps_I, eps_B."""

    def __init__(self, kind, par, h, p, eps_i, eps_b):
        self.kind, self.par, self.h, self.p = kind, par, h, p
        self.eps_i, self.eps_b = eps_i, eps_b
        # Taylor coefficients of Kh(rbar) = K(h rbar): h^j K^{(j)}/j!
        hj = h ** np.arange(p)
        ci = taylor_coeffs(kind, par, h * eps_i, p) * hj
        cb = taylor_coeffs(kind, par, h * (0.5 - eps_b), p) * hj
        sign = (-1.0) ** np.arange(p)
        self._ci = (ci * sign, ci)                 # at -eps_I (mirror) and +eps_I
        self.k_b = float(two_point_taylor(0.5 - eps_b, 0.5 + eps_b, cb, cb * sign, 0.5))
        flat = np.zeros(p)
        flat[0] = self.k_b
        self._cb = (cb, flat)                      # at 1/2 - eps_B and at 1/2 (flat)

    def inner(self, rbar):
        return two_point_taylor(-self.eps_i, self.eps_i, self._ci[0], self._ci[1], rbar)

    def boundary(self, rbar):
        return two_point_taylor(0.5 - self.eps_b, 0.5, self._cb[0], self._cb[1], rbar)

    def __call__(self, rbar):
        r = np.asarray(rbar, dtype=np.float64)
        out = kernel(self.kind, self.par, self.h * r)
        lo = r < self.eps_i
        out = np.where(lo, self.inner(np.where(lo, r, 0.0)), out)
        hi = r > 0.5 - self.eps_b
        rb = np.minimum(np.where(hi, r, 0.5), 0.5)
        out = np.where(hi, self.boundary(rb), out)
        return np.where(r > 0.5, self.k_b, out)


def coeffs(KR: RegKernel, N: int, d: int):
    """b_k on I_N^d (shape (N,)*d, index k + N/2 per axis): the DFT of the samples
    K_R(||l||/N), l in I_N^d, divided by N^d (real: K_R is even)."""
    l = np.arange(-N // 2, N // 2, dtype=np.float64) / N
    grids = np.meshgrid(*([l] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    samples = KR(r)
    # DFT over the index set: move l = 0 to position 0, transform, move k = 0 back
    B = np.fft.fftn(np.fft.ifftshift(samples)) / N ** d
    return np.real(np.fft.fftshift(B))


def near_field(KR: RegKernel, src, w, tgt):
    """sum over |x_i - y_j| < eps_I h of w_j (K - K_R): brute force over all pairs."""
    src = np.atleast_2d(np.asarray(src, dtype=np.float64))
    tgt = np.atleast_2d(np.asarray(tgt, dtype=np.float64))
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(tgt.shape[0])
    for i in range(tgt.shape[0]):
        r = np.sqrt(np.sum((src - tgt[i]) ** 2, axis=1))
        near = r < KR.eps_i * KR.h
        if np.any(near):
            rn = r[near]
            out[i] = np.sum(w[near] * (kernel(KR.kind, KR.par, rn) - KR.inner(rn / KR.h)))
    return out


def plan(kind, par, src, tgt, N, p, eps_i=None, eps_b=None):
    """Centre, period and regularised kernel for the joint bounding box of the two
    clouds: h = (Euclidean diameter of the box) / (1/2 - eps_B), so that every
    difference stays in the region where K_R = K or the near field corrects it.
    eps_I = eps_B = p/N unless given."""
    pts = np.vstack([np.atleast_2d(src), np.atleast_2d(tgt)]).astype(np.float64)
    lo, hi = pts.min(0), pts.max(0)
    eps_i = p / N if eps_i is None else eps_i
    eps_b = p / N if eps_b is None else eps_b
    diam = float(np.sqrt(np.sum((hi - lo) ** 2)))
    h = max(diam, 1e-30) / (0.5 - eps_b)
    return 0.5 * (lo + hi), h, RegKernel(kind, par, h, p, eps_i, eps_b)


def fastsum_ndft(kind, par, src, w, tgt, N, p, eps_i=None, eps_b=None):
    """s_j = sum_i w_i K(|src_i - tgt_j|) by the regularised fast summation with
    exact trigonometric sums (no window) plus the near field."""
    center, h, KR = plan(kind, par, src, tgt, N, p, eps_i, eps_b)
    us = _nfft.torus_coords(src, center, h)
    ut = _nfft.torus_coords(tgt, center, h)
    d = us.shape[1]
    k1 = np.arange(-N // 2, N // 2, dtype=np.float64)
    grids = np.meshgrid(*([k1] * d), indexing="ij")
    K = np.stack([g.reshape(-1) for g in grids], axis=1)
    bk = coeffs(KR, N, d).reshape(-1)
    w = np.asarray(w, dtype=np.float64)
    ahat = np.exp(-2j * np.pi * (K @ us.T)) @ w
    smooth = np.real(np.exp(2j * np.pi * (ut @ K.T)) @ (bk * ahat))
    return smooth + near_field(KR, src, w, tgt)


def fastsum_window(kind, par, src, w, tgt, N, p, m, eps_i=None, eps_b=None):
    """The same with the Kaiser-Bessel window NFFT (oversampling 2, cut-off m)
    in place of the exact trigonometric sums."""
    center, h, KR = plan(kind, par, src, tgt, N, p, eps_i, eps_b)
    n = 2 * N
    us = _nfft.torus_coords(src, center, h)
    ut = _nfft.torus_coords(tgt, center, h)
    d = us.shape[1]
    g = _nfft.spread(us, w, n, N, m)
    G = np.fft.fftn(g)
    sel = np.ix_(*([_nfft._on_IN(n, N, d)] * d))
    kk = np.arange(-N // 2, N // 2)
    ph = n * _nfft.kb_phihat(kk, n, N, m)
    dec = 1.0 / (ph * ph)
    full = dec
    for _ in range(d - 1):
        full = np.multiply.outer(full, dec)
    H = np.zeros_like(G)
    H[sel] = G[sel] * coeffs(KR, N, d) * full
    hg = np.real(np.fft.ifftn(H)) * n ** d
    return _nfft.gather_window(hg, ut, N, m) + near_field(KR, src, w, tgt)
