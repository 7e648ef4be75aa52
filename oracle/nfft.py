"""NFFT fast summation, plain numpy FP64 (Sec. 4 of arXiv 2306.13618).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Shares no code with the
CUDA library.

The fast summation replaces the kernel K(v) = exp(-||v||^2/eps) by an
h-periodic trigonometric polynomial (Eq. ansatz_NFFT)

    K(v) ~ sum_{k in I_N^d} b_k exp(2 pi i k.v/h),   I_N = {-N/2, ..., N/2-1},

and evaluates s(x_i) = sum_j w_j K(x_i - y_j) in the factorised form of
Eq. (1724): an adjoint NFFT of the weights at the scaled nodes, a multiply by
b_k, and an NFFT at the scaled targets.  Nodes are scaled onto the torus
(Eq. boundaries) as  xbar = (x - c)/h  in [-1/2, 1/2)^d.  For the grid we
translate the torus by 1/2, u = xbar + 1/2 in [0, 1)^d, grid node l <-> u = l/n;
a common translation of sources and targets leaves every difference, hence
every sum, unchanged.

Window (the paper leaves it to the NFFT library; reading: Kaiser-Bessel, the
standard choice of that library family) with oversampled grid n = sigma*N,
cut-off m and b = pi (2 - 1/sigma):

    phi(v)    = sinh(b sqrt(m^2 - n^2 v^2)) / (pi sqrt(m^2 - n^2 v^2)),  |v| <= m/n,
    phihat(k) = I_0(m sqrt(b^2 - (2 pi k/n)^2)) / n,                     |k| <= N/2.

Adjoint NFFT:  g_l = sum_j w_j prod_t phi~(u_jt - l_t/n);  ghat = FFT(g);
               ahat_k = ghat_k / prod_t (n phihat(k_t)).
NFFT:          hhat_k = fhat_k / prod_t (n phihat(k_t)) on I_N, 0 elsewhere;
               h = unnormalised inverse FFT(hhat);  f(u) = sum_l h_l prod_t phi~(u_t - l_t/n).
Gaussian Fourier coefficients (the h-periodised kernel, whose tails beyond one
period are negligible when h is chosen as below):
               b_k = (pi eps / h^2)^{d/2} exp(-pi^2 eps ||k||^2 / h^2).
"""
from __future__ import annotations

import numpy as np
from scipy.special import i0


def kb_params(n: int, N: int) -> float:
    """Kaiser-Bessel shape parameter b = pi (2 - 1/sigma), sigma = n/N."""
    sigma = n / N
    return np.pi * (2.0 - 1.0 / sigma)


def kb_phi(v, n: int, N: int, m: int):
    """Truncated Kaiser-Bessel window phi(v), zero for |v| > m/n (v not periodised)."""
    v = np.asarray(v, dtype=np.float64)
    b = kb_params(n, N)
    s2 = m * m - (n * v) ** 2
    out = np.zeros_like(v)
    pos = s2 > 0
    s = np.sqrt(s2[pos])
    out[pos] = np.sinh(b * s) / (np.pi * s)
    edge = s2 == 0
    out[edge] = b / np.pi
    return out


def kb_phihat(k, n: int, N: int, m: int):
    """Fourier coefficient phihat(k) = int phi(v) e^{-2 pi i k v} dv of the window."""
    k = np.asarray(k, dtype=np.float64)
    b = kb_params(n, N)
    return i0(m * np.sqrt(b * b - (2.0 * np.pi * k / n) ** 2)) / n


def gauss_coeffs(N: int, d: int, eps: float, h: float):
    """b_k on I_N^d (array of shape (N,)*d, index k + N/2 along each axis)."""
    k = np.arange(-N // 2, N // 2, dtype=np.float64)
    one = np.sqrt(np.pi * eps) / h * np.exp(-np.pi ** 2 * eps * k * k / (h * h))
    out = one
    for _ in range(d - 1):
        out = np.multiply.outer(out, one)
    return out


def torus_coords(p, center, h):
    """u = (p - c)/h + 1/2, reduced mod 1 into [0, 1)^d (FP64)."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    u = (p - np.asarray(center, dtype=np.float64)) / h + 0.5
    return u - np.floor(u)


def cell_index_f32(p, center, inv_h, n):
    """Grid cell of each coordinate in FP32 arithmetic, one IEEE rounding per step:
    u = ((p - c) * inv_h + 0.5) * n;  cell = floor(u) mod n.  Inputs are taken as
    FP32 values.  This is the binning rule stated bit for bit."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float32))
    c = np.asarray(center, dtype=np.float32)
    t = np.subtract(p, c, dtype=np.float32)
    t = np.multiply(t, np.float32(inv_h), dtype=np.float32)
    t = np.add(t, np.float32(0.5), dtype=np.float32)
    t = np.multiply(t, np.float32(n), dtype=np.float32)
    cell = np.floor(t).astype(np.int64)
    return np.mod(cell, n)


def _footprint(u, n, N, m):
    """For coordinates u (P,) in [0,1): grid indices (P, 2m) and window weights (P, 2m).

    The window touches the 2m nodes l = floor(n u) - m + 1 .. floor(n u) + m."""
    base = np.floor(n * u).astype(np.int64)
    off = np.arange(-m + 1, m + 1)
    idx = base[:, None] + off[None, :]
    dist = u[:, None] - idx / n          # distance to the node, |dist| < m/n
    wts = kb_phi(dist, n, N, m)
    return np.mod(idx, n), wts


def spread(u, w, n, N, m):
    """Adjoint-NFFT step 1: g_l = sum_j w_j prod_t phi~(u_jt - l_t/n) on the n^d grid."""
    u = np.atleast_2d(u)
    P, d = u.shape
    w = np.asarray(w, dtype=np.float64)
    g = np.zeros((n,) * d)
    fp = [_footprint(u[:, t], n, N, m) for t in range(d)]
    if d == 1:
        np.add.at(g, fp[0][0], w[:, None] * fp[0][1])
    elif d == 2:
        (ix, wx), (iy, wy) = fp
        # axis order of the grid: (x1, x2) -> g[x1, x2]
        val = w[:, None, None] * wx[:, :, None] * wy[:, None, :]
        np.add.at(g, (ix[:, :, None], iy[:, None, :]), val)
    else:
        (ix, wx), (iy, wy), (iz, wz) = fp
        for s in range(0, P, 256):
            sl = slice(s, s + 256)
            val = (w[sl, None, None, None] * wx[sl, :, None, None]
                   * wy[sl, None, :, None] * wz[sl, None, None, :])
            np.add.at(g, (ix[sl, :, None, None], iy[sl, None, :, None],
                          iz[sl, None, None, :]), val)
    return g


def gather_window(hgrid, u, N, m):
    """NFFT final step: f(u_i) = sum_l h_l prod_t phi~(u_it - l_t/n)."""
    u = np.atleast_2d(u)
    P, d = u.shape
    n = hgrid.shape[0]
    fp = [_footprint(u[:, t], n, N, m) for t in range(d)]
    out = np.empty(P)
    if d == 1:
        out[:] = np.sum(hgrid[fp[0][0]] * fp[0][1], axis=1)
    elif d == 2:
        (ix, wx), (iy, wy) = fp
        vals = hgrid[ix[:, :, None], iy[:, None, :]]
        out[:] = np.einsum("pab,pa,pb->p", vals, wx, wy)
    else:
        (ix, wx), (iy, wy), (iz, wz) = fp
        for s in range(0, P, 256):
            sl = slice(s, s + 256)
            vals = hgrid[ix[sl, :, None, None], iy[sl, None, :, None], iz[sl, None, None, :]]
            out[sl] = np.einsum("pabc,pa,pb,pc->p", vals, wx[sl], wy[sl], wz[sl])
    return out


def _on_IN(n, N, d):
    """Index arrays selecting I_N^d inside an n^d FFT array, in k = -N/2..N/2-1 order."""
    k = np.arange(-N // 2, N // 2)
    return np.mod(k, n)


def deconv_scale(n, N, m, d, eps, h):
    """scale_k = b_k / prod_t (n phihat(k_t))^2 on I_N^d: the multiply of Eq. (1724)
    together with the deconvolutions of the adjoint and of the forward NFFT."""
    k = np.arange(-N // 2, N // 2)
    ph = n * kb_phihat(k, n, N, m)
    one = 1.0 / (ph * ph)
    dec = one
    for _ in range(d - 1):
        dec = np.multiply.outer(dec, one)
    return gauss_coeffs(N, d, eps, h) * dec


def convolve_grid(g, N, m, eps, h):
    """FFT(g) -> multiply by scale_k on I_N^d (zero elsewhere) -> unnormalised inverse FFT."""
    d = g.ndim
    n = g.shape[0]
    G = np.fft.fftn(g)
    sel = np.ix_(*([_on_IN(n, N, d)] * d))
    H = np.zeros_like(G)
    H[sel] = G[sel] * deconv_scale(n, N, m, d, eps, h)
    return np.real(np.fft.ifftn(H)) * n ** d


def fastsum_window(src, w, tgt, eps, center, h, n, N, m):
    """NFFT fast summation with the window method, all steps in FP64."""
    us = torus_coords(src, center, h)
    ut = torus_coords(tgt, center, h)
    g = spread(us, w, n, N, m)
    hg = convolve_grid(g, N, m, eps, h)
    return gather_window(hg, ut, N, m)


def fastsum_ndft(src, w, tgt, eps, center, h, N):
    """Fast summation Eq. (1724) with exact trigonometric sums (no window):
    ahat_k = sum_j w_j e^{-2 pi i k.u_j}, s_i = sum_k b_k ahat_k e^{2 pi i k.u_i}."""
    us = torus_coords(src, center, h)
    ut = torus_coords(tgt, center, h)
    d = us.shape[1]
    k1 = np.arange(-N // 2, N // 2, dtype=np.float64)
    grids = np.meshgrid(*([k1] * d), indexing="ij")
    K = np.stack([g.reshape(-1) for g in grids], axis=1)        # (N^d, d)
    bk = gauss_coeffs(N, d, eps, h).reshape(-1)
    w = np.asarray(w, dtype=np.float64)
    ahat = np.exp(-2j * np.pi * (K @ us.T)) @ w                   # (N^d,)
    return np.real(np.exp(2j * np.pi * (ut @ K.T)) @ (bk * ahat))


def choose_h(points_span: float, eps: float, tail: float = 1e-8) -> float:
    """Torus period: every difference x_i - y_j has to stay inside one period
    together with the kernel's effective support sqrt(eps ln(1/tail)):
    h >= span + sqrt(eps ln(1/tail))."""
    return points_span + np.sqrt(eps * np.log(1.0 / tail))
