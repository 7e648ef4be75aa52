"""Pins of the oracle's regularised fast summation for the non-smooth kernels
(Sec. 4.2; oracle/nfft_reg.py), CPU only.

* Two-point Taylor interpolation: exact on polynomials of degree <= 2p - 1, and
  its Taylor coefficients at both end points are the prescribed ones.
* Kernel Taylor coefficients: closed-form first and second derivatives, and the
  Taylor series summed to high order reproduces the kernel.
* K_R: equal to K between the two regularised pieces, continuous with matching
  first derivatives at every joint, flat at 1/2.
* b_k: the inverse DFT returns the samples of K_R; real and even.
* Splitting: the dense sum of K_R plus the near field is the exact kernel sum
  (no Fourier error), and the Fourier series (exact trigonometric sums, and the
  windowed NFFT) approaches the exact sum as N grows."""
import math

import numpy as np
import pytest

import oracle
from oracle import nfft_reg as R
from paper_2306_13618_gb300 import inputs


@pytest.mark.parametrize("P", [2, 4, 6])
def test_two_point_taylor_reproduces_polynomials(P):
    g = inputs.rng(30 + P)
    coef = g.standard_normal(2 * P)          # degree 2P - 1
    a, b = -0.3, 0.45
    poly = np.polynomial.Polynomial(coef)
    ca = [poly.deriv(j)(a) / math.factorial(j) if j else poly(a) for j in range(P)]
    cb = [poly.deriv(j)(b) / math.factorial(j) if j else poly(b) for j in range(P)]
    x = np.linspace(a - 0.1, b + 0.1, 41)
    assert np.allclose(R.two_point_taylor(a, b, ca, cb, x), poly(x), rtol=0, atol=1e-11)


def test_two_point_taylor_end_derivatives():
    P = 5
    g = inputs.rng(37)
    ca, cb = g.standard_normal(P), g.standard_normal(P)
    a, b = 0.1, 0.6
    # T is a polynomial of degree 2P - 1: recover it from 2P + 6 samples
    x = np.linspace(a, b, 2 * P + 6)
    T = np.polynomial.Polynomial.fit(x, R.two_point_taylor(a, b, ca, cb, x), 2 * P - 1)
    for j in range(P):
        f = math.factorial(j)
        dj = T.deriv(j) if j else T
        assert abs(dj(a) / f - ca[j]) <= 1e-7 * max(1.0, abs(ca[j])), (j, dj(a) / f, ca[j])
        assert abs(dj(b) / f - cb[j]) <= 1e-7 * max(1.0, abs(cb[j])), (j, dj(b) / f, cb[j])


def test_kernel_taylor_coefficients_closed_forms():
    r0, p = 0.37, 0.8
    c = R.taylor_coeffs("imq", p, r0, 3)
    g0 = r0 * r0 + p * p
    assert c[1] == pytest.approx(-r0 * g0 ** -1.5, rel=1e-14)
    assert c[2] == pytest.approx((2 * r0 * r0 - p * p) * g0 ** -2.5 / 2, rel=1e-13)
    c = R.taylor_coeffs("gauss", p, r0, 3)
    e = np.exp(-r0 * r0 / (p * p))
    assert c[1] == pytest.approx(-2 * r0 / p ** 2 * e, rel=1e-14)
    assert c[2] == pytest.approx((2 * r0 ** 2 / p ** 4 - 1 / p ** 2) * e, rel=1e-13)
    c = R.taylor_coeffs("laplace", p, r0, 4)
    assert c[3] == pytest.approx(-np.exp(-r0 / p) / (6 * p ** 3), rel=1e-14)
    assert list(R.taylor_coeffs("energy", 1.0, r0, 4)) == [-r0, -1.0, 0.0, 0.0]


@pytest.mark.parametrize("kind,p", [("laplace", 0.5), ("imq", 1.0), ("gauss", 0.7)])
def test_kernel_taylor_series_sums_to_kernel(kind, p):
    r0 = 0.6
    c = R.taylor_coeffs(kind, p, r0, 40)
    for t in (-0.2, 0.05, 0.3):
        series = sum(c[j] * t ** j for j in range(40))
        assert abs(series - R.kernel(kind, p, r0 + t)) <= 1e-13


@pytest.mark.parametrize("kind,par", [("laplace", 0.5), ("imq", 1.0), ("energy", 1.0)])
def test_regularised_kernel_joints(kind, par):
    h, p, ei, eb = 3.2, 5, 0.07, 0.09
    KR = R.RegKernel(kind, par, h, p, ei, eb)
    mid = np.linspace(ei, 0.5 - eb, 17)
    assert np.allclose(KR(mid), R.kernel(kind, par, h * mid), rtol=1e-14, atol=1e-14)
    # value and first derivative continuous across eps_I, 1/2 - eps_B and 1/2
    dx = 1e-6
    for r in (ei, 0.5 - eb, 0.5):
        left, right = KR(r - dx), KR(r + dx)
        scale = max(1.0, abs(float(KR(r))))
        assert abs(right - left) <= 1e-4 * scale * h, (r, left, right)
        dl = (KR(r - dx) - KR(r - 2 * dx)) / dx
        dr = (KR(r + 2 * dx) - KR(r + dx)) / dx
        assert abs(dl - dr) <= 1e-3 * max(1.0, abs(dl)) * h, (r, dl, dr)
    # even in rbar and flat beyond 1/2
    assert abs(KR(0.6) - KR.k_b) == 0.0
    d1 = (KR(0.5 - 1e-5) - KR(0.5 - 2e-5)) / 1e-5
    assert abs(d1) <= 1e-6 * h * max(1.0, abs(KR.k_b))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_coefficients_are_the_dft_of_the_samples(d):
    N = 16
    KR = R.RegKernel("laplace", 0.5, 2.5, 4, 4 / N, 4 / N)
    B = R.coeffs(KR, N, d)
    l = np.arange(-N // 2, N // 2) / N
    grids = np.meshgrid(*([l] * d), indexing="ij")
    samples = KR(np.sqrt(sum(g * g for g in grids)))
    # s_l = sum_k b_k e^{2 pi i k.l / N}: the inverse of the transform in coeffs()
    back = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(B))) * N ** d
    assert np.allclose(back.real, samples, rtol=0, atol=1e-13)
    # real and even (K_R is even): b_{-k} = b_k for -k inside I_N
    flip = B[(slice(1, None),) * d][(slice(None, None, -1),) * d]
    assert np.allclose(B[(slice(1, None),) * d], flip, rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind,par", [("laplace", 0.5), ("imq", 1.0), ("energy", 1.0)])
def test_dense_regularised_sum_plus_near_field_is_exact(kind, par):
    g = inputs.rng(41)
    x = g.uniform(0, 1, (120, 2))
    y = g.uniform(0, 1, (90, 2))
    w = g.uniform(0.1, 1.0, 120)
    center, h, KR = R.plan(kind, par, x, y, 32, 4)
    r = np.sqrt(np.sum((x[None, :, :] - y[:, None, :]) ** 2, axis=2)) / h
    assert r.max() <= 0.5 - KR.eps_b
    dense = (KR(r) * w[None, :]).sum(1)
    got = dense + R.near_field(KR, x, w, y)
    ref = oracle.ksum_kernel(kind, par, x, w, y)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)
    assert np.any(r < KR.eps_i)                 # the near field is exercised


@pytest.mark.parametrize("kind,par", [("laplace", 0.5), ("imq", 1.0), ("energy", 1.0)])
def test_fast_summation_converges_to_the_kernel_sum(kind, par):
    g = inputs.rng(43)
    x = g.uniform(0, 1, (150, 2))
    y = g.uniform(0, 1, (140, 2))
    w = g.uniform(0.0, 1.0, 150)
    ref = oracle.ksum_kernel(kind, par, x, w, y)
    scale = np.sum(w) * np.max(np.abs(ref)) / np.sum(w)
    errs = []
    for N in (16, 32, 64):
        s = R.fastsum_ndft(kind, par, x, w, y, N, 4)
        errs.append(np.max(np.abs(s - ref)) / scale)
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= 1e-5, errs


def test_window_nfft_matches_exact_trigonometric_sums():
    g = inputs.rng(47)
    x = g.uniform(0, 1, (100, 3))
    y = g.uniform(0, 1, (80, 3))
    w = g.uniform(0.1, 1.0, 100)
    a = R.fastsum_ndft("laplace", 0.5, x, w, y, 16, 4)
    b = R.fastsum_window("laplace", 0.5, x, w, y, 16, 4, 8)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.sum(w)
