"""Pins of the NFFT fast-summation oracle (Sec. 4) against quadrature, exact
trigonometric sums, the exact kernel sum and special cases.  CPU only."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
import oracle.nfft as nf


@pytest.mark.parametrize("n,N,m", [(128, 64, 6), (64, 32, 8), (32, 16, 4)])
def test_phihat_is_fourier_transform_of_window(n, N, m):
    """phihat(k) against adaptive quadrature of the truncated window; they differ
    only by the window's tail beyond m/n, of relative size about exp(-b m)."""
    tol = max(1e-11, 10 * np.exp(-nf.kb_params(n, N) * m))
    for k in (0, 1, N // 4, N // 2 - 1, N // 2):
        f = lambda v: nf.kb_phi(np.array([v]), n, N, m)[0] * np.cos(2 * np.pi * k * v)
        val, err = quad(f, -m / n, m / n, limit=400, epsabs=0, epsrel=1e-13)
        ph = nf.kb_phihat(k, n, N, m)
        assert abs(val - ph) <= tol * abs(ph), (k, val, ph)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_gauss_coeffs_match_dft_of_samples(d):
    """b_k analytic against the DFT of the h-periodised kernel sampled on a grid."""
    eps, h, N, M = 0.05, 1.6, 16, 64
    t = (np.arange(M) - M // 2) / M * h
    per = sum(np.exp(-(t + r * h) ** 2 / eps) for r in (-2, -1, 0, 1, 2))
    one = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(per))) / M
    one = one[M // 2 - N // 2: M // 2 + N // 2].real
    want = one
    for _ in range(d - 1):
        want = np.multiply.outer(want, one)
    got = nf.gauss_coeffs(N, d, eps, h)
    assert np.allclose(got, want, rtol=0, atol=1e-14)


def _cloud(g, n, d, lo=-0.3, hi=0.3):
    return g.uniform(lo, hi, (n, d))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_window_matches_exact_trig_sums(d):
    """Spread + FFT + deconvolution + gather (window method) equals the exact
    trigonometric sums of Eq. (1724) up to the window error (m = 8)."""
    g = np.random.default_rng(d)
    src, tgt = _cloud(g, 300, d), _cloud(g, 200, d)
    w = g.uniform(0.5, 1.5, 300)
    eps, N = 0.05, 16
    h = nf.choose_h(0.6, eps)
    fw = nf.fastsum_window(src, w, tgt, eps, np.zeros(d), h, 2 * N, N, 8)
    fn = nf.fastsum_ndft(src, w, tgt, eps, np.zeros(d), h, N)
    assert np.max(np.abs(fw - fn)) <= 1e-11 * w.sum()


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fastsum_matches_exact_kernel_sum(oracle_lib, d):
    """Eq. (1724) with N = 32 against the exact kernel sum: the truncation of b_k
    at |k| = N/2 and the periodisation are below 1e-12 relative to sum |w|."""
    g = np.random.default_rng(10 + d)
    src, tgt = _cloud(g, 250, d), _cloud(g, 150, d)
    w = g.uniform(0.5, 1.5, 250)
    eps, N = 0.05, 32
    h = nf.choose_h(0.6, eps, tail=1e-16)
    fn = nf.fastsum_window(src, w, tgt, eps, np.zeros(d), h, 2 * N, N, 8)
    ex = oracle.ksum(src, w, tgt, eps)
    assert np.max(np.abs(fn - ex)) <= 1e-12 * w.sum()


def test_single_source_delta(oracle_lib):
    """One source: s(x) = w exp(-||x - x0||^2 / eps) at every target."""
    g = np.random.default_rng(5)
    x0 = np.array([[0.05, -0.1, 0.12]])
    tgt = _cloud(g, 100, 3)
    eps = 0.03
    h = nf.choose_h(0.6, eps, tail=1e-14)
    f = nf.fastsum_window(x0, [2.5], tgt, eps, np.zeros(3), h, 64, 32, 8)
    want = 2.5 * np.exp(-np.sum((tgt - x0) ** 2, 1) / eps)
    assert np.max(np.abs(f - want)) < 1e-11


def test_error_decreases_with_cutoff(oracle_lib):
    g = np.random.default_rng(6)
    src, tgt = _cloud(g, 200, 3), _cloud(g, 100, 3)
    w = g.uniform(0.5, 1.5, 200)
    eps, N = 0.05, 16
    h = nf.choose_h(0.6, eps)
    ref = nf.fastsum_ndft(src, w, tgt, eps, np.zeros(3), h, N)
    errs = [np.max(np.abs(nf.fastsum_window(src, w, tgt, eps, np.zeros(3), h, 2 * N, N, m) - ref))
            for m in (2, 3, 4, 5, 6)]
    assert all(errs[i + 1] < 0.2 * errs[i] for i in range(len(errs) - 1)), errs


def test_adjoint_nfft_stage_against_ndft():
    """Spread + FFT + deconvolution alone reproduces the exact adjoint NDFT
    ahat_k = sum_j w_j exp(-2 pi i k.u_j) on I_N^3."""
    g = np.random.default_rng(7)
    n, N, m = 32, 16, 7
    u = g.uniform(0, 1, (150, 3))
    w = g.uniform(-1, 1, 150)
    G = np.fft.fftn(nf.spread(u, w, n, N, m))
    k = np.arange(-N // 2, N // 2)
    sel = np.ix_(*([np.mod(k, n)] * 3))
    ph = n * nf.kb_phihat(k, n, N, m)
    ahat = G[sel] / np.einsum("i,j,k->ijk", ph, ph, ph)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    exact = (np.exp(-2j * np.pi * (K @ u.T)) @ w).reshape(N, N, N)
    assert np.max(np.abs(ahat - exact)) <= 1e-9 * np.abs(w).sum()


def test_cell_index_f32_agrees_with_exact_away_from_edges():
    """The FP32 binning rule agrees with exact floor((x-c)/h + 1/2) n except for
    coordinates within a few FP32 ulps of a cell edge."""
    g = np.random.default_rng(8)
    p = g.uniform(-0.4, 0.4, (20000, 3)).astype(np.float32)
    c = np.array([0.01, -0.02, 0.0], dtype=np.float32)
    h = 1.7
    inv_h = np.float32(1.0 / h)
    cells = nf.cell_index_f32(p, c, inv_h, 128)
    u = ((p.astype(np.float64) - c.astype(np.float64)) * float(inv_h) + 0.5) * 128
    exact = np.mod(np.floor(u).astype(np.int64), 128)
    near = np.abs(u - np.round(u)) < 1e-4
    assert np.array_equal(cells[~near], exact[~near])
    assert near.mean() < 1e-3


@pytest.mark.parametrize("m", [4, 6, 8])
def test_footprint_holds_the_window_support(m):
    """The 2m nodes floor(nu) - m + 1 .. floor(nu) + m per axis hold the whole
    support |v| <= m/n of the window: the nodes one further out on either side
    carry phi = 0, except node floor(nu) - m when u sits on a grid node (f = 0),
    where v = m/n exactly and phi = b/pi, a fraction bm/sinh(bm) of phi(0)
    (3e-11 at m = 6, sigma = 2)."""
    n, N = 128, 64
    g = np.random.default_rng(5)
    u = np.concatenate([g.uniform(0, 1, 4000), np.arange(n) / n])
    base = np.floor(n * u)
    f = n * u - base
    for off in (-m - 1, m + 1, m + 2):
        assert np.all(nf.kb_phi(u - (base + off) / n, n, N, m) == 0.0)
    edge = nf.kb_phi(u - (base - m) / n, n, N, m)
    assert np.all(edge[f > 0] == 0.0)
    b = nf.kb_params(n, N)
    assert np.allclose(edge[f == 0], b / np.pi, rtol=1e-14)
    ratio = b / np.pi / nf.kb_phi(0.0, n, N, m)
    assert ratio == pytest.approx(b * m / np.sinh(b * m), rel=1e-12)
    if m >= 6:
        assert ratio < 1e-10
    for off in range(-m + 1, m + 1):
        assert np.all(np.abs(u - (base + off) / n) <= m / n)


def test_gaussian_convolution_is_three_circulants():
    """For the Gaussian, b_k / prod_t (n phihat(k_t))^2 is a product over the
    axes, so the grid convolution of Eq. (1724) is one real circulant n x n
    operator, C[a, i] = sum_k s(k) cos(2 pi k (a - i)/n), applied along each
    axis: a dense restatement of the oracle's FFT pipeline.  The unpaired
    frequency -N/2 of I_N contributes a sine part of relative size
    exp(-pi^2 eps N^2 / (4 h^2)), e^-63 here and e^-64 for the 2^20 workload."""
    n, N, m, eps, h = 32, 16, 4, 0.1, 1.0
    g = np.random.default_rng(7).standard_normal((n, n, n))
    want = nf.convolve_grid(g, N, m, eps, h)
    k = np.arange(-N // 2, N // 2)
    s = nf.gauss_coeffs(N, 1, eps, h) / (n * nf.kb_phihat(k, n, N, m)) ** 2
    a = np.arange(n)
    C = np.cos(2 * np.pi * np.subtract.outer(a, a)[:, :, None] * k / n) @ s
    got = np.einsum("ai,bj,ck,ijk->abc", C, C, C, g, optimize=True)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
