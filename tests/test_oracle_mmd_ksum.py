"""Pins of the oracle's kernel sum and MMD^2 (Eq. 1205, Gaussian kernel of
Table tab:0) against closed forms, invariants and bounds.  CPU only."""
import numpy as np
import pytest

import oracle


def test_ksum_separable_grid(oracle_lib):
    """On a tensor-product source grid with product weights the Gaussian sum
    factorises into 1-D sums: a check of the squared distance over every axis."""
    g = np.random.default_rng(0)
    a = g.uniform(-0.3, 0.3, 7); b = g.uniform(-0.3, 0.3, 5); c = g.uniform(-0.3, 0.3, 4)
    wa = g.uniform(0.5, 1.5, 7); wb = g.uniform(0.5, 1.5, 5); wc = g.uniform(0.5, 1.5, 4)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    src = np.stack([A.ravel(), B.ravel(), C.ravel()], 1)
    w = np.einsum("i,j,k->ijk", wa, wb, wc).ravel()
    tgt = g.uniform(-0.4, 0.4, (9, 3))
    eps = 0.07
    got = oracle.ksum(src, w, tgt, eps)
    f = lambda p, wp, t: np.sum(wp * np.exp(-(p - t) ** 2 / eps))
    want = np.array([f(a, wa, t[0]) * f(b, wb, t[1]) * f(c, wc, t[2]) for t in tgt])
    assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_ksum_gaussian_integral(oracle_lib):
    """Riemann sum of a Gaussian on a fine 1-D lattice: spacing*sum = sqrt(pi eps)
    up to exp(-pi^2 eps/spacing^2) (Poisson summation) -- exact to ~1e-15 here."""
    eps, hsp = 0.01, 0.01
    src = np.arange(-200, 201) * hsp
    out = oracle.ksum(src, np.full(src.size, hsp), np.array([0.0, 0.003, -0.0071]), eps)
    assert np.allclose(out, np.sqrt(np.pi * eps), rtol=1e-13, atol=0)


def test_ksum_translation_and_symmetry(oracle_lib):
    g = np.random.default_rng(1)
    x = g.uniform(-0.3, 0.3, (40, 3)); y = g.uniform(-0.3, 0.3, (30, 3))
    u = g.uniform(0.5, 1.5, 40); v = g.uniform(0.5, 1.5, 30)
    s = np.array([0.7, -1.1, 0.4])
    k1 = oracle.ksum(x, u, y, 0.05)
    k2 = oracle.ksum(x + s, u, y + s, 0.05)
    assert np.allclose(k1, k2, rtol=1e-13)
    # v^T (K u) = u^T (K^T v)
    assert np.isclose(v @ k1, u @ oracle.ksum(y, v, x, 0.05), rtol=1e-13)


def test_mmd_one_point(oracle_lib):
    """One atom each: MMD^2 = a^2 + b^2 - 2ab exp(-D/ell^2)."""
    x = np.array([[0.1, 0.2, -0.1]]); y = np.array([[-0.2, 0.0, 0.3]])
    a, b, ell = 0.7, 1.9, 0.3
    D = np.sum((x - y) ** 2)
    want = a * a + b * b - 2 * a * b * np.exp(-D / ell ** 2)
    assert np.isclose(oracle.mmd2(x, [a], y, [b], ell), want, rtol=1e-14)


def test_mmd_identity_symmetry_bound(oracle_lib):
    g = np.random.default_rng(2)
    x = g.uniform(-0.25, 0.25, (200, 2)); y = g.uniform(-0.2, 0.3, (150, 2))
    mu = g.uniform(0.5, 1.5, 200); mu /= mu.sum()
    nu = g.uniform(0.5, 1.5, 150); nu *= 1.3 / nu.sum()
    v, (A, B, C) = oracle.mmd2(x, mu, y, nu, 0.2, return_parts=True)
    assert v > 0
    assert np.isclose(v, oracle.mmd2(y, nu, x, mu, 0.2), rtol=1e-13)
    assert v <= mu.sum() ** 2 + nu.sum() ** 2            # Eq. (731), ||k||_inf = 1
    z = oracle.mmd2(x, mu, x, mu, 0.2)
    assert abs(z) <= 8 * np.finfo(float).eps * (A + 2 * abs(B) + C)


def _E(var, delta2, ell, d):
    """E exp(-||Z||^2/ell^2) for Z ~ N(delta, var I_d)."""
    return (ell ** 2 / (ell ** 2 + 2 * var)) ** (d / 2) * np.exp(-delta2 / (ell ** 2 + 2 * var))


def test_mmd_gaussian_measures_expectation(oracle_lib):
    """mu = m1 * empirical N(alpha, s1^2 I), nu = m2 * empirical N(beta, s2^2 I) with
    uniform weights: the expected V-statistic is
      m1^2 [1/n + (1-1/n) E(2 s1^2, 0)] + m2^2 [1/m + (1-1/m) E(2 s2^2, 0)]
      - 2 m1 m2 E(s1^2 + s2^2, alpha - beta),
    checked on the mean over seeded replicates within 5 standard errors."""
    d, n, m, ell = 3, 60, 45, 0.4
    s1, s2, m1, m2 = 0.15, 0.25, 1.0, 0.8
    al = np.array([0.1, 0.0, -0.05]); be = np.array([-0.1, 0.1, 0.05])
    want = (m1 ** 2 * (1 / n + (1 - 1 / n) * _E(2 * s1 ** 2, 0.0, ell, d))
            + m2 ** 2 * (1 / m + (1 - 1 / m) * _E(2 * s2 ** 2, 0.0, ell, d))
            - 2 * m1 * m2 * _E(s1 ** 2 + s2 ** 2, np.sum((al - be) ** 2), ell, d))
    g = np.random.default_rng(3)
    vals = []
    for _ in range(400):
        x = al + s1 * g.standard_normal((n, d))
        y = be + s2 * g.standard_normal((m, d))
        vals.append(oracle.mmd2(x, np.full(n, m1 / n), y, np.full(m, m2 / m), ell))
    vals = np.array(vals)
    se = vals.std(ddof=1) / np.sqrt(len(vals))
    assert abs(vals.mean() - want) < 5 * se
    assert se < 0.05 * want


def test_mmd_detects_planted_error(oracle_lib):
    """The Gaussian-measure pin is sharp enough to catch a wrong length-scale
    convention (exp(-d^2/(2 ell^2)) instead of exp(-d^2/ell^2))."""
    d, n, m, ell = 2, 80, 80, 0.3
    g = np.random.default_rng(4)
    al = np.zeros(d); be = np.array([0.2, 0.0])
    want_wrong = (1 / n + (1 - 1 / n) * _E(2 * 0.01, 0, np.sqrt(2) * ell, d)) * 2 \
        - 2 * _E(0.02, 0.04, np.sqrt(2) * ell, d)
    want = (1 / n + (1 - 1 / n) * _E(2 * 0.01, 0, ell, d)) * 2 - 2 * _E(0.02, 0.04, ell, d)
    vals = [oracle.mmd2(al + 0.1 * g.standard_normal((n, d)), np.full(n, 1 / n),
                        be + 0.1 * g.standard_normal((m, d)), np.full(m, 1 / m), ell)
            for _ in range(200)]
    se = np.std(vals, ddof=1) / np.sqrt(len(vals))
    assert abs(np.mean(vals) - want) < 5 * se
    assert abs(np.mean(vals) - want_wrong) > 20 * se
