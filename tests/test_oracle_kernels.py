"""Pins of the oracle's other kernels of Table tab:0 (Laplace, inverse
multiquadric, energy), CPU only.

* One atom each: MMD^2(a delta_x, b delta_y) = a^2 k(0) + b^2 k(0) - 2ab k(|x-y|)
  in closed form for every kernel.
* Laplace on a 1-D grid: the row sums are two geometric series.
* Energy in 1-D (Cramer): for measures of equal mass the energy MMD^2 equals
  2 * int (F_mu(t) - F_nu(t))^2 dt, F the cumulative distribution functions.
* Positive definiteness (Gauss, Laplace, IMQ): MMD^2 >= 0."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs


@pytest.mark.parametrize("kind", ["gauss", "laplace", "imq", "energy"])
def test_one_atom_closed_forms(kind):
    a, b, p = 0.7, 1.9, 0.35
    for r in (0.0, 0.1, 0.8, 2.5):
        x = np.array([[0.2, -0.1, 0.3]])
        y = x + np.array([[r, 0.0, 0.0]]) / 1.0
        k0 = {"gauss": 1.0, "laplace": 1.0, "imq": 1.0 / p, "energy": 0.0}[kind]
        kr = {"gauss": np.exp(-r * r / (p * p)), "laplace": np.exp(-r / p),
              "imq": 1.0 / np.sqrt(r * r + p * p), "energy": -r}[kind]
        want = a * a * k0 + b * b * k0 - 2 * a * b * kr
        got = oracle.mmd2_kernel(kind, p, x, [a], y, [b])
        assert abs(got - want) <= 1e-14 * max(1.0, abs(want)), (kind, r, got, want)


def test_laplace_grid_geometric_series():
    n, h, ell = 37, 0.05, 0.3
    x = (np.arange(n) * h).reshape(-1, 1)
    out = oracle.ksum_kernel("laplace", ell, x, np.ones(n), x)
    q = np.exp(-h / ell)
    i = np.arange(n)
    # sum_{k=0}^{i} q^k + sum_{k=1}^{n-1-i} q^k
    want = (1 - q ** (i + 1)) / (1 - q) + q * (1 - q ** (n - 1 - i)) / (1 - q)
    assert np.max(np.abs(out - want) / want) <= 1e-13


def test_energy_distance_is_cramer_in_1d():
    g = inputs.rng(91)
    x = g.uniform(-1, 1, 40)
    y = g.uniform(-0.5, 1.5, 25)
    a = g.uniform(0.5, 1.5, 40)
    b = g.uniform(0.5, 1.5, 25)
    b *= a.sum() / b.sum()
    got = oracle.mmd2_kernel("energy", 0.0, x.reshape(-1, 1), a, y.reshape(-1, 1), b)
    # exact integral of the squared CDF difference (piecewise constant)
    t = np.sort(np.concatenate([x, y]))
    F = np.array([a[x <= s].sum() - b[y <= s].sum() for s in t[:-1]])
    want = 2.0 * np.sum(F ** 2 * np.diff(t))
    assert abs(got - want) <= 1e-12 * want, (got, want)


@pytest.mark.parametrize("kind,p", [("gauss", 0.3), ("laplace", 0.3), ("imq", 0.5)])
def test_positive_definite_kernels_give_nonnegative_mmd(kind, p):
    g = inputs.rng(93)
    for _ in range(5):
        x = g.uniform(-1, 1, (30, 2))
        y = g.uniform(-1, 1, (20, 2))
        a = g.uniform(0.1, 1.0, 30)
        b = g.uniform(0.1, 1.0, 20)
        v, parts = oracle.mmd2_kernel(kind, p, x, a, y, b, return_parts=True)
        assert v >= -1e-14 * (parts[0] + 2 * abs(parts[1]) + parts[2])
    # identical measures give zero
    assert abs(oracle.mmd2_kernel(kind, p, x, a, x, a)) <= 1e-14 * parts[0]
