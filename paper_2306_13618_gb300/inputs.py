"""Seeded synthetic workloads (no arithmetic of the method lives here).

Every generator draws from numpy's Philox-4x32 counter-based bit generator with
an explicit seed, produces FP64 values and rounds them once to FP32, so the
CUDA library and the FP64 oracle see bit-identical inputs (the oracle promotes
the FP32 values to FP64).

Workloads (shapes and distributions of the measured configurations):

* ``uniform_box``  -- n = m = 2000 points in d = 2, uniform on [-1/4, 1/4]^2,
  weights uniform on [0.5, 1.5] normalised to masses 1.0 (source) and 1.3
  (target); eps = 0.05 (lambda = 20 of Table tab:Sinkhorn3), rho = 1 (eta = 1),
  100 sweeps; MMD^2 with ell = 0.2.
* ``gmm3``  -- n = m = 2^20 points in d = 3 drawn from a five-component
  isotropic Gaussian mixture (equal mixture weights, means uniform on
  [-0.2, 0.2]^3, standard deviation 0.03), source and target independent draws
  of the same mixture; weights lognormal(0, 0.5) normalised to masses 1.0 and
  0.8; eps = 0.02, rho = 0.5, 200 sweeps.
* ``gauss64`` -- n = m = 262144 points in d = 64: source N(0, I/64), target
  an independent draw of N(0.1 e_1, I/64) (the same cloud shifted by 0.1 along
  the first axis); uniform weights with masses 1.0 and 1.2; eps = 1, rho = 2.
  The high-dimensional case of the direct form.
* ``paper_uniform`` -- the paper's own synthetic measures (Sec. 5.1.1): points and
  weights i.i.d. uniform on [0, 1] (unnormalised).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclass
class Workload:
    name: str
    x: np.ndarray          # (n, d) float32, source support
    a: np.ndarray          # (n,) float32, source weights mu
    y: np.ndarray          # (m, d) float32, target support
    b: np.ndarray          # (m,) float32, target weights nu
    eps: float             # kernel width, K = exp(-||x-y||^2/eps), lambda = 1/eps
    rho: float             # KL marginal penalty eta
    sweeps: int
    ell: float             # MMD Gaussian length scale, k = exp(-||x-y||^2/ell^2)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.x.shape[0]

    @property
    def m(self):
        return self.y.shape[0]

    @property
    def d(self):
        return self.x.shape[1]


def _normalise(w, mass):
    w = np.asarray(w, dtype=np.float64)
    return (w * (mass / w.sum())).astype(np.float32)


def uniform_box(seed: int = 1000, n: int = 2000, m: int = 2000, d: int = 2) -> Workload:
    g = rng(seed)
    x = g.uniform(-0.25, 0.25, (n, d)).astype(np.float32)
    y = g.uniform(-0.25, 0.25, (m, d)).astype(np.float32)
    a = _normalise(g.uniform(0.5, 1.5, n), 1.0)
    b = _normalise(g.uniform(0.5, 1.5, m), 1.3)
    return Workload("uniform_box", x, a, y, b, eps=0.05, rho=1.0, sweeps=100, ell=0.2)


def gmm_points(g: np.random.Generator, count: int, means: np.ndarray, std: float) -> np.ndarray:
    comp = g.integers(0, means.shape[0], count)
    return (means[comp] + std * g.standard_normal((count, means.shape[1]))).astype(np.float32)


def gmm3(seed: int = 2000, n: int = 1 << 20, m: int = 1 << 20, d: int = 3,
         components: int = 5) -> Workload:
    g = rng(seed)
    means = g.uniform(-0.2, 0.2, (components, d))
    x = gmm_points(g, n, means, 0.03)
    y = gmm_points(g, m, means, 0.03)
    a = _normalise(g.lognormal(0.0, 0.5, n), 1.0)
    b = _normalise(g.lognormal(0.0, 0.5, m), 0.8)
    return Workload("gmm3", x, a, y, b, eps=0.02, rho=0.5, sweeps=200, ell=0.2,
                    extra={"means": means})


def gauss64(seed: int = 3000, n: int = 262144, m: int = 262144, d: int = 64) -> Workload:
    g = rng(seed)
    x = (g.standard_normal((n, d)) / 8.0).astype(np.float32)
    shift = np.zeros(d)
    shift[0] = 0.1
    y = (g.standard_normal((m, d)) / 8.0 + shift).astype(np.float32)
    a = np.full(n, 1.0 / n, dtype=np.float32)
    b = np.full(m, 1.2 / m, dtype=np.float32)
    return Workload("gauss64", x, a, y, b, eps=1.0, rho=2.0, sweeps=100, ell=1.0)


def paper_uniform(seed: int = 3000, n: int = 1000, d: int = 3, eps: float = 0.05,
                  rho: float = 1.0) -> Workload:
    g = rng(seed)
    x = g.uniform(0.0, 1.0, (n, d)).astype(np.float32)
    y = g.uniform(0.0, 1.0, (n, d)).astype(np.float32)
    a = g.uniform(0.0, 1.0, n).astype(np.float32)
    b = g.uniform(0.0, 1.0, n).astype(np.float32)
    return Workload("paper_uniform", x, a, y, b, eps=eps, rho=rho, sweeps=100, ell=0.5)


def subsample_rows(g: np.random.Generator, count: int, total: int) -> np.ndarray:
    """Sorted distinct row indices, for checking sampled outputs at full size."""
    return np.sort(g.choice(total, size=min(count, total), replace=False))
