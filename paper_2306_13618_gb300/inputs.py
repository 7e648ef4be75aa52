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
* ``pair_batch`` -- many independent problems of uneven sizes: per pair, n and
  m log-uniform in [1024, 65536], both clouds uniform in one ball of radius 0.2
  whose centre is uniform in [-1, 1]^3, weights uniform in [0.5, 1.5]
  normalised to masses uniform in [0.5, 2], eps in {0.01, 0.05} and rho in
  {0.1, 1, 10} drawn per pair.
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


@dataclass
class PairBatch:
    x: np.ndarray          # (sum n_p, d) float32, pairs concatenated
    a: np.ndarray
    x_off: np.ndarray      # (npairs + 1,) int64
    y: np.ndarray
    b: np.ndarray
    y_off: np.ndarray
    eps: np.ndarray        # (npairs,) float64
    rho: np.ndarray        # (npairs,) float64

    @property
    def npairs(self):
        return self.x_off.size - 1

    def pair(self, p):
        """(x, a, y, b, eps, rho) of pair p."""
        xs = slice(self.x_off[p], self.x_off[p + 1])
        ys = slice(self.y_off[p], self.y_off[p + 1])
        return self.x[xs], self.a[xs], self.y[ys], self.b[ys], self.eps[p], self.rho[p]


def _ball(g: np.random.Generator, count: int, centre: np.ndarray, radius: float) -> np.ndarray:
    d = centre.size
    v = g.standard_normal((count, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * g.uniform(0.0, 1.0, count) ** (1.0 / d)
    return (centre + v * r[:, None]).astype(np.float32)


def pair_batch(seed: int = 4000, npairs: int = 512, nmin: int = 1024, nmax: int = 65536,
               d: int = 3, eps_choices=(0.01, 0.05), rho_choices=(0.1, 1.0, 10.0)) -> PairBatch:
    g = rng(seed)
    xs, as_, ys, bs = [], [], [], []
    x_off, y_off = [0], [0]
    eps = np.empty(npairs)
    rho = np.empty(npairs)
    for p in range(npairs):
        n, m = (int(round(np.exp(g.uniform(np.log(nmin), np.log(nmax))))) for _ in range(2))
        centre = g.uniform(-1.0, 1.0, d)
        xs.append(_ball(g, n, centre, 0.2))
        ys.append(_ball(g, m, centre, 0.2))
        as_.append(_normalise(g.uniform(0.5, 1.5, n), g.uniform(0.5, 2.0)))
        bs.append(_normalise(g.uniform(0.5, 1.5, m), g.uniform(0.5, 2.0)))
        x_off.append(x_off[-1] + n)
        y_off.append(y_off[-1] + m)
        eps[p] = eps_choices[g.integers(0, len(eps_choices))]
        rho[p] = rho_choices[g.integers(0, len(rho_choices))]
    return PairBatch(np.concatenate(xs), np.concatenate(as_), np.asarray(x_off, np.int64),
                     np.concatenate(ys), np.concatenate(bs), np.asarray(y_off, np.int64),
                     eps, rho)


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
