"""The NFFT work split on point sets chosen to stress it, against the FP64
oracle at the NFFT bar (max|s - s*| / sum|w| <= 1e-5, relative L2 <= 1e-4).

The spread and the gather cut the cell-sorted points into chunks of equal cost,
one per CTA the GPU holds at once, and cut each chunk again where a tile of
8^3 grid cells ends.  The cases here cover
* sizes around the split's boundaries: a single point, odd counts (the spread
  pairs consecutive points, so an odd count leaves a half-empty pair), and
  counts below, at and above one chunk per resident CTA;
* one dense cluster inside a single tile (many chunks of one tile, folded from
  many pieces) next to points scattered over the grid (many tiles, each with a
  few points, inside one chunk);
* empty sources (the sums are zero) and empty targets;
* a Sinkhorn solve on the clustered set, so the spread that forms its own
  weights and the gather that runs the dual update see the same split."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uotk():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f64(a):
    return np.asarray(a, dtype=np.float64)


def errors(got, ref, w):
    got, ref = f64(got), f64(ref)
    return (np.max(np.abs(got - ref)) / np.sum(np.abs(f64(w))),
            np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def clustered(seed, n_dense, n_sparse, d=3):
    """A tight cluster (inside one tile at the default grid) and points spread
    uniformly over the same box, shuffled together."""
    g = inputs.rng(seed)
    dense = g.normal(0.0, 0.004, (n_dense, d))
    sparse = g.uniform(-0.3, 0.3, (n_sparse, d))
    pts = np.concatenate([dense, sparse])[g.permutation(n_dense + n_sparse)]
    return pts.astype(np.float32)


@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 607, 608, 609, 4097])
def test_sizes_around_the_split(uotk, n):
    g = inputs.rng(7100 + n)
    src = g.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    tgt = g.uniform(-0.3, 0.3, (n + 5, 3)).astype(np.float32)
    w = g.uniform(0.5, 1.5, n).astype(np.float32)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft").cpu().numpy()
    ref = oracle.ksum(f64(src), f64(w), f64(tgt), 0.02)
    e_inf, e_l2 = errors(got, ref, w)
    assert e_inf <= 1e-5 and e_l2 <= 1e-4, (n, e_inf, e_l2)


@pytest.mark.parametrize("n_dense,n_sparse", [(200000, 3000), (3000, 60000)])
def test_dense_cluster_and_scattered_points(uotk, n_dense, n_sparse):
    """Sources and targets each a cluster plus scattered points; targets are
    sampled for the oracle."""
    src = clustered(7200 + n_dense, n_dense, n_sparse)
    tgt = clustered(7300 + n_dense, n_dense, n_sparse)
    w = inputs.rng(7400).lognormal(0.0, 0.5, src.shape[0]).astype(np.float32)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft").cpu().numpy()
    idx = inputs.subsample_rows(inputs.rng(7500), 400, tgt.shape[0])
    ref = oracle.ksum(f64(src), f64(w), f64(tgt[idx]), 0.02)
    e_inf, e_l2 = errors(got[idx], ref, w)
    assert e_inf <= 1e-5 and e_l2 <= 1e-4, (e_inf, e_l2)
    # the split is deterministic: a second call gives the same bits
    again = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft").cpu().numpy()
    assert np.array_equal(got, again)


def test_empty_sources_and_targets(uotk):
    pts = inputs.rng(7600).uniform(-0.3, 0.3, (100, 3)).astype(np.float32)
    w = np.ones(100, np.float32)
    zero = uotk.kernel_sum(dev(pts[:0]), dev(w[:0]), dev(pts), 0.02, method="nfft")
    assert zero.shape == (100,) and torch.count_nonzero(zero).item() == 0
    none = uotk.kernel_sum(dev(pts), dev(w), dev(pts[:0]), 0.02, method="nfft")
    assert none.shape == (0,)


def test_sinkhorn_on_clustered_set(uotk):
    """Alg. 2 on clustered measures (cluster plus scattered points on both
    sides) against the FP64 Alg. 1, 60 sweeps: the NFFT residual bar."""
    x = clustered(7700, 5000, 1500)
    y = clustered(7800, 4000, 2000)
    g = inputs.rng(7900)
    a = (g.uniform(0.5, 1.5, x.shape[0]) / x.shape[0]).astype(np.float32)
    b = (g.uniform(0.5, 1.5, y.shape[0]) / y.shape[0]).astype(np.float32)
    eps, rho = 0.02, 0.5
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), eps, rho,
                                                      max_sweeps=60, method="nfft")
    rb, rg = oracle.uot_sinkhorn(f64(x), f64(a), f64(y), f64(b), eps, rho, sweeps=60)
    res = (np.linalg.norm(beta.cpu().numpy() - rb) / np.linalg.norm(rb)
           + np.linalg.norm(gamma.cpu().numpy() - rg) / np.linalg.norm(rg))
    assert sweeps == 60 and res <= 1e-4, res
