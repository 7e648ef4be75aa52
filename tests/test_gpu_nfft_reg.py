"""GPU parity of the NFFT form of the non-smooth kernels of Table tab:0
(Laplace, inverse multiquadric, energy; Sec. 4.2) against the FP64 oracle's
exact kernel sums, through the C ABI.

Error model: the regularised fast summation with grid 256, N = 128, p = 4 has a
method error about 5e-7 of max|s| on uniform clouds (the FP64 oracle of the same
construction, tests/test_oracle_nfft_reg.py and its explorations); the FP32
spread / FFT / gather add about 1e-6 of sum|w| max|K|, as for the Gaussian.
Tested at 5e-6 of max|s| per output; MMD^2 parts at 5e-6 relative, the value
at that times its condition (|A| + 2|B| + |C|)/|MMD^2|."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = [("laplace", 0.5), ("imq", 1.0), ("energy", 1.0)]


@pytest.fixture(scope="module")
def uotk():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f64(a):
    return np.asarray(a, dtype=np.float64)


def uniform(seed, n, d):
    """The paper's empirical measures (Sec. 5.1.1): points and weights U[0, 1]."""
    g = inputs.rng(seed)
    return g.uniform(0, 1, (n, d)).astype(np.float32), g.uniform(0, 1, n).astype(np.float32)


def rel_max(got, ref):
    return np.max(np.abs(f64(got) - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("kind,p", KINDS)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_kernel_sum_nfft_vs_exact(uotk, kind, p, d):
    src, w = uniform(700 + d, 3001, d)
    tgt, _ = uniform(720 + d, 1999, d)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), p, method="nfft", kernel=kind)
    ref = oracle.ksum_kernel(kind, p, f64(src), f64(w), f64(tgt))
    err = rel_max(got.cpu().numpy(), ref)
    assert err <= 5e-6, (kind, d, err)


@pytest.mark.parametrize("kind,p", KINDS)
def test_kernel_sum_nfft_clustered(uotk, kind, p):
    """Five tight clusters: most pairs of a cluster fall in the near field."""
    W = inputs.gmm3(seed=2301, n=4000, m=3000)
    got = uotk.kernel_sum(dev(W.y), dev(W.b), dev(W.x), p, method="nfft", kernel=kind)
    ref = oracle.ksum_kernel(kind, p, f64(W.y), f64(W.b), f64(W.x))
    err = rel_max(got.cpu().numpy(), ref)
    assert err <= 5e-6, (kind, err)


@pytest.mark.parametrize("kind,p", KINDS)
def test_mmd2_nfft(uotk, kind, p):
    """Table Tab:Accuracy_analysis3's setting: d = 2, c = 1, ell = 1/2, uniform
    points and weights (unbalanced)."""
    x, a = uniform(731, 5000, 2)
    y, b = uniform(732, 4000, 2)
    v, parts = uotk.mmd2(dev(x), dev(a), dev(y), dev(b), p, method="nfft", kernel=kind)
    rv, rp = oracle.mmd2_kernel(kind, p, f64(x), f64(a), f64(y), f64(b), return_parts=True)
    assert np.allclose(parts, rp, rtol=5e-6, atol=0), (parts, rp)
    kappa = (abs(rp[0]) + 2 * abs(rp[1]) + abs(rp[2])) / abs(rv)
    assert abs(v - rv) <= 5e-6 * kappa * abs(rv), (v, rv, kappa)


def test_kernel_sum_nfft_large_sampled(uotk):
    """n = m = 2^20, d = 3, Laplace ell = 1/2: sampled targets against the oracle."""
    src, w = uniform(741, 1 << 20, 3)
    tgt, _ = uniform(742, 1 << 20, 3)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.5, method="nfft", kernel="laplace")
    idx = inputs.subsample_rows(inputs.rng(743), 256, tgt.shape[0])
    ref = oracle.ksum_kernel("laplace", 0.5, f64(src), f64(w), f64(tgt[idx]))
    err = rel_max(got.cpu().numpy()[idx], ref)
    assert err <= 5e-6, err


@pytest.mark.parametrize("kind,p", KINDS)
def test_degenerate_clouds(uotk, kind, p):
    # every point identical: the box has no extent, every pair is in the near field
    q = np.tile(np.array([[0.3, -0.2, 0.1]], np.float32), (10, 1))
    w = np.linspace(0.5, 1.5, 10).astype(np.float32)
    got = uotk.kernel_sum(dev(q), dev(w), dev(q[:3]), p, method="nfft", kernel=kind)
    ref = oracle.ksum_kernel(kind, p, f64(q), f64(w), f64(q[:3]))
    assert np.allclose(got.cpu().numpy(), ref, rtol=1e-5, atol=1e-6 * np.sum(w))
    # one source, targets from the near field to the far end of the box
    s = np.array([[0.0, 0.0, 0.0]], np.float32)
    t = np.array([[r, 0.0, 0.0] for r in (0.0, 0.01, 0.05, 0.3, 1.0, 2.0)], np.float32)
    got = uotk.kernel_sum(dev(s), dev(np.ones(1, np.float32)), dev(t), p, method="nfft",
                          kernel=kind)
    ref = oracle.ksum_kernel(kind, p, f64(s), np.ones(1), f64(t))
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got.cpu().numpy() - ref)) <= 5e-6 * scale, (got, ref)


def test_options_and_validation(uotk):
    src, w = uniform(751, 1500, 3)
    ref = oracle.ksum_kernel("laplace", 0.5, f64(src), f64(w), f64(src[:64]))
    for kw, tol in (({"grid": 128}, 2e-5), ({"reg_degree": 6}, 5e-6),
                    ({"grid": 128, "reg_degree": 8}, 2e-5)):
        got = uotk.kernel_sum(dev(src), dev(w), dev(src[:64]), 0.5, method="nfft",
                              kernel="laplace", **kw)
        err = rel_max(got.cpu().numpy(), ref)
        assert err <= tol, (kw, err)
    for kw in ({"reg_degree": 13}, {"reg_degree": 1}, {"grid": 64, "bandwidth": 64},
               {"grid": 32, "reg_degree": 4}, {"period": 0.5}):
        with pytest.raises(uotk.UotkError) as e:
            uotk.kernel_sum(dev(src), dev(w), dev(src[:64]), 0.5, method="nfft",
                            kernel="laplace", **kw)
        assert e.value.status == 1, kw
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(dev(np.zeros((8, 4), np.float32)), dev(np.ones(8, np.float32)),
                        dev(np.zeros((8, 4), np.float32)), 0.5, method="nfft", kernel="imq")
    assert e.value.status == 4
    # a plan too coarse for the kernel is refused by its self-check, not run
    # (grid 64, p = 2, ell = 0.1 on [0, 1]^3: error bound per unit weight about
    # 3e-3 > 1e-3 on the FP64 oracle of the same construction)
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(dev(src), dev(w), dev(src[:64]), 0.1, method="nfft", kernel="laplace",
                        grid=64, reg_degree=2)
    assert e.value.status == 4
    # ... and runs when the caller accepts that bound
    got = uotk.kernel_sum(dev(src), dev(w), dev(src[:64]), 0.1, method="nfft", kernel="laplace",
                          grid=64, reg_degree=2, target_err=1e-2)
    ref = oracle.ksum_kernel("laplace", 0.1, f64(src), f64(w), f64(src[:64]))
    assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-2 * np.sum(w)
