"""The summation autotuner (uotk_autotune_sum, method UOTK_AUTO) through the C
ABI: it measures the candidate forms on the GPU and keeps the fastest whose
error, max |s - s*| / sum|w| at sampled targets against their FP64 sums, meets
the target.  Checked against the FP64 oracle on other targets than the
autotuner's own sample, with the NFFT's error metric.  The sampled error of a
form is a lower bound of its maximum error over all targets; the bar below
allows it twice the target."""
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


def err_vs_oracle(out, W, idx):
    ref = oracle.ksum(f64(W.y), f64(W.b), f64(W.x[idx]), W.eps)
    return np.max(np.abs(f64(out)[idx] - ref)) / np.sum(np.abs(f64(W.b)))


def test_autotune_meets_target_and_is_cached(uotk):
    W = inputs.gmm3(seed=2030, n=200000, m=150001)
    src, w, tgt = dev(W.y), dev(W.b), dev(W.x)
    ctx = uotk.Context(0)
    opts, rep = uotk.autotune_sum(src, w, tgt, W.eps, target_err=1e-5, ctx=ctx)
    assert rep["forms"] >= 2 and rep["samples"] == 256
    assert opts["method"] == "direct" or rep["err"] <= 1e-5, (opts, rep)
    # a sum this large is far cheaper by the NFFT at this accuracy
    assert opts["method"] == "nfft" and rep["ms"] < rep["direct_ms"], (opts, rep)
    opts2, rep2 = uotk.autotune_sum(src, w, tgt, W.eps, target_err=1e-5, ctx=ctx)
    assert opts2 == opts and rep2 == rep        # the cached choice
    out = uotk.kernel_sum(src, w, tgt, W.eps, method="auto", ctx=ctx).cpu().numpy()
    idx = inputs.subsample_rows(inputs.rng(31), 300, W.m)
    assert err_vs_oracle(out, W, idx) <= 2e-5
    ctx.close()


def test_autotune_unreachable_target_gives_direct(uotk):
    W = inputs.gmm3(seed=2031, n=20000, m=15000)
    opts, rep = uotk.autotune_sum(dev(W.y), dev(W.b), dev(W.x), W.eps, target_err=1e-12)
    assert opts["method"] == "direct", (opts, rep)


def test_autotune_fixed_grid_and_cutoff(uotk):
    """Only the caller's grid and cut-off are tried when given: the mixture
    workload's 128^3 grid and m = 6."""
    W = inputs.gmm3(seed=2032, n=1 << 18, m=1 << 18)
    opts, rep = uotk.autotune_sum(dev(W.y), dev(W.b), dev(W.x), W.eps, target_err=1e-5,
                                  grid=128, cutoff=6)
    assert opts["method"] == "nfft" and opts["grid"] == 128 and opts["cutoff"] == 6, opts
    assert rep["err"] <= 1e-5 and rep["forms"] == 2, rep


def test_autotune_high_dimension(uotk):
    """d = 64: the direct FP32 form against the tensor-core forms; whichever is
    kept meets the target on other targets too."""
    W = inputs.gauss64(seed=3010, n=16384, m=16384)
    opts, rep = uotk.autotune_sum(dev(W.y), dev(W.b), dev(W.x), W.eps, target_err=1e-4)
    assert opts["method"] in ("direct", "direct_bf16x3", "direct_bf16"), opts
    assert rep["forms"] == 3
    out = uotk.kernel_sum(dev(W.y), dev(W.b), dev(W.x), W.eps, method="auto").cpu().numpy()
    idx = inputs.subsample_rows(inputs.rng(32), 128, W.m)
    ref = oracle.ksum(f64(W.y), f64(W.b), f64(W.x[idx]), W.eps)
    assert np.max(np.abs(f64(out)[idx] - ref)) / np.sum(f64(W.b)) <= 2e-4


def test_sinkhorn_auto_matches_oracle(uotk):
    """Alg. 1/2 with the autotuned form (the beta half-step's sum y -> x with the
    weights nu), against the FP64 Alg. 1 at the NFFT bar."""
    W = inputs.gmm3(seed=2033, n=4096, m=3500)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b),
                                                      W.eps, W.rho, max_sweeps=30,
                                                      method="auto", target_err=1e-5)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=30)
    res = (np.linalg.norm(beta.cpu().numpy() - rb) / np.linalg.norm(rb)
           + np.linalg.norm(gamma.cpu().numpy() - rg) / np.linalg.norm(rg))
    assert sweeps == 30 and res <= 1e-4, res
