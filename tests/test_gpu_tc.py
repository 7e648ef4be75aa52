"""GPU parity of the tensor-core direct forms (UOTK_DIRECT_BF16, UOTK_DIRECT_BF16X3)
against the FP64 oracle, through the C ABI.

Error model.  The library forms ||x - y||^2 = |x|^2 + |y|^2 - 2 x.y from points
centred on the middle of the joint bounding box, with R = max |p - o| the
largest centred norm.  An error e in x.y changes a term exp(-||x-y||^2/eps)
by the factor exp(2 e / eps), so every (positive) term, and therefore every
sum of positive terms, has relative error about 2 e / eps, plus the FP32
error of the FP32 form:
  * BF16: each factor is rounded to 8 significant bits, e <= 2^-8 R^2
    (two roundings of 2^-9), bound 2^-7 R^2 / eps;
  * BF16x3: v = hi + lo leaves 2^-18 |v|, and the dropped lo.lo term is
    2^-18 |x||y|, so e <= 3 * 2^-18 R^2 and the bound is 6 * 2^-18 R^2 / eps,
    plus the FP32 accumulation of 3d products (2^-22 R^2) and the FP32
    exponent arithmetic (a few 2^-24 c R^2).
Each test computes R from the data and checks max relative error <= 2 x bound
+ 2e-6 (the FP32 sum bar)."""
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


def rel_err(got, ref):
    got, ref = f64(got), f64(ref)
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))


def radius(*clouds):
    lo = np.min([np.min(f64(c), 0) for c in clouds], 0)
    hi = np.max([np.max(f64(c), 0) for c in clouds], 0)
    o = (f64(lo.astype(np.float32)) + f64(hi.astype(np.float32))) / 2
    return max(np.max(np.linalg.norm(f64(c) - o, axis=1)) for c in clouds)


def bound(method, R, eps):
    per = 2.0 ** -7 if method == "direct_bf16" else 6 * 2.0 ** -18 + 2.0 ** -21
    return 2 * per * R * R / eps + 2e-6


@pytest.mark.parametrize("method", ["direct_bf16x3", "direct_bf16"])
@pytest.mark.parametrize("d,n,m,eps", [(64, 1000, 777, 0.5), (3, 300, 129, 0.5),
                                       (17, 128, 128, 0.5), (100, 513, 250, 0.5),
                                       (128, 129, 1, 0.5), (1, 1, 300, 0.5),
                                       (64, 700, 300, 0.05)])
def test_kernel_sum_tc_parity(uotk, method, d, n, m, eps):
    """eps = 0.5 takes the epilogue that scales each row sum once (c R^2 <= 64);
    eps = 0.05 takes the per-term one."""
    g = inputs.rng(400 + d)
    src = (g.standard_normal((n, d)) / np.sqrt(d)).astype(np.float32)
    tgt = (g.standard_normal((m, d)) / np.sqrt(d) + 0.05).astype(np.float32)
    w = g.uniform(0.1, 2.0, n).astype(np.float32)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), eps, method=method).cpu().numpy()
    ref = oracle.ksum(f64(src), f64(w), f64(tgt), eps)
    err = rel_err(got, ref)
    assert err <= bound(method, radius(src, tgt), eps), (err, bound(method, radius(src, tgt), eps))


@pytest.mark.parametrize("method", ["direct_bf16x3", "direct_bf16"])
def test_kernel_sum_tc_narrow_kernel(uotk, method):
    """eps = 0.01 on dense uniform clouds in [-1/2, 1/2]^3 (c R^2 ~ 108: the
    per-term epilogue).  Every target has sources within a few hundredths, so
    the sums stay inside the FP32 range (a sum below ~1e-38 would flush to 0 in
    any FP32 form)."""
    g = inputs.rng(460)
    src = g.uniform(-0.5, 0.5, (4000, 3)).astype(np.float32)
    tgt = g.uniform(-0.5, 0.5, (700, 3)).astype(np.float32)
    w = g.uniform(0.1, 2.0, 4000).astype(np.float32)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.01, method=method).cpu().numpy()
    ref = oracle.ksum(f64(src), f64(w), f64(tgt), 0.01)
    assert np.min(ref) > 1e-30
    err = rel_err(got, ref)
    assert err <= bound(method, radius(src, tgt), 0.01), (err, bound(method, radius(src, tgt), 0.01))


def test_kernel_sum_tc_edges(uotk):
    g = inputs.rng(450)
    tgt = (g.standard_normal((200, 64)) / 8).astype(np.float32)
    for method in ("direct_bf16x3", "direct_bf16"):
        # zero weights contribute exactly zero; far outliers underflow to zero
        src = np.concatenate([tgt, tgt + 50.0]).astype(np.float32)
        w = np.concatenate([np.zeros(200), np.ones(200)]).astype(np.float32)
        out = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 1.0, method=method).cpu().numpy()
        assert np.all(out == 0), method
        # no sources -> zeros
        out = uotk.kernel_sum(dev(np.zeros((0, 64), np.float32)), dev(np.zeros(0, np.float32)),
                              dev(tgt), 1.0, method=method).cpu().numpy()
        assert np.all(out == 0)
    # negative weight rejected, d > 128 unsupported
    w = np.ones(200, np.float32)
    w[3] = -1
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(dev(tgt), dev(w), dev(tgt), 1.0, method="direct_bf16x3")
    assert e.value.status == 1
    big = np.zeros((10, 129), np.float32)
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(dev(big), dev(np.ones(10, np.float32)), dev(big), 1.0,
                        method="direct_bf16")
    assert e.value.status == 4


def test_kernel_sum_tc_large_sampled(uotk):
    """n = m = 262144, d = 64 (the high-dimensional workload): 256 sampled
    targets against the oracle over all sources, both precisions."""
    W = inputs.gauss64()
    idx = inputs.subsample_rows(inputs.rng(7), 256, W.m)
    ref = oracle.ksum(f64(W.x), f64(W.a), f64(W.y[idx]), W.eps)
    R = radius(W.x, W.y)
    for method in ("direct_bf16x3", "direct_bf16"):
        out = uotk.kernel_sum(dev(W.x), dev(W.a), dev(W.y), W.eps, method=method).cpu().numpy()
        err = rel_err(out[idx], ref)
        assert err <= bound(method, R, W.eps), (method, err, bound(method, R, W.eps))


def residual(b, g, rb, rg):
    return (np.linalg.norm(b - rb) / np.linalg.norm(rb)
            + np.linalg.norm(g - rg) / np.linalg.norm(rg))


def test_sinkhorn_tc_vs_oracle(uotk):
    """Alg. 1 with the BF16x3 cross term on a 1024 + 1024 subsample of the
    high-dimensional workload, 100 sweeps, against the FP64 oracle."""
    W = inputs.gauss64(seed=3001, n=1024, m=1024)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b),
                                                      W.eps, W.rho, max_sweeps=W.sweeps,
                                                      method="direct_bf16x3")
    # per-sum relative error delta moves the duals by about q*delta per
    # half-step, accumulated over the contraction: residual ~ delta (1 + eta lambda)
    delta = bound("direct_bf16x3", radius(W.x, W.y), W.eps)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert res <= delta * (1 + W.rho / W.eps), (res, delta)
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= delta * abs(v) * (1 + W.rho / W.eps)


@pytest.mark.parametrize("log_domain", [False, True])
def test_sinkhorn_tc_subsample_4096(uotk, log_domain):
    """The high-dimensional workload's check as stated: a full 100-sweep solve
    (eps = 1, rho = 2, BF16x3 cross term, FP64 dual updates) on a 4096-point
    subsample of each cloud, plain and log-domain, against the FP64 oracle at
    the tensor-core bar."""
    W = inputs.gauss64()
    idx = inputs.subsample_rows(inputs.rng(31), 4096, W.n)
    x, y = W.x[idx], W.y[idx]
    a = (W.a[idx] * (1.0 / W.a[idx].sum())).astype(np.float32)
    b = (W.b[idx] * (1.2 / W.b[idx].sum())).astype(np.float32)
    X, Y, A, B = f64(x), f64(y), f64(a), f64(b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps,
                                 logdomain=log_domain)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), W.eps,
                                                      W.rho, max_sweeps=W.sweeps,
                                                      method="direct_bf16x3",
                                                      log_domain=log_domain)
    delta = bound("direct_bf16x3", radius(x, y), W.eps)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert sweeps == W.sweeps and res <= delta * (1 + W.rho / W.eps), (res, delta)
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= delta * abs(v) * (1 + W.rho / W.eps)


def test_mmd2_tc(uotk):
    W = inputs.gauss64(seed=3002, n=1500, m=1300)
    rv, rp = oracle.mmd2(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.ell, return_parts=True)
    delta = bound("direct_bf16x3", radius(W.x, W.y), W.ell ** 2)
    v, parts = uotk.mmd2(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.ell, method="direct_bf16x3")
    assert np.allclose(parts, rp, rtol=delta, atol=0)
    assert abs(v - rv) <= delta * (rp[0] + 2 * rp[1] + rp[2])


@pytest.mark.parametrize("method", ["direct_bf16x3", "direct_bf16"])
def test_sinkhorn_tc_log_domain_matches_oracle(uotk, method):
    """UOTK_LOG_DOMAIN with the tensor-core cross term (per-row log-sum-exp in
    the epilogue) on the high-dimensional workload's subsample: the same bar as
    the plain tensor-core solve, and the same duals as it."""
    W = inputs.gauss64(seed=3001, n=1024, m=1024)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps, logdomain=True)
    args = (dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho)
    beta, gamma, _, value, _ = uotk.uot_sinkhorn(*args, max_sweeps=W.sweeps, method=method,
                                                 log_domain=True)
    delta = bound(method, radius(W.x, W.y), W.eps)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert res <= delta * (1 + W.rho / W.eps), (res, delta)
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= delta * abs(v) * (1 + W.rho / W.eps)
    b2, g2, _, _, _ = uotk.uot_sinkhorn(*args, max_sweeps=W.sweeps, method=method)
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), b2.cpu().numpy(),
                    g2.cpu().numpy()) <= delta * (1 + W.rho / W.eps)


@pytest.mark.parametrize("method", ["direct_bf16x3", "direct_bf16"])
def test_sinkhorn_tc_log_domain_tiny_eps(uotk, method):
    """eps = 5e-4 on clouds 0.3 apart along x: the farthest targets see no
    source within exp2(-260), so the plain form underflows (NONFINITE) while the
    log domain follows the FP64 oracle.  Bound: per half-step the log of a sum
    carries the tensor-core term error delta_tc (the bound of this file, in
    relative terms of every summand) and the FP32 rounding of the exponents
    (2^-22 A ln2, A the largest exponent in log2 units), amplified by at most q
    per half-step over S sweeps."""
    g = inputs.rng(78)
    n = m = 400
    x = np.column_stack([g.uniform(0, 0.3, n), g.uniform(0, 0.1, n)]).astype(np.float32)
    y = np.column_stack([g.uniform(0.3, 0.6, m), g.uniform(0, 0.1, m)]).astype(np.float32)
    a = np.full(n, 1.0 / n, np.float32)
    b = np.full(m, 1.2 / m, np.float32)
    eps, rho, S = 5e-4, 1.0, 20
    args = (dev(x), dev(a), dev(y), dev(b), eps, rho)
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(*args, max_sweeps=S, method=method)
    assert e.value.status == 5
    beta, gamma, _, value, _ = uotk.uot_sinkhorn(*args, max_sweeps=S, method=method,
                                                 log_domain=True)
    X, Y, A, B = f64(x), f64(y), f64(a), f64(b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, eps, rho, sweeps=S, logdomain=True)
    lam, c = 1.0 / eps, 1.4426950408889634 / eps
    R = radius(x, y)
    spread = max(np.ptp(lam * rb), np.ptp(lam * rg)) * 1.4426950408889634
    big = c * R * R + spread
    q = rho / (1 + rho * lam)
    delta = bound(method, R, eps) + 2.0 ** -22 * big * np.log(2)
    tol = 4 * S * q * delta
    assert np.max(np.abs(beta.cpu().numpy() - rb)) <= tol, tol
    assert np.max(np.abs(gamma.cpu().numpy() - rg)) <= tol, tol
    v = oracle.dual_value(X, A, Y, B, eps, rho, rho, rb, rg)
    assert np.isfinite(value) and abs(value - v) <= max(delta, 1e-4) * abs(v)
