"""GPU parity of the direct (exact O(nm)) form against the FP64 oracle, through
the C ABI.  Tolerances derived from FP32 arithmetic (see the derivation in the
design notes): every kernel-sum term is positive, so the relative error of an
output is bounded by the relative error of its terms -- ex2.approx (~2 ulp),
the FP32 squared distance (a few ulp of the exponent) and the FP32 partial sums
of 32 terms -- about 4e-7; we test at 2e-6 per output (5e-6 for d >= 8, whose
squared distance carries d roundings).  Sinkhorn duals after a fixed number of
sweeps are compared with the paper's residual (Table Tab:Accuracy_analysis2):
||beta - beta*||/||beta*|| + ||gamma - gamma*||/||gamma*|| <= 1e-6."""
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
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 64])
@pytest.mark.parametrize("n,m", [(3001, 1777), (257, 2049), (1, 5)])
def test_kernel_sum_parity(uotk, d, n, m):
    g = inputs.rng(100 + d)
    src = g.uniform(-0.3, 0.3, (n, d)).astype(np.float32)
    tgt = g.uniform(-0.3, 0.3, (m, d)).astype(np.float32)
    w = g.uniform(0.1, 2.0, n).astype(np.float32)
    eps = 0.05 * d
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), eps).cpu().numpy()
    ref = oracle.ksum(f64(src), f64(w), f64(tgt), eps)
    assert rel_err(got, ref) <= (2e-6 if d <= 3 else 5e-6)


def test_kernel_sum_large_sampled(uotk):
    """n = m = 2^20, d = 3 Gaussian mixture (the scale workload): 512 sampled
    outputs against the oracle over all 2^20 sources."""
    W = inputs.gmm3(seed=2000)
    out = uotk.kernel_sum(dev(W.y), dev(W.b), dev(W.x), W.eps).cpu().numpy()
    idx = inputs.subsample_rows(inputs.rng(5), 512, W.n)
    ref = oracle.ksum(f64(W.y), f64(W.b), f64(W.x[idx]), W.eps)
    assert rel_err(out[idx], ref) <= 2e-6


def test_kernel_sum_edge_cases(uotk):
    g = inputs.rng(7)
    tgt = g.uniform(-0.3, 0.3, (100, 3)).astype(np.float32)
    # no sources -> zeros
    out = uotk.kernel_sum(dev(np.zeros((0, 3), np.float32)), dev(np.zeros(0, np.float32)),
                          dev(tgt), 0.1).cpu().numpy()
    assert np.all(out == 0)
    # no targets -> empty
    out = uotk.kernel_sum(dev(tgt), dev(np.ones(100, np.float32)),
                          dev(np.zeros((0, 3), np.float32)), 0.1)
    assert out.numel() == 0
    # coincident points: every term is w exactly
    src = np.repeat(tgt[:1], 1000, axis=0)
    w = np.full(1000, 0.5, np.float32)
    out = uotk.kernel_sum(dev(src), dev(w), dev(src[:7]), 0.1).cpu().numpy()
    assert np.allclose(out, 500.0, rtol=1e-6)
    # zero weights and far outliers contribute exactly zero
    src2 = np.concatenate([tgt, tgt + 100.0]).astype(np.float32)
    w2 = np.concatenate([np.zeros(100), np.ones(100)]).astype(np.float32)
    out = uotk.kernel_sum(dev(src2), dev(w2), dev(tgt), 0.1).cpu().numpy()
    assert np.all(out == 0)


def test_kernel_sum_rejects_bad_weights(uotk):
    g = inputs.rng(8)
    p = dev(g.uniform(-0.3, 0.3, (64, 3)).astype(np.float32))
    w = np.ones(64, np.float32)
    w[5] = -1.0
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(p, dev(w), p, 0.1)
    assert e.value.status == 1
    w[5] = np.nan
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(p, dev(w), p, 0.1)
    assert e.value.status == 5
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(p, dev(np.ones(64, np.float32)), p, -1.0)
    assert e.value.status == 1
    q = dev(g.uniform(-0.3, 0.3, (64, 4)).astype(np.float32))
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(q, dev(np.ones(64, np.float32)), q, 0.1, method="nfft")
    assert e.value.status == 4


def residual(b, g, rb, rg):
    return (np.linalg.norm(b - rb) / np.linalg.norm(rb)
            + np.linalg.norm(g - rg) / np.linalg.norm(rg))


@pytest.mark.parametrize("ref", ["product", "counting"])
def test_sinkhorn_uniform_box(uotk, ref):
    """n = m = 2000, d = 2, eps = 0.05, rho = 1, 100 sweeps: duals and D(beta, gamma)."""
    W = inputs.uniform_box()
    r = 0 if ref == "product" else 1
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(
        dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho, max_sweeps=W.sweeps, ref=ref)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps, ref=r)
    assert sweeps == W.sweeps
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert res <= 1e-6, res
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg, ref=r)
    assert abs(value - v) <= 1e-6 * abs(v), (value, v)


def test_sinkhorn_ragged_unequal_penalties_warm_start(uotk):
    g = inputs.rng(9)
    n, m, d = 1537, 999, 3
    x = g.uniform(-0.3, 0.3, (n, d)).astype(np.float32)
    y = g.uniform(-0.2, 0.35, (m, d)).astype(np.float32)
    a = g.uniform(0.5, 1.5, n).astype(np.float32) / n
    b = g.uniform(0.5, 1.5, m).astype(np.float32) * 1.7 / m
    g0 = g.uniform(-0.05, 0.05, m)
    beta, gamma, _, value, _ = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), 0.04, 0.7, 2.5,
                                                 max_sweeps=37, gamma0=torch.from_numpy(g0))
    rb, rg = oracle.uot_sinkhorn(f64(x), f64(a), f64(y), f64(b), 0.04, 0.7, 2.5, sweeps=37,
                                 gamma0=g0)
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg) <= 1e-6
    v = oracle.dual_value(f64(x), f64(a), f64(y), f64(b), 0.04, 0.7, 2.5, rb, rg)
    assert abs(value - v) <= 1e-6 * abs(v)


def test_sinkhorn_constant_cost_closed_form(uotk):
    """All x_i equal, all y_j equal: converged duals equal the closed form of Eq. (561)."""
    n, m, lam, eta = 300, 200, 20.0, 1.0
    x = np.tile(np.float32([0.1, -0.05]), (n, 1))
    y = np.tile(np.float32([-0.1, 0.15]), (m, 1))
    a = np.full(n, 1.0 / n, np.float32)
    b = np.full(m, 1.3 / m, np.float32)
    D = float(np.sum((f64(x[0]) - f64(y[0])) ** 2))
    m1, m2 = f64(a).sum(), f64(b).sum()
    den = 2 * eta + 1 / lam
    c = np.exp(-D / den) * (m1 * m2) ** (-eta / den)
    beta, gamma, sweeps, _, conv = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), 1 / lam, eta,
                                                     max_sweeps=2000, tol=1e-12)
    assert conv and sweeps < 2000
    assert np.allclose(beta.cpu().numpy(), -eta * np.log(c * m2), atol=2e-7, rtol=0)
    assert np.allclose(gamma.cpu().numpy(), -eta * np.log(c * m1), atol=2e-7, rtol=0)


def test_sinkhorn_not_converged_status(uotk):
    W = inputs.uniform_box(n=300, m=200)
    _, _, sweeps, _, conv = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps,
                                              W.rho, max_sweeps=20, tol=1e-14)
    assert sweeps == 20 and not conv


def test_mmd2_uniform_box(uotk):
    W = inputs.uniform_box()
    v, parts = uotk.mmd2(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.ell)
    rv, rp = oracle.mmd2(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.ell, return_parts=True)
    assert np.allclose(parts, rp, rtol=1e-6, atol=0)
    # the FP32 sums' relative error is amplified by (A + 2B + C)/MMD^2
    kappa = (rp[0] + 2 * rp[1] + rp[2]) / rv
    assert abs(v - rv) <= 1e-6 * kappa * abs(rv), (v, rv, kappa)
    z, _ = uotk.mmd2(dev(W.x), dev(W.a), dev(W.x), dev(W.a), W.ell)
    assert abs(z) <= 1e-6 * rp[0]


def test_sinkhorn_divergence_uniform_box(uotk):
    W = inputs.uniform_box(n=800, m=700)
    sd, parts = uotk.sinkhorn_divergence(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho,
                                         max_sweeps=W.sweeps)
    rsd, rparts = oracle.sinkhorn_divergence(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.eps, W.rho,
                                             sweeps=W.sweeps, return_parts=True)
    assert np.allclose(parts, rparts, rtol=1e-6, atol=0)
    kappa = sum(abs(p) for p in rparts) / abs(rsd)
    assert abs(sd - rsd) <= 1e-6 * kappa * abs(rsd), (sd, rsd, kappa)


def test_graph_replay_matches_eager(uotk):
    """Sweeps replayed from the captured CUDA graph equal eager launches bit for
    bit (the direct form is deterministic); profiling forces eager launches."""
    W = inputs.uniform_box(n=1000, m=900)
    ctx = uotk.default_context()
    args = (dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho)
    ctx.set_profiling(True)
    b1, g1, s1, v1, _ = uotk.uot_sinkhorn(*args, max_sweeps=37)
    ctx.set_profiling(False)
    ctx.profile_reset()
    b2, g2, s2, v2, _ = uotk.uot_sinkhorn(*args, max_sweeps=37)
    assert s1 == s2 == 37 and v1 == v2
    assert torch.equal(b1, b2) and torch.equal(g1, g2)


def test_measure_unit_rates(uotk):
    """The roofline denominators measured on this GPU: exp2 and FP32 FMA per
    clock per SM within the range of any recent NVIDIA SM (16 or 32 exp2,
    128 FMA lanes)."""
    ex2, ffma = uotk.measure_unit_rates()
    assert 8.0 <= ex2 <= 40.0, ex2
    assert 64.0 <= ffma <= 140.0, ffma


def test_sinkhorn_log_domain_matches_oracle(uotk):
    """UOTK_LOG_DOMAIN on the uniform box (both domains representable): the
    same residual bar as the direct form."""
    W = inputs.uniform_box(n=900, m=700)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(
        dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho, max_sweeps=W.sweeps,
        log_domain=True)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps, logdomain=True)
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg) <= 1e-6
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= 1e-6 * abs(v)


def test_sinkhorn_log_domain_tiny_eps(uotk):
    """eps = 1e-4 on half-overlapping clouds: some targets see no source closer
    than exp(-368), and the weights e^{lambda gamma - M} span e^{-460}, so the
    FP32 form underflows (NONFINITE) while the log domain follows the FP64
    oracle.  Bound: each half-step's log t carries the FP32 rounding of its
    largest exponent A (in log2 units), delta = 2^-22 A ln2, amplified by at
    most q per half-step and accumulated over the sweeps (q lambda < 1)."""
    g = inputs.rng(77)
    n = m = 500
    x = g.uniform(0, 0.25, (n, 2)).astype(np.float32)
    y = g.uniform(0.125, 0.375, (m, 2)).astype(np.float32)
    a = np.full(n, 1.0 / n, np.float32)
    b = np.full(m, 1.3 / m, np.float32)
    eps, rho, S = 1e-4, 1.0, 20
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), eps, rho, max_sweeps=S)
    assert e.value.status == 5
    beta, gamma, _, value, _ = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), eps, rho,
                                                 max_sweeps=S, log_domain=True)
    X, Y, A, B = f64(x), f64(y), f64(a), f64(b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, eps, rho, sweeps=S, logdomain=True)
    lam, c = 1.0 / eps, 1.4426950408889634 / eps
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    spread = max(np.ptp(lam * rb), np.ptp(lam * rg)) * 1.4426950408889634
    big = max(np.max(np.min(c * d2, 1)), np.max(np.min(c * d2, 0))) + spread
    q = rho / (1 + rho * lam)
    delta = 2.0 ** -22 * big * np.log(2)
    bound = 4 * S * q * delta
    assert np.max(np.abs(beta.cpu().numpy() - rb)) <= bound
    assert np.max(np.abs(gamma.cpu().numpy() - rg)) <= bound
    v = oracle.dual_value(X, A, Y, B, eps, rho, rho, rb, rg)
    assert np.isfinite(value) and abs(value - v) <= 1e-4 * abs(v)


def test_log_domain_rejected_off_direct(uotk):
    W = inputs.uniform_box(n=100, m=100)
    for method in ("nfft",):
        with pytest.raises(uotk.UotkError) as e:
            uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho,
                              max_sweeps=3, log_domain=True, method=method)
        assert e.value.status == 4


def test_lambda_scaling_matches_oracle_schedule(uotk):
    """uotk_uot_sinkhorn_scaled against the oracle run of the same stages (the
    oracle replays the GPU's per-stage sweep counts, warm-started the same
    way): the direct form's residual bar on the last stage's duals."""
    W = inputs.uniform_box(n=600, m=500)
    sched = [1.0, 0.2, 0.05]
    # tol above the FP32 noise of the half-step sums (lambda * |change| ~ 1e-7)
    beta, gamma, sweeps, value, conv = uotk.uot_sinkhorn_scaled(
        dev(W.x), dev(W.a), dev(W.y), dev(W.b), sched, 2.0, max_sweeps=3000, tol=1e-5)
    assert conv and np.all(sweeps > 0)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    g = None
    for eps, s in zip(sched, sweeps):
        rb, g = oracle.uot_sinkhorn(X, A, Y, B, eps, 2.0, sweeps=int(s), gamma0=g)
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, g) <= 1e-6
    v = oracle.dual_value(X, A, Y, B, sched[-1], 2.0, 2.0, rb, g)
    assert abs(value - v) <= 1e-6 * abs(v)


def test_lambda_scaling_reaches_the_cold_fixed_point(uotk):
    """The setting of the paper's lambda-scaling experiment (probability
    measures, eta1 = eta2 = 25, lambda in {1, 20, 100}): the staged solve and a
    cold solve at lambda = 100, both stopped at tol, agree on the duals.  Each
    is within tol / (1 - (q lambda)^2) (in lambda * dual units) of the unique
    fixed point, q lambda = eta lambda / (1 + eta lambda) per half-step."""
    g = inputs.rng(61)
    x = g.uniform(0.0, 1.0, (800, 2)).astype(np.float32)
    y = (g.uniform(0.0, 1.0, (700, 2)) ** 2).astype(np.float32)
    a = np.full(800, 1.0 / 800, np.float32)
    b = np.full(700, 1.0 / 700, np.float32)
    args = (dev(x), dev(a), dev(y), dev(b))
    tol, lam, eta = 1e-6, 100.0, 25.0
    bs, gs, sweeps, vs, conv = uotk.uot_sinkhorn_scaled(*args, [1.0, 1 / 20, 1 / 100], eta,
                                                        max_sweeps=30000, tol=tol)
    bc, gc, cold, vc, conv_cold = uotk.uot_sinkhorn(*args, 1 / lam, eta, max_sweeps=30000,
                                                    tol=tol)
    assert conv and conv_cold
    rate = (eta * lam / (1 + eta * lam)) ** 2
    bound = 2 * tol / (1 - rate) / lam
    assert torch.max(torch.abs(bs - bc)).item() <= bound
    assert torch.max(torch.abs(gs - gc)).item() <= bound
    assert abs(vs - vc) <= 1e-4 * abs(vc)
