"""GPU parity of the Sinkhorn solves with the cost |x - y| (r = 1; Gibbs kernel
e^{-|x-y|/eps}, the Laplace kernel of Table tab:0) against the FP64 oracle run
with r = 1, through the C ABI; and the Cor. cor:477 setting.

Error model.  A direct Laplace kernel sum carries 2e-6 + 4 * 2^-22 * max r/eps of
relative error per output (tests/test_gpu_kernels.py); at eps = 0.2 on [0, 1]^2
(r/eps <= 7) that is <= 9e-6, and the dual update maps a relative error e of t
to an absolute error q e of beta (q = rho/(1 + rho/eps) < eps).  The residual
of Table Tab:Accuracy_analysis2 is held to 2e-5 (direct) and 1e-4 (NFFT, the
NFFT bar), the dual value to the same, and each divergence to that times its
condition sum |UOT parts| / |sd|."""
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


def residual(b, g, rb, rg):
    return (np.linalg.norm(b - rb) / np.linalg.norm(rb)
            + np.linalg.norm(g - rg) / np.linalg.norm(rg))


def clouds(seed, n, m, d):
    g = inputs.rng(seed)
    return (g.uniform(0, 1, (n, d)).astype(np.float32), g.uniform(0.2, 1, n).astype(np.float32),
            g.uniform(0, 1, (m, d)).astype(np.float32), g.uniform(0.2, 1, m).astype(np.float32))


@pytest.mark.parametrize("method,tol", [("direct", 2e-5), ("nfft", 1e-4)])
@pytest.mark.parametrize("d", [2, 3])
def test_uot_sinkhorn_r1(uotk, method, tol, d):
    x, a, y, b = clouds(900 + d, 1500, 1200, d)
    eps, rho, S = 0.2, 1.0, 40
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(x), dev(a), dev(y), dev(b), eps, rho,
                                                      max_sweeps=S, method=method,
                                                      kernel="laplace")
    X, A, Y, B = f64(x), f64(a), f64(y), f64(b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, eps, rho, sweeps=S, r=1)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert sweeps == S and res <= tol, (method, d, res)
    v = oracle.dual_value(X, A, Y, B, eps, rho, rho, rb, rg, r=1)
    assert abs(value - v) <= tol * abs(v), (value, v)
    # the cost is used: the r = 2 duals are far from these
    r2b, _ = oracle.uot_sinkhorn(X, A, Y, B, eps, rho, sweeps=S)
    assert np.max(np.abs(r2b - rb)) > 100 * tol * np.max(np.abs(rb))


@pytest.mark.parametrize("method,tol", [("direct", 2e-5), ("nfft", 1e-4)])
def test_sinkhorn_divergence_r1(uotk, method, tol):
    x, a, y, b = clouds(911, 1200, 1000, 2)
    eps, rho, S = 0.2, 1.0, 40
    sd, parts = uotk.sinkhorn_divergence(dev(x), dev(a), dev(y), dev(b), eps, rho, max_sweeps=S,
                                         method=method, kernel="laplace")
    rsd, rparts = oracle.sinkhorn_divergence(f64(x), f64(a), f64(y), f64(b), eps, rho,
                                             sweeps=S, return_parts=True, r=1)
    assert np.allclose(parts, rparts, rtol=tol, atol=0), (parts, rparts)
    kappa = sum(abs(p) for p in rparts) / abs(rsd)
    assert abs(sd - rsd) <= tol * kappa * abs(rsd), (sd, rsd, kappa)


def test_cor477_setting(uotk):
    """Probability measures on [0, 1] (the paper's Cor. cor:477 experiment), eta
    large against 1/lambda: the GPU divergence equals the oracle's within its
    condition, and both lie within lambda/2 (relative) of MMD^2_{k_e}/2."""
    g = inputs.rng(921)
    n, m = 400, 300
    x = g.uniform(0, 1, (n, 1)).astype(np.float32)
    y = g.uniform(0, 1, (m, 1)).astype(np.float32)
    P, Q = np.full(n, 1 / n, np.float32), np.full(m, 1 / m, np.float32)
    lam, eta = 1e-2, 1e3
    S = int(40 * (1 + eta * lam))
    sd, parts = uotk.sinkhorn_divergence(dev(x), dev(P), dev(y), dev(Q), 1 / lam, eta,
                                         max_sweeps=S, kernel="laplace")
    rsd, rparts = oracle.sinkhorn_divergence(f64(x), f64(P), f64(y), f64(Q), 1 / lam, eta,
                                             sweeps=S, return_parts=True, r=1)
    kappa = sum(abs(p) for p in rparts) / abs(rsd)
    assert abs(sd - rsd) <= 2e-5 * kappa * abs(rsd), (sd, rsd, kappa)
    half_e = 0.5 * oracle.mmd2_kernel("energy", 1.0, f64(x), f64(P), f64(y), f64(Q))
    assert abs(rsd - half_e) <= 0.5 * lam * half_e
    assert abs(sd - half_e) <= 0.5 * lam * half_e + 2e-5 * kappa * abs(rsd), (sd, half_e)


@pytest.mark.parametrize("method,tol", [("direct", 2e-6), ("nfft", 5e-6)])
def test_mean_cost_and_cstar_r1(uotk, method, tol):
    x, a, y, b = clouds(931, 3000, 2500, 3)
    cost, m1, m2 = uotk.mean_cost(dev(x), dev(a), dev(y), dev(b), r=1, method=method)
    ref = oracle.mean_cost(f64(x), f64(a), f64(y), f64(b), 1)
    assert abs(cost - ref) <= tol * ref, (cost, ref)
    c, bound, c1 = uotk.cstar(dev(x), dev(a), dev(y), dev(b), 0.2, 1.0, 0.5, r=1, method=method)
    rc, rbound, _ = oracle.cstar(f64(x), f64(a), f64(y), f64(b), 0.2, 1.0, 0.5, r=1)
    # c* depends on the cost through exp(-C / (m1 m2 (eta1 + eta2 + eps)))
    assert abs(c - rc) <= 2 * tol * ref / (m1 * m2 * 1.7) * rc + 1e-14, (c, rc)


def test_r1_init_and_unsupported(uotk):
    x, a, y, b = clouds(941, 700, 500, 2)
    args = (dev(x), dev(a), dev(y), dev(b), 0.2, 1.0)
    beta, gamma, _, _, _ = uotk.uot_sinkhorn(*args, max_sweeps=20, kernel="laplace",
                                             cstar_init=True)
    X, A, Y, B = f64(x), f64(a), f64(y), f64(b)
    c = oracle.cstar(X, A, Y, B, 0.2, 1.0, 1.0, r=1)[0]
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, 0.2, 1.0, sweeps=20, r=1, gamma0=np.full(500, c))
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg) <= 2e-5
    for kw in ({"kernel": "imq"}, {"kernel": "energy"}, {"kernel": "laplace", "log_domain": True},
               {"kernel": "laplace", "method": "direct_bf16x3"}):
        with pytest.raises(uotk.UotkError) as e:
            uotk.uot_sinkhorn(*args, max_sweeps=5, **kw)
        assert e.value.status == 4, kw
