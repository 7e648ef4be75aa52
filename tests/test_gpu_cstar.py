"""GPU parity of the mean cost, c* (Prop. prop:536, Eq. 561) and the c*
initialisation of Sinkhorn's algorithm against the FP64 oracle, through the C ABI.

Tolerances: r = 2 is FP64 moments of the same FP32 inputs the oracle reads, so
the two differ by rounding order only (1e-12 relative).  r = 1 is one energy-kernel
sum in the direct FP32 form (2e-6 per output, as the other-kernel tests) and an
FP64 dot product with non-negative weights: 2e-6 relative.  A solve started from
gamma^0 = c* is held to the bar of the solve started from 0: the dual residual
1e-6 (direct) or 1e-4 (NFFT) against the oracle run from the same start."""
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


def clouds(seed, n, m, d, shift=0.0):
    g = inputs.rng(seed)
    x = (g.uniform(-0.5, 0.5, (n, d)) + shift).astype(np.float32)
    y = (g.uniform(-0.3, 0.7, (m, d)) + shift).astype(np.float32)
    a = g.uniform(0.1, 1.0, n).astype(np.float32)
    b = g.uniform(0.1, 1.0, m).astype(np.float32)
    return x, a, y, b


@pytest.mark.parametrize("d,n,m,shift", [(1, 3001, 2500, 0.0), (3, 4099, 1000, 25.0),
                                         (64, 777, 1500, 0.0), (128, 1000, 333, 3.0),
                                         (3, 1, 1, 0.0)])
def test_mean_cost_r2(uotk, d, n, m, shift):
    x, a, y, b = clouds(800 + d, n, m, d, shift)
    cost, m1, m2 = uotk.mean_cost(dev(x), dev(a), dev(y), dev(b), r=2)
    ref = oracle.mean_cost(f64(x), f64(a), f64(y), f64(b), 2)
    assert abs(cost - ref) <= 1e-12 * ref, (cost, ref)
    assert abs(m1 - f64(a).sum()) <= 1e-12 * m1 and abs(m2 - f64(b).sum()) <= 1e-12 * m2


@pytest.mark.parametrize("d,n,m", [(1, 1500, 999), (3, 3001, 1777), (7, 513, 600)])
def test_mean_cost_r1_energy(uotk, d, n, m):
    x, a, y, b = clouds(810 + d, n, m, d)
    cost, _, _ = uotk.mean_cost(dev(x), dev(a), dev(y), dev(b), r=1)
    ref = oracle.mean_cost(f64(x), f64(a), f64(y), f64(b), 1)
    assert abs(cost - ref) <= 2e-6 * ref, (cost, ref)


@pytest.mark.parametrize("eps,rho1,rho2", [(0.02, 1.0, 1.0), (0.1, 0.5, 3.0)])
def test_cstar(uotk, eps, rho1, rho2):
    W = inputs.gmm3(seed=2101, n=5000, m=4000)
    c, bound, cost = uotk.cstar(dev(W.x), dev(W.a), dev(W.y), dev(W.b), eps, rho1, rho2)
    rc, rbound, rcost = oracle.cstar(f64(W.x), f64(W.a), f64(W.y), f64(W.b), eps, rho1, rho2)
    assert abs(cost - rcost) <= 1e-12 * rcost
    assert abs(c - rc) <= 1e-12 * rc, (c, rc)
    assert abs(bound - rbound) <= 1e-11 * abs(rbound), (bound, rbound)


@pytest.mark.parametrize("method,tol", [("direct", 1e-6), ("nfft", 1e-4)])
def test_cstar_init_matches_oracle(uotk, method, tol):
    W = inputs.gmm3(seed=2102, n=3000, m=2500)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b),
                                                      W.eps, W.rho, max_sweeps=40,
                                                      cstar_init=True, method=method)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    c = oracle.cstar(X, A, Y, B, W.eps, W.rho, W.rho)[0]
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=40,
                                 gamma0=np.full(W.m, c))
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert sweeps == 40 and res <= tol, res
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= tol * abs(v), (value, v)


def _workload(name):
    if name == "uniform_box":
        W = inputs.uniform_box(n=900, m=700, d=3)
        return W.x, W.a, W.y, W.b, W.eps, W.rho
    if name == "gmm3":
        W = inputs.gmm3(seed=2103, n=4096, m=4096)
        return W.x, W.a, W.y, W.b, W.eps, W.rho
    # the probability measures of the lambda-scaling experiment, lambda = 100, eta = 25
    g = inputs.rng(61)
    x = g.uniform(0.0, 1.0, (800, 2)).astype(np.float32)
    y = (g.uniform(0.0, 1.0, (700, 2)) ** 2).astype(np.float32)
    return (x, np.full(800, 1.0 / 800, np.float32), y, np.full(700, 1.0 / 700, np.float32),
            0.01, 25.0)


@pytest.mark.parametrize("name", ["uniform_box", "gmm3", "probability"])
def test_cstar_init_reaches_the_same_fixed_point(uotk, name):
    """Started from 0, from c* (the Remark read literally) or from the gamma of
    the constant-cost optimum at the mean cost, gamma_j = -eta log(c* mu(X)),
    and stopped at tol, each solve lands within tol / (1 - (q lambda)^2) (in
    lambda * dual units) of the unique maximiser, so any two agree to twice
    that.  Prints the three sweep counts."""
    x, a, y, b, eps, rho = _workload(name)
    args = (dev(x), dev(a), dev(y), dev(b), eps, rho)
    tol = 1e-6
    c = uotk.cstar(*args)[0]
    m1 = float(np.sum(a, dtype=np.float64))
    g_dual = torch.full((y.shape[0],), -rho * np.log(c * m1), dtype=torch.float64)
    runs = {"0": uotk.uot_sinkhorn(*args, max_sweeps=30000, tol=tol),
            "c*": uotk.uot_sinkhorn(*args, max_sweeps=30000, tol=tol, cstar_init=True),
            "dual of c*": uotk.uot_sinkhorn(*args, max_sweeps=30000, tol=tol, gamma0=g_dual)}
    lam = 1.0 / eps
    rate = (rho * lam / (1 + rho * lam)) ** 2
    bound = 2 * tol / (1 - rate) / lam
    b0, g0, _, v0, _ = runs["0"]
    for key, (b1, g1, s1, v1, conv) in runs.items():
        assert conv, key
        assert torch.max(torch.abs(b1 - b0)).item() <= bound, key
        assert torch.max(torch.abs(g1 - g0)).item() <= bound, key
        assert abs(v1 - v0) <= 1e-5 * abs(v0), key
    print(f"{name}: sweeps to tol {tol}: "
          + ", ".join(f"gamma0 = {k}: {r[2]}" for k, r in runs.items()))


def test_validation(uotk):
    x, a, y, b = clouds(820, 100, 80, 3)
    args = (dev(x), dev(a), dev(y), dev(b))
    with pytest.raises(uotk.UotkError) as e:
        uotk.mean_cost(*args, r=3)
    assert e.value.status == 1
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(*args, 0.1, 1.0, max_sweeps=5, cstar_init=True,
                          gamma0=torch.zeros(80, dtype=torch.float64))
    assert e.value.status == 1
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(*args, 0.1, 1.0, max_sweeps=5, cstar_init=True, ref="counting")
    assert e.value.status == 1
    bn = b.copy()
    bn[7] = -1.0
    with pytest.raises(uotk.UotkError) as e:
        uotk.mean_cost(dev(x), dev(a), dev(y), dev(bn), r=2)
    assert e.value.status == 1
    xn = x.copy()
    xn[3, 1] = np.nan
    with pytest.raises(uotk.UotkError) as e:
        uotk.cstar(dev(xn), dev(a), dev(y), dev(b), 0.1, 1.0)
    assert e.value.status == 5
    z = np.zeros_like(a)
    with pytest.raises(uotk.UotkError) as e:
        uotk.cstar(dev(x), dev(z), dev(y), dev(b), 0.1, 1.0)
    assert e.value.status == 1
