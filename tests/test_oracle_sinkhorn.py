"""Pins of the FP64 oracle's Sinkhorn / dual / divergence functions against what
the paper and the mathematics fix (closed forms, an independent Newton solver,
limits and invariants).  CPU only."""
import numpy as np
import pytest

import oracle


def _closed_form_constant_cost(D, m1, m2, lam, eta1, eta2):
    """Constant cost D between every pair: the optimum is pi* = c* mu (x) nu with
    c* of Eq. (561) (Prop. prop:536), the duals follow from the first-order
    conditions of Eq. (dual_euot), and the value is the objective of Eq. (1117)
    at c* (signs of the appendix corrected: -c mu nu + mu(X), not +c mu nu - mu(X))."""
    den = eta1 + eta2 + 1.0 / lam
    c = np.exp(-D / den) * m1 ** (-eta2 / den) * m2 ** (-eta1 / den)
    beta = -eta1 * np.log(c * m2)
    gamma = -eta2 * np.log(c * m1)
    val = (m1 * m2 * (c * D + (c * np.log(c) - c + 1.0) / lam)
           + eta1 * m1 * (c * m2 * np.log(c * m2) - c * m2 + 1.0)
           + eta2 * m2 * (c * m1 * np.log(c * m1) - c * m1 + 1.0))
    return c, beta, gamma, val


@pytest.mark.parametrize("eta1,eta2,lam", [(1.0, 1.0, 20.0), (0.5, 2.0, 5.0), (3.0, 0.7, 50.0)])
def test_constant_cost_closed_form(oracle_lib, eta1, eta2, lam):
    g = np.random.default_rng(1)
    n, m, d = 7, 5, 3
    x0 = np.array([0.1, -0.2, 0.05])
    y0 = np.array([-0.15, 0.1, 0.2])
    x = np.tile(x0, (n, 1))
    y = np.tile(y0, (m, 1))
    mu = g.uniform(0.5, 1.5, n)
    nu = g.uniform(0.5, 1.5, m) * 0.4
    D = float(np.sum((x0 - y0) ** 2))
    c, bstar, gstar, val = _closed_form_constant_cost(D, mu.sum(), nu.sum(), lam, eta1, eta2)
    beta, gamma = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta1, eta2, sweeps=3000)
    assert np.allclose(beta, bstar, rtol=0, atol=1e-12)
    assert np.allclose(gamma, gstar, rtol=0, atol=1e-12)
    dv = oracle.dual_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, beta, gamma)
    pv = oracle.primal_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, beta, gamma)
    assert abs(dv - val) <= 1e-12 * abs(val)
    assert abs(pv - val) <= 1e-12 * abs(val)
    pi = oracle.plan(x, mu, y, nu, 1.0 / lam, beta, gamma)
    assert np.allclose(pi, c * np.outer(mu, nu), rtol=1e-11, atol=0)


def test_constant_cost_divergence(oracle_lib):
    """Eq. (586) on one-point supports: every UOT value has the closed form above."""
    g = np.random.default_rng(2)
    n, m, lam, eta = 4, 6, 10.0, 0.8
    x = np.tile([0.3, 0.1], (n, 1))
    y = np.tile([-0.1, 0.2], (m, 1))
    mu = g.uniform(0.5, 1.5, n)
    nu = g.uniform(0.5, 1.5, m)
    D = 0.4 ** 2 + 0.1 ** 2
    m1, m2 = mu.sum(), nu.sum()
    v_xy = _closed_form_constant_cost(D, m1, m2, lam, eta, eta)[3]
    v_xx = _closed_form_constant_cost(0.0, m1, m1, lam, eta, eta)[3]
    v_yy = _closed_form_constant_cost(0.0, m2, m2, lam, eta, eta)[3]
    want = v_xy - 0.5 * v_xx - 0.5 * v_yy + (m1 - m2) ** 2 / (2 * lam)
    got, parts = oracle.sinkhorn_divergence(x, mu, y, nu, 1.0 / lam, eta, sweeps=2000,
                                            return_parts=True)
    assert np.allclose(parts, [v_xy, v_xx, v_yy], rtol=1e-12, atol=0)
    assert abs(got - want) <= 1e-11 * max(1.0, abs(want))


def _dual_np(beta, gamma, x, mu, y, nu, lam, eta1, eta2, ref):
    """Dual objective written independently for the Newton pin (Eq. dual_euot)."""
    C = np.sum((x[:, None, :] - y[None, :, :]) ** 2, axis=2)
    E = np.exp(lam * (beta[:, None] + gamma[None, :]) - lam * C)
    ref_mass = mu.sum() * nu.sum()
    if ref == 0:
        E = E * np.outer(mu, nu)
    else:
        ref_mass = len(mu) * len(nu)
    return (-eta1 * np.sum(mu * np.exp(-beta / eta1)) - eta2 * np.sum(nu * np.exp(-gamma / eta2))
            + eta1 * mu.sum() + eta2 * nu.sum() - (E.sum() - ref_mass) / lam), E


def _newton_dual(x, mu, y, nu, lam, eta1, eta2, ref, tol=1e-13):
    """Damped Newton maximisation of the strictly concave dual: an algorithm
    independent of Sinkhorn's alternating maximisation that reaches the same
    unique maximiser (Theorem thm:dual_EUOT)."""
    n, m = len(mu), len(nu)
    z = np.zeros(n + m)
    for _ in range(200):
        b, gm = z[:n], z[n:]
        f, P = _dual_np(b, gm, x, mu, y, nu, lam, eta1, eta2, ref)
        ea, eb = mu * np.exp(-b / eta1), nu * np.exp(-gm / eta2)
        grad = np.concatenate([ea - P.sum(1), eb - P.sum(0)])
        if np.max(np.abs(grad)) < tol:
            break
        H = np.zeros((n + m, n + m))
        H[:n, :n] = np.diag(-ea / eta1 - lam * P.sum(1))
        H[n:, n:] = np.diag(-eb / eta2 - lam * P.sum(0))
        H[:n, n:] = -lam * P
        H[n:, :n] = -lam * P.T
        step = -np.linalg.solve(H, grad)
        t = 1.0
        while _dual_np(b + t * step[:n], gm + t * step[n:], x, mu, y, nu, lam, eta1, eta2,
                       ref)[0] < f - 1e-15 * abs(f) and t > 1e-8:
            t *= 0.5
        z = z + t * step
    return z[:n], z[n:], np.max(np.abs(grad))


@pytest.mark.parametrize("ref", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_newton_tiny(oracle_lib, ref, seed):
    g = np.random.default_rng(10 + seed)
    n, m, d = 1 + seed * 3, 8 - seed, 2
    x = g.uniform(-0.3, 0.3, (n, d))
    y = g.uniform(-0.3, 0.3, (m, d))
    mu = g.uniform(0.5, 1.5, n)
    nu = g.uniform(0.2, 1.0, m)
    lam, eta1, eta2 = 8.0, 1.0, 0.6
    bn, gn, gres = _newton_dual(x, mu, y, nu, lam, eta1, eta2, ref)
    assert gres < 1e-12
    bs, gs = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta1, eta2, sweeps=4000, ref=ref)
    assert np.allclose(bs, bn, rtol=0, atol=1e-11)
    assert np.allclose(gs, gn, rtol=0, atol=1e-11)
    dv = oracle.dual_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, bs, gs, ref=ref)
    want = _dual_np(bn, gn, x, mu, y, nu, lam, eta1, eta2, ref)[0]
    if ref == 1:  # the oracle drops the constant reference mass n*m/lambda
        want -= n * m / lam
    assert abs(dv - want) <= 1e-11 * max(1.0, abs(want))


def test_two_point_fixed_point_and_rate(oracle_lib):
    """n = m = 1: the iteration is affine; fixed point beta (1 - q^2 lambda^2) =
    -q log(k nu) + q^2 lambda log(k mu), error contracting by p^2 = (q lambda)^2 per sweep."""
    lam, eta = 20.0, 1.0
    q = eta / (1 + eta * lam)
    x = np.array([[0.1, 0.0]]); y = np.array([[0.0, 0.2]])
    mu, nu = np.array([1.0]), np.array([1.3])
    k = np.exp(-lam * 0.05)
    bstar = (-q * np.log(k * nu[0]) + q * q * lam * np.log(k * mu[0])) / (1 - (q * lam) ** 2)
    errs = []
    for s in (1, 2, 3, 4):
        b, _ = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta, sweeps=s)
        errs.append(b[0] - bstar)
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.allclose(ratios, (q * lam) ** 2, rtol=1e-9)
    b, _ = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta, sweeps=2000)
    assert abs(b[0] - bstar) < 1e-13


def test_logdomain_matches_plain(oracle_lib):
    g = np.random.default_rng(3)
    x = g.uniform(-0.25, 0.25, (40, 2)); y = g.uniform(-0.25, 0.25, (30, 2))
    mu = g.uniform(0.5, 1.5, 40) / 40; nu = g.uniform(0.5, 1.5, 30) * 1.3 / 30
    for ref in (0, 1):
        b1, g1 = oracle.uot_sinkhorn(x, mu, y, nu, 0.05, 1.0, sweeps=50, ref=ref)
        b2, g2 = oracle.uot_sinkhorn(x, mu, y, nu, 0.05, 1.0, sweeps=50, ref=ref, logdomain=True)
        assert np.allclose(b1, b2, atol=1e-13, rtol=0) and np.allclose(g1, g2, atol=1e-13, rtol=0)


def test_weak_duality_gap_closes(oracle_lib):
    """primal(pi(beta,gamma)) >= D(beta,gamma) at every iterate; the gap tends to 0."""
    g = np.random.default_rng(4)
    x = g.uniform(-0.25, 0.25, (30, 2)); y = g.uniform(-0.25, 0.25, (25, 2))
    mu = g.uniform(0.5, 1.5, 30) / 30; nu = g.uniform(0.5, 1.5, 25) * 1.3 / 25
    gaps = []
    for s in (1, 5, 20, 80, 400):
        b, gm = oracle.uot_sinkhorn(x, mu, y, nu, 0.05, 1.0, sweeps=s)
        pv = oracle.primal_value(x, mu, y, nu, 0.05, 1.0, 1.0, b, gm)
        dv = oracle.dual_value(x, mu, y, nu, 0.05, 1.0, 1.0, b, gm)
        gaps.append(pv - dv)
    assert all(gp >= -1e-14 for gp in gaps)
    assert gaps[-1] < 1e-13 and gaps[0] > 1e-6


def test_fixed_point_and_marginal_identity(oracle_lib):
    """At convergence: beta_i + q log t_i(gamma) = 0 and sum_j pi_ij = mu_i e^{-beta_i/eta}."""
    g = np.random.default_rng(5)
    lam, eta = 20.0, 1.0
    x = g.uniform(-0.25, 0.25, (35, 2)); y = g.uniform(-0.25, 0.25, (28, 2))
    mu = g.uniform(0.5, 1.5, 35) / 35; nu = g.uniform(0.5, 1.5, 28) * 1.3 / 28
    b, gm = oracle.uot_sinkhorn(x, mu, y, nu, 1 / lam, eta, sweeps=600)
    t = oracle.ksum(y, nu * np.exp(lam * gm), x, 1 / lam)
    q = eta / (1 + eta * lam)
    assert np.max(np.abs(b + q * np.log(t))) < 1e-13
    pi = oracle.plan(x, mu, y, nu, 1 / lam, b, gm)
    assert np.allclose(pi.sum(1), mu * np.exp(-b / eta), rtol=1e-12)
    assert np.allclose(pi.sum(0), nu * np.exp(-gm / eta), rtol=1e-12)


def test_balanced_limit(oracle_lib):
    """Rem. rem:813: equal masses, eta -> infinity gives the balanced plan; the
    L1 distance shrinks roughly like 1/eta."""
    g = np.random.default_rng(6)
    lam = 10.0
    x = g.uniform(-0.3, 0.3, (20, 2)); y = g.uniform(-0.3, 0.3, (16, 2))
    P = g.uniform(0.5, 1.5, 20); P /= P.sum()
    Q = g.uniform(0.5, 1.5, 16); Q /= Q.sum()
    f, gb = oracle.balanced_sinkhorn(x, P, y, Q, 1 / lam, 3000)
    pib = oracle.plan(x, P, y, Q, 1 / lam, f, gb)
    assert np.allclose(pib.sum(1), P, atol=1e-12) and np.allclose(pib.sum(0), Q, atol=1e-12)
    dists = []
    for eta in (1e2, 1e3, 1e4):
        b, gm = oracle.uot_sinkhorn(x, P, y, Q, 1 / lam, eta, sweeps=int(60 * eta))
        pi = oracle.plan(x, P, y, Q, 1 / lam, b, gm)
        dists.append(np.abs(pi - pib).sum())
    assert dists[0] > dists[1] > dists[2]
    assert 5 < dists[0] / dists[1] < 20 and 5 < dists[1] / dists[2] < 20


def test_eta_to_zero_limit(oracle_lib):
    """eta -> 0 removes the marginal penalties of Eq. (W4); what is left,
    <pi, d^2> + (1/lambda) D(pi || mu (x) nu), is minimised by pi = (mu (x) nu) * k,
    and q = eta/(1+eta lambda) -> 0 drives both duals to 0 at rate O(eta).
    (Rem. rem:813's pi -> 0 is the unregularised limit of Eq. (W3).)"""
    g = np.random.default_rng(7)
    lam = 20.0
    x = g.uniform(-0.3, 0.3, (10, 2)); y = g.uniform(-0.3, 0.3, (12, 2))
    mu = g.uniform(0.5, 1.5, 10); nu = g.uniform(0.5, 1.5, 12)
    C = np.sum((x[:, None, :] - y[None, :, :]) ** 2, axis=2)
    lim = np.outer(mu, nu) * np.exp(-lam * C)
    dist = []
    for eta in (1e-2, 1e-3, 1e-4):
        b, gm = oracle.uot_sinkhorn(x, mu, y, nu, 1 / lam, eta, sweeps=200)
        dist.append(np.abs(oracle.plan(x, mu, y, nu, 1 / lam, b, gm) - lim).sum())
    assert dist[0] > dist[1] > dist[2]
    assert 5 < dist[0] / dist[1] < 20 and 5 < dist[1] / dist[2] < 20


def test_lambda_scaling_reaches_the_fixed_point_of_the_last_lambda():
    """lambda-scaling (Sec. 5.1.2): stages at increasing lambda, each started
    from the previous gamma, converge to the same duals as a cold start at the
    last lambda (the fixed point of Alg. 1 is unique)."""
    g = np.random.default_rng(12)
    x = g.uniform(-0.25, 0.25, (9, 2))
    y = g.uniform(-0.25, 0.25, (7, 2))
    a = np.full(9, 1.0 / 9)
    b = np.full(7, 1.0 / 7)
    eta = 25.0
    gam = None
    for eps in (1.0, 0.05, 0.01):
        be, gam = oracle.uot_sinkhorn(x, a, y, b, eps, eta, sweeps=60000, gamma0=gam)
    rb, rg = oracle.uot_sinkhorn(x, a, y, b, 0.01, eta, sweeps=60000)
    assert np.max(np.abs(be - rb)) <= 1e-12 and np.max(np.abs(gam - rg)) <= 1e-12


@pytest.mark.parametrize("eta1,eta2,lam", [(1.0, 1.0, 20.0), (0.5, 2.0, 5.0)])
def test_constant_cost_closed_form_r1(oracle_lib, eta1, eta2, lam):
    """The cost |x - y| (r = 1): with every pair at distance D the optimum is again
    c* mu (x) nu of Eq. (561), now with D the distance, not its square."""
    g = np.random.default_rng(11)
    n, m = 5, 6
    x = np.tile([0.1, -0.2, 0.05], (n, 1))
    y = np.tile([-0.15, 0.1, 0.2], (m, 1))
    mu = g.uniform(0.5, 1.5, n)
    nu = g.uniform(0.5, 1.5, m) * 0.6
    D = float(np.linalg.norm(np.array([0.25, -0.3, -0.15])))
    c, bstar, gstar, val = _closed_form_constant_cost(D, mu.sum(), nu.sum(), lam, eta1, eta2)
    beta, gamma = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta1, eta2, sweeps=3000, r=1)
    assert np.allclose(beta, bstar, rtol=0, atol=1e-12)
    assert np.allclose(gamma, gstar, rtol=0, atol=1e-12)
    dv = oracle.dual_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, beta, gamma, r=1)
    pv = oracle.primal_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, beta, gamma, r=1)
    assert abs(dv - val) <= 1e-12 * abs(val) and abs(pv - val) <= 1e-12 * abs(val)
    pi = oracle.plan(x, mu, y, nu, 1.0 / lam, beta, gamma, r=1)
    assert np.allclose(pi, c * np.outer(mu, nu), rtol=1e-11, atol=0)


def test_strong_duality_r1(oracle_lib):
    g = np.random.default_rng(12)
    x, y = g.uniform(0, 1, (30, 2)), g.uniform(0, 1, (25, 2))
    mu, nu = g.uniform(0.2, 1.0, 30), g.uniform(0.2, 1.0, 25)
    beta, gamma = oracle.uot_sinkhorn(x, mu, y, nu, 0.1, 0.7, 1.3, sweeps=2000, r=1)
    dv = oracle.dual_value(x, mu, y, nu, 0.1, 0.7, 1.3, beta, gamma, r=1)
    pv = oracle.primal_value(x, mu, y, nu, 0.1, 0.7, 1.3, beta, gamma, r=1)
    assert abs(pv - dv) <= 1e-10 * abs(dv)
    # and the r = 1 solve differs from the r = 2 one (the cost is used)
    b2, _ = oracle.uot_sinkhorn(x, mu, y, nu, 0.1, 0.7, 1.3, sweeps=2000)
    assert np.max(np.abs(b2 - beta)) > 1e-3


@pytest.mark.parametrize("lam", [1e-2, 1e-3])
def test_cor477_divergence_tends_to_the_energy_distance(oracle_lib, lam):
    """Cor. cor:477 (with Lemma lem:inter_ot_mmd): for probability measures the
    debiased UOT with cost |x - y| tends, as eta -> infinity and then lambda -> 0,
    to the energy distance; in the squared-RKHS convention of Eq. (1205) the
    limit is MMD^2_{k_e} / 2 = E|X-Y| - E|X-X'|/2 - E|Y-Y'|/2 (the paper's setting:
    uniform samples on [0, 1]).  The gap shrinks like lambda."""
    g = np.random.default_rng(3)
    x, y = g.uniform(0, 1, (120, 1)), g.uniform(0, 1, (100, 1))
    P, Q = np.full(120, 1 / 120), np.full(100, 1 / 100)
    half_e = 0.5 * oracle.mmd2_kernel("energy", 1.0, x, P, y, Q)
    eta = 1e5
    sweeps = int(min(20000, 40 * (1 + eta * lam)))
    sd = oracle.sinkhorn_divergence(x, P, y, Q, 1.0 / lam, eta, sweeps=sweeps, r=1)
    assert abs(sd - half_e) <= 0.5 * lam * half_e, (sd, half_e)
