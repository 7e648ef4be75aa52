"""Pins of the oracle's mean cost and c* (Prop. prop:536, Eq. 561), CPU only.

* The mean cost <mu (x) nu|d^2> against the moment identity
  m2 sum mu|x|^2 + m1 sum nu|y|^2 - 2 (sum mu x).(sum nu y), and <mu (x) nu|d>
  against -(energy-kernel cross term) of Eq. (1205) (d = -k_e, Sec. 4.4).
* Constant cost: the converged Sinkhorn plan is exactly c* mu (x) nu, with
  unequal eta and masses so that swapping the exponents of Eq. (561) fails.
* General cost: c* minimises the Eq. (W4) objective over plans c mu (x) nu; the
  scalar form of that objective equals the entry-wise definition; and it bounds
  the converged UOT value from above (Remark on upper bounds)."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs


def _clouds(seed, n=23, m=17, d=3, shift=0.0):
    g = inputs.rng(seed)
    x = g.uniform(-0.5, 0.5, (n, d)) + shift
    y = g.uniform(-0.3, 0.7, (m, d)) + shift
    mu = g.uniform(0.2, 1.0, n)
    nu = g.uniform(0.2, 1.0, m) * 1.7
    return x, mu, y, nu


@pytest.mark.parametrize("shift", [0.0, 40.0])
def test_mean_cost_moment_identity(shift):
    x, mu, y, nu = _clouds(5, shift=shift)
    m1, m2 = mu.sum(), nu.sum()
    want = (m2 * np.sum(mu * np.sum(x * x, 1)) + m1 * np.sum(nu * np.sum(y * y, 1))
            - 2.0 * np.dot(mu @ x, nu @ y))
    got = oracle.mean_cost(x, mu, y, nu, 2)
    scale = m2 * np.sum(mu * np.sum(x * x, 1))   # cancellation of the identity at shift 40
    assert abs(got - want) <= 1e-14 * scale, (got, want)


def test_mean_cost_r1_is_minus_energy_cross_term():
    x, mu, y, nu = _clouds(6)
    _, parts = oracle.mmd2_kernel("energy", 1.0, x, mu, y, nu, return_parts=True)
    got = oracle.mean_cost(x, mu, y, nu, 1)
    assert abs(got + parts[1]) <= 1e-13 * got
    # and r = 1 is the plain sum of distances: one pair by hand
    assert oracle.mean_cost(x[:1], [2.0], y[:1], [3.0], 1) == pytest.approx(
        6.0 * np.linalg.norm(x[0] - y[0]), rel=1e-15)


@pytest.mark.parametrize("eta1,eta2,lam", [(0.5, 2.0, 5.0), (3.0, 0.7, 50.0)])
def test_cstar_is_the_constant_cost_optimum(eta1, eta2, lam):
    g = inputs.rng(7)
    n, m = 6, 9
    x = np.tile([0.1, -0.2, 0.05], (n, 1))
    y = np.tile([-0.15, 0.1, 0.2], (m, 1))
    mu = g.uniform(0.5, 1.5, n)
    nu = g.uniform(0.5, 1.5, m) * 0.3
    c, bound, cost = oracle.cstar(x, mu, y, nu, 1.0 / lam, eta1, eta2)
    beta, gamma = oracle.uot_sinkhorn(x, mu, y, nu, 1.0 / lam, eta1, eta2, sweeps=4000)
    pi = oracle.plan(x, mu, y, nu, 1.0 / lam, beta, gamma)
    assert np.allclose(pi, c * np.outer(mu, nu), rtol=1e-11, atol=0)
    dv = oracle.dual_value(x, mu, y, nu, 1.0 / lam, eta1, eta2, beta, gamma)
    assert abs(dv - bound) <= 1e-12 * abs(bound)


def _w4_dense(x, mu, y, nu, eps, eta1, eta2, pi):
    """Eq. (W4) by its definition, entry by entry, for a dense plan pi."""
    d2 = np.sum((x[:, None, :] - y[None, :, :]) ** 2, axis=2)
    mn = np.outer(mu, nu)
    kl = lambda p, q: np.sum(p * np.log(p / q) - p + q)
    return (np.sum(pi * d2) + eps * kl(pi, mn) + eta1 * kl(pi.sum(1), mu)
            + eta2 * kl(pi.sum(0), nu))


def test_independent_objective_matches_definition():
    x, mu, y, nu = _clouds(8)
    eps, eta1, eta2 = 0.05, 0.8, 1.9
    cost = oracle.mean_cost(x, mu, y, nu, 2)
    for c in (0.03, 0.4, 1.7):
        got = oracle.independent_objective(c, cost, mu.sum(), nu.sum(), eps, eta1, eta2)
        want = _w4_dense(x, mu, y, nu, eps, eta1, eta2, c * np.outer(mu, nu))
        assert abs(got - want) <= 1e-13 * abs(want), (c, got, want)


@pytest.mark.parametrize("eps,eta1,eta2", [(0.05, 0.8, 1.9), (0.2, 3.0, 0.4)])
def test_cstar_minimises_over_scaled_independent_plans(eps, eta1, eta2):
    x, mu, y, nu = _clouds(9)
    c, bound, cost = oracle.cstar(x, mu, y, nu, eps, eta1, eta2)
    m1, m2 = mu.sum(), nu.sum()
    for f in (0.5, 0.9, 0.99, 1.01, 1.1, 2.0):
        assert oracle.independent_objective(f * c, cost, m1, m2, eps, eta1, eta2) > bound
    # and with the exponents of Eq. (561) swapped the value is worse (m1 != m2, eta1 != eta2)
    den = eta1 + eta2 + eps
    c_sw = np.exp(-cost / (m1 * m2 * den)) * m1 ** (-eta1 / den) * m2 ** (-eta2 / den)
    assert oracle.independent_objective(c_sw, cost, m1, m2, eps, eta1, eta2) > bound


@pytest.mark.parametrize("eps,eta", [(0.05, 1.0), (0.5, 0.3)])
def test_cstar_objective_bounds_uot_from_above(eps, eta):
    x, mu, y, nu = _clouds(10)
    _, bound, _ = oracle.cstar(x, mu, y, nu, eps, eta, eta)
    beta, gamma = oracle.uot_sinkhorn(x, mu, y, nu, eps, eta, eta, sweeps=3000)
    dv = oracle.dual_value(x, mu, y, nu, eps, eta, eta, beta, gamma)
    pv = oracle.primal_value(x, mu, y, nu, eps, eta, eta, beta, gamma)
    assert abs(pv - dv) <= 1e-9 * abs(dv)        # converged: strong duality
    assert dv < bound
