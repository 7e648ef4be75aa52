"""Pins of the oracle's gradient functions (CPU only).

The gradients are pinned by central finite differences of the oracle's own
VALUES (MMD^2 of Eq. 1205, D of Eq. dual_euot, the Sinkhorn divergence of
Eq. 586), which are pinned in the other oracle tests; a dropped term, a wrong
sign or a swapped role in a gradient shows up as an O(1) mismatch.  Plus
invariants the mathematics fixes: translation invariance (the gradients in
the points sum to zero), Euler's relation for the 2-homogeneous MMD^2, and
stationarity of the divergence at nu = mu (its minimum)."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs

H = 1e-6


def clouds(seed, n=7, m=5, d=2, mass=1.3):
    g = inputs.rng(seed)
    x = g.uniform(-0.3, 0.3, (n, d))
    y = g.uniform(-0.2, 0.4, (m, d))
    a = g.uniform(0.5, 1.5, n) / n
    b = g.uniform(0.5, 1.5, m) * mass / m
    return x, a, y, b


def fd_grad(f, args, name):
    """Central differences of f(**args) in every entry of args[name]."""
    arr = args[name]
    out = np.zeros_like(arr)
    for idx in np.ndindex(arr.shape):
        p, q = arr.copy(), arr.copy()
        p[idx] += H
        q[idx] -= H
        out[idx] = (f(**{**args, name: p}) - f(**{**args, name: q})) / (2 * H)
    return out


def close(got, fd, rtol):
    return np.max(np.abs(got - fd)) <= rtol * np.max(np.abs(fd))


@pytest.mark.parametrize("d", [1, 3])
def test_mmd2_grad_matches_finite_differences(d):
    x, a, y, b = clouds(11 + d, d=d)
    ell = 0.3
    ga, gx, gb, gy = oracle.mmd2_grad(x, a, y, b, ell)

    def f(x, a, y, b):
        return oracle.mmd2(x, a, y, b, ell)

    args = dict(x=x, a=a, y=y, b=b)
    for name, g in (("a", ga), ("x", gx), ("b", gb), ("y", gy)):
        assert close(g, fd_grad(f, args, name), 1e-7), name


def test_mmd2_grad_invariants():
    x, a, y, b = clouds(21, n=9, m=6, d=3)
    ell = 0.25
    ga, gx, gb, gy = oracle.mmd2_grad(x, a, y, b, ell)
    # translation invariance: sum of all point gradients is 0
    tot = gx.sum(0) + gy.sum(0)
    assert np.max(np.abs(tot)) <= 1e-13 * np.max(np.abs(gx))
    # Euler: MMD^2 is homogeneous of degree 2 in (a, b)
    v = oracle.mmd2(x, a, y, b, ell)
    assert abs(a @ ga + b @ gb - 2 * v) <= 1e-13 * (a @ np.abs(ga) + b @ np.abs(gb))
    # identical measures: all gradients vanish
    z = oracle.mmd2_grad(x, a, x, a, ell)
    for g in z:
        assert np.max(np.abs(g)) <= 1e-14


def test_mmd2_grad_rows_equal_full():
    x, a, y, b = clouds(23, n=9, m=6, d=3)
    ga, gx, gb, gy = oracle.mmd2_grad(x, a, y, b, 0.25)
    rows = [5, 0, 8]
    w, p = oracle.mmd2_grad_rows(x, a, y, b, 0.25, 0, rows)
    assert np.array_equal(w, ga[rows]) and np.array_equal(p, gx[rows])
    w, p = oracle.mmd2_grad_rows(x, a, y, b, 0.25, 1, [3])
    assert np.array_equal(w, gb[[3]]) and np.array_equal(p, gy[[3]])


def test_dual_grad_matches_finite_differences_at_any_duals():
    """Partial derivatives of D at fixed (unconverged) duals."""
    x, a, y, b = clouds(31, d=2)
    eps, e1, e2 = 0.1, 0.7, 1.9
    be, gm = oracle.uot_sinkhorn(x, a, y, b, eps, e1, e2, sweeps=3)
    ga, gx, gb, gy = oracle.dual_grad(x, a, y, b, eps, e1, e2, be, gm)

    def f(x, a, y, b):
        return oracle.dual_value(x, a, y, b, eps, e1, e2, be, gm)

    args = dict(x=x, a=a, y=y, b=b)
    for name, g in (("a", ga), ("x", gx), ("b", gb), ("y", gy)):
        assert close(g, fd_grad(f, args, name), 1e-7), name
    tot = gx.sum(0) + gy.sum(0)
    assert np.max(np.abs(tot)) <= 1e-13 * np.max(np.abs(gx))


@pytest.mark.parametrize("d", [1, 2])
def test_sinkhorn_divergence_grad_matches_finite_differences_at_convergence(d):
    """Envelope theorem: at the fixed point the partial derivative of D is the
    derivative of the value (and of the divergence built from three values)."""
    x, a, y, b = clouds(41 + d, d=d)
    eps, eta, S = 0.1, 0.7, 1500
    v, ga, gx, gb, gy = oracle.sinkhorn_divergence_grad(x, a, y, b, eps, eta, S)
    assert v == oracle.sinkhorn_divergence(x, a, y, b, eps, eta, S)

    def f(x, a, y, b):
        return oracle.sinkhorn_divergence(x, a, y, b, eps, eta, S)

    args = dict(x=x, a=a, y=y, b=b)
    for name, g in (("a", ga), ("x", gx), ("b", gb), ("y", gy)):
        assert close(g, fd_grad(f, args, name), 1e-6), name


def test_sinkhorn_divergence_grad_invariants():
    x, a, y, b = clouds(51, n=6, m=8, d=2)
    eps, eta = 0.08, 1.0
    # translation invariance holds at any sweep count (D depends on the points
    # only through the kernel)
    _, _, gx, _, gy = oracle.sinkhorn_divergence_grad(x, a, y, b, eps, eta, 20)
    tot = gx.sum(0) + gy.sum(0)
    assert np.max(np.abs(tot)) <= 1e-12 * np.max(np.abs(gx))
    # nu = mu is the minimum of the divergence: the nu- and y-gradients vanish
    # at convergence
    v, ga, gx, gb, gy = oracle.sinkhorn_divergence_grad(x, a, x, a, eps, eta, 2000)
    assert abs(v) <= 1e-12
    assert np.max(np.abs(gb)) <= 1e-9 and np.max(np.abs(gy)) <= 1e-9
