"""GPU parity of the NFFT fast summation (Sec. 4) against the oracle: every
stage against its numpy FP64 restatement, the whole summation against the
exact kernel sum, and the NFFT Sinkhorn (Alg. 2) against the FP64 Alg. 1.

Tolerances.  The binning is integer work: bit-exact.  Stages run in FP32 with
window weights accurate to ~1e-6 relative: grids are compared elementwise at
2e-5 of their max.  The approximation error of the fast sum is absolute,
proportional to sum |w| (the window and truncation errors are below 1e-9 at
the plan's m and h), so the end-to-end bound is max|s - s*| <= 1e-5 sum|w|,
and the relative L2 error ||s - s*|| / ||s*|| <= 1e-4 (the NFFT tolerance).
"""
import numpy as np
import pytest

import oracle
import oracle.nfft as onf
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


def cloud(seed, n, d, kind="uniform"):
    g = inputs.rng(seed)
    if kind == "uniform":
        return g.uniform(-0.3, 0.3, (n, d)).astype(np.float32)
    means = g.uniform(-0.2, 0.2, (5, d))
    return inputs.gmm_points(g, n, means, 0.03)


def plan_for(uotk, src, tgt, eps, **kw):
    p = uotk.nfft_plan(dev(src), dev(tgt), eps, **kw)
    return p, p.as_dict()


def torus(P, pts):
    d = pts.shape[1]
    c = np.array(P["center"][:d], dtype=np.float32).astype(np.float64)
    u = np.full((pts.shape[0], 3), 0.5)
    u[:, :d] = onf.torus_coords(f64(pts), c, P["h"])
    return u


@pytest.mark.parametrize("d", [1, 2, 3])
def test_cells_bit_exact(uotk, d):
    src = cloud(1, 5000, d)
    tgt = cloud(2, 3000, d)
    p, P = plan_for(uotk, src, tgt, 0.05)
    cells = uotk.nfft_cells(p, dev(src)).cpu().numpy()
    want = onf.cell_index_f32(src, np.array(P["center"][:d], np.float32), np.float32(P["inv_h"]),
                              P["grid"])
    assert np.array_equal(cells[:, :d], want)
    if d < 3:
        assert np.all(cells[:, d:] == P["grid"] // 2)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_spread_stage(uotk, d):
    src = cloud(3, 3000, d, "gmm")
    w = inputs.rng(4).uniform(0.2, 2.0, 3000).astype(np.float32)
    p, P = plan_for(uotk, src, src, 0.02, grid=64)
    g = uotk.nfft_spread(p, dev(src), dev(w)).cpu().numpy().astype(np.float64)
    u = torus(P, src)
    want = onf.spread(u, f64(w), P["grid"], P["bandwidth"], P["cutoff"])
    # oracle axes (x, y, z) -> GPU layout [z][y][x]; oracle window is unnormalised
    want = np.transpose(want, (2, 1, 0)) / onf.kb_phi(np.zeros(1), P["grid"], P["bandwidth"],
                                                      P["cutoff"])[0] ** 3
    assert np.max(np.abs(g - want)) <= 2e-5 * np.max(np.abs(want))


@pytest.mark.parametrize("grid,cutoff", [(16, 6), (16, 3)])
def test_spread_stage_small_grids(uotk, grid, cutoff):
    """The smallest grid, two tiles per axis: the tile offsets -1 and +1 of the
    fold name the same tile, whose block wraps onto itself and covers some nodes
    twice (the torus case of the fixed-order fold)."""
    src = cloud(11, 2500, 3, "gmm")
    w = inputs.rng(12).uniform(0.2, 2.0, 2500).astype(np.float32)
    p, P = plan_for(uotk, src, src, 0.02, grid=grid, cutoff=cutoff, period=1.0)
    g = uotk.nfft_spread(p, dev(src), dev(w)).cpu().numpy().astype(np.float64)
    u = torus(P, src)
    want = onf.spread(u, f64(w), P["grid"], P["bandwidth"], P["cutoff"])
    want = np.transpose(want, (2, 1, 0)) / onf.kb_phi(np.zeros(1), P["grid"], P["bandwidth"],
                                                      P["cutoff"])[0] ** 3
    assert np.max(np.abs(g - want)) <= 2e-5 * np.max(np.abs(want))


def test_spread_and_sum_are_deterministic(uotk):
    """The spread stage and the NFFT kernel sum give bit-identical results on
    repeated calls, also from a second context (other workspace addresses):
    the points of a cell keep their caller order (stable binning) and the unit
    blocks are folded into the grid in a fixed order, without atomics."""
    src = cloud(13, 30000, 3, "gmm")
    tgt = cloud(14, 20001, 3, "gmm")
    w = inputs.rng(15).lognormal(0.0, 0.5, 30000).astype(np.float32)
    p, P = plan_for(uotk, src, tgt, 0.02)
    g1 = uotk.nfft_spread(p, dev(src), dev(w))
    g2 = uotk.nfft_spread(p, dev(src), dev(w))
    assert torch.equal(g1, g2)
    s1 = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft")
    s2 = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft")
    ctx2 = uotk.Context(0)
    s3 = uotk.kernel_sum(dev(src), dev(w), dev(tgt), 0.02, method="nfft", ctx=ctx2)
    ctx2.close()
    assert torch.equal(s1, s2) and torch.equal(s1, s3)


def test_sinkhorn_nfft_is_deterministic(uotk):
    """Alg. 2 solved twice on the graph path, and once with eager launches
    (per-stage profiling on), gives bit-identical duals and dual values."""
    W = inputs.gmm3(seed=2007, n=40000, m=33001)
    args = (dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho)
    ctx = uotk.Context(0)
    r1 = uotk.uot_sinkhorn(*args, max_sweeps=24, method="nfft", ctx=ctx)
    r2 = uotk.uot_sinkhorn(*args, max_sweeps=24, method="nfft", ctx=ctx)
    ctx.set_profiling(True)
    r3 = uotk.uot_sinkhorn(*args, max_sweeps=24, method="nfft", ctx=ctx)
    ctx.set_profiling(False)
    ctx.close()
    for r in (r2, r3):
        assert torch.equal(r1[0], r[0]) and torch.equal(r1[1], r[1]) and r1[3] == r[3]


@pytest.mark.parametrize("grid", [64, 128])
def test_convolve_stage(uotk, grid):
    """The grid convolution against its FP64 restatement: the pruned 3-D FFT
    (grid 64) and the three separable circulant passes of the Gaussian
    (grid 128), on a standard normal grid (every frequency present)."""
    src = cloud(5, 2000, 3)
    p, P = plan_for(uotk, src, src, 0.05, grid=grid)
    n, N, m = P["grid"], P["bandwidth"], P["cutoff"]
    g = inputs.rng(6).standard_normal((n, n, n)).astype(np.float32)
    out = uotk.nfft_convolve(p, dev(g)).cpu().numpy().astype(np.float64)
    # oracle in its own axis order with the normalised window: scale by phi(0)^2
    phi0 = onf.kb_phi(np.zeros(1), n, N, m)[0]
    want = onf.convolve_grid(np.transpose(f64(g), (2, 1, 0)), N, m, P["eps"], P["h"]) * phi0 ** 6
    want = np.transpose(want, (2, 1, 0))
    assert np.max(np.abs(out - want)) <= 2e-5 * np.max(np.abs(want))


@pytest.mark.parametrize("d", [1, 3])
def test_gather_stage(uotk, d):
    tgt = cloud(7, 2500, d, "gmm")
    p, P = plan_for(uotk, tgt, tgt, 0.02, grid=64)
    n, N, m = P["grid"], P["bandwidth"], P["cutoff"]
    grid = inputs.rng(8).standard_normal((n, n, n)).astype(np.float32)
    out = uotk.nfft_gather(p, dev(grid), dev(tgt)).cpu().numpy().astype(np.float64)
    phi0 = onf.kb_phi(np.zeros(1), n, N, m)[0]
    want = onf.gather_window(np.transpose(f64(grid), (2, 1, 0)), torus(P, tgt), N, m) / phi0 ** 3
    assert np.max(np.abs(out - want)) <= 2e-5 * np.max(np.abs(want))


def err_metrics(got, ref, w):
    got, ref = f64(got), f64(ref)
    return (np.max(np.abs(got - ref)) / np.sum(np.abs(w)),
            np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("d,kind", [(1, "uniform"), (2, "uniform"), (3, "uniform"), (3, "gmm")])
def test_kernel_sum_nfft_vs_exact(uotk, d, kind):
    src = cloud(20 + d, 3001, d, kind)
    tgt = cloud(40 + d, 1999, d, kind)
    w = inputs.rng(9).lognormal(0.0, 0.5, 3001).astype(np.float32)
    eps = 0.02
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), eps, method="nfft").cpu().numpy()
    ref = oracle.ksum(f64(src), f64(w), f64(tgt), eps)
    e_inf, e_l2 = err_metrics(got, ref, w)
    assert e_inf <= 1e-5 and e_l2 <= 1e-4, (e_inf, e_l2)


def test_kernel_sum_nfft_large_sampled(uotk):
    W = inputs.gmm3(seed=2000)
    out = uotk.kernel_sum(dev(W.y), dev(W.b), dev(W.x), W.eps, method="nfft").cpu().numpy()
    idx = inputs.subsample_rows(inputs.rng(5), 512, W.n)
    ref = oracle.ksum(f64(W.y), f64(W.b), f64(W.x[idx]), W.eps)
    e_inf, e_l2 = err_metrics(out[idx], ref, W.b)
    assert e_inf <= 1e-5 and e_l2 <= 1e-4, (e_inf, e_l2)


def test_kernel_sum_nfft_options_and_edges(uotk):
    src = cloud(30, 800, 3)
    w = np.ones(800, np.float32)
    ref = oracle.ksum(f64(src), f64(w), f64(src[:50]), 0.05)
    for kw in ({"grid": 64}, {"grid": 32, "bandwidth": 16, "cutoff": 4, "target_err": 1e-3},
               {"cutoff": 8}):
        got = uotk.kernel_sum(dev(src), dev(w), dev(src[:50]), 0.05, method="nfft", **kw)
        e_inf, _ = err_metrics(got.cpu().numpy(), ref, w)
        tol = 1e-3 if kw.get("cutoff") == 4 else 1e-5
        assert e_inf <= tol, (kw, e_inf)
    # one source, coincident targets
    one = uotk.kernel_sum(dev(src[:1]), dev(w[:1]), dev(np.repeat(src[:1], 3, 0)), 0.05,
                          method="nfft").cpu().numpy()
    assert np.allclose(one, 1.0, atol=1e-5)
    # too coarse a grid for a tiny eps is refused, not silently wrong
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(dev(src), dev(w), dev(src), 1e-5, method="nfft", grid=32)
    assert e.value.status == 4


def residual(b, g, rb, rg):
    return (np.linalg.norm(b - rb) / np.linalg.norm(rb)
            + np.linalg.norm(g - rg) / np.linalg.norm(rg))


def test_sinkhorn_nfft_vs_oracle(uotk):
    """Alg. 2 (NFFT) vs the FP64 Alg. 1 on the Gaussian-mixture workload at
    n = m = 4096, 200 sweeps: the paper's dual residual within 1e-4."""
    W = inputs.gmm3(seed=2001, n=4096, m=4096)
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b),
                                                      W.eps, W.rho, max_sweeps=W.sweeps,
                                                      method="nfft")
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=W.sweeps)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert sweeps == W.sweeps and res <= 1e-4, res
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg)
    assert abs(value - v) <= 1e-4 * abs(v), (value, v)


@pytest.mark.parametrize("ref", ["product", "counting"])
def test_sinkhorn_nfft_tracking_warm_start(uotk, ref):
    """Alg. 2 with the convergence test on, from a warm start, with either
    reference measure: every dual update of the NFFT form (done inside its
    gather kernel) against the FP64 Alg. 1 run for the sweeps the GPU took."""
    W = inputs.gmm3(seed=2004, n=2000, m=1500)
    r = 0 if ref == "product" else 1
    g0 = inputs.rng(2005).uniform(-0.02, 0.02, W.m)
    beta, gamma, sweeps, value, conv = uotk.uot_sinkhorn(
        dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho, max_sweeps=1000, tol=1e-5,
        ref=ref, gamma0=torch.from_numpy(g0), method="nfft")
    assert conv and 10 <= sweeps < 1000 and sweeps % 10 == 0, (conv, sweeps)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=sweeps, ref=r, gamma0=g0)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    assert res <= 1e-4, res
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg, ref=r)
    assert abs(value - v) <= 1e-4 * abs(v), (value, v)
    # where the GPU stopped, the oracle's last sweep changes lambda * duals by
    # about tol as well (slack 10x for the NFFT's own error)
    pb, pg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=sweeps - 1, ref=r, gamma0=g0)
    change = max(np.max(np.abs(rb - pb)), np.max(np.abs(rg - pg))) / W.eps
    assert change < 1e-4, change


@pytest.mark.parametrize("cutoff", [3, 4, 5, 7, 8])
def test_sinkhorn_nfft_cutoffs(uotk, cutoff):
    """Alg. 2 at every other window cut-off: the spread's thread boxes and
    weight threads differ with m (several chunk points per weight thread at
    m = 3, 5, 7), the gather is the per-warp form at m = 4 and the CTA-staged
    form at m = 3, 5, 7, 8 (without its footprint cache at m >= 7).  Against the
    FP64 Alg. 1 after 30 sweeps, both reference measures.  Tolerances follow the
    Kaiser-Bessel error bound of the cut-off (about 1e-4 at m = 3, below 1e-7
    at m = 7)."""
    W = inputs.gmm3(seed=2006, n=2000, m=1500)
    ref = "counting" if cutoff in (4, 8) else "product"
    r = 0 if ref == "product" else 1
    beta, gamma, sweeps, value, _ = uotk.uot_sinkhorn(
        dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho, max_sweeps=30, ref=ref,
        method="nfft", cutoff=cutoff, target_err=1e-3)
    X, Y, A, B = f64(W.x), f64(W.y), f64(W.a), f64(W.b)
    rb, rg = oracle.uot_sinkhorn(X, A, Y, B, W.eps, W.rho, sweeps=30, ref=r)
    res = residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg)
    tol = 1e-2 if cutoff <= 4 else 1e-3
    assert sweeps == 30 and res <= tol, (cutoff, res)
    v = oracle.dual_value(X, A, Y, B, W.eps, W.rho, W.rho, rb, rg, ref=r)
    assert abs(value - v) <= tol * abs(v), (cutoff, value, v)


def test_mmd2_nfft(uotk):
    W = inputs.gmm3(seed=2002, n=3000, m=2500)
    v, parts = uotk.mmd2(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.ell, method="nfft")
    rv, rp = oracle.mmd2(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.ell, return_parts=True)
    assert np.allclose(parts, rp, rtol=1e-5, atol=0)
    kappa = (rp[0] + 2 * rp[1] + rp[2]) / rv
    assert abs(v - rv) <= 1e-5 * kappa * abs(rv), (v, rv, kappa)


def test_sinkhorn_divergence_nfft(uotk):
    W = inputs.gmm3(seed=2003, n=1500, m=1200)
    sd, parts = uotk.sinkhorn_divergence(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho,
                                         max_sweeps=50, method="nfft")
    rsd, rparts = oracle.sinkhorn_divergence(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.eps, W.rho,
                                             sweeps=50, return_parts=True)
    assert np.allclose(parts, rparts, rtol=1e-4, atol=0)
    kappa = sum(abs(p) for p in rparts) / abs(rsd)
    assert abs(sd - rsd) <= 1e-4 * kappa * abs(rsd)


def test_sinkhorn_nfft_vs_direct_at_scale(uotk):
    """The scale workload itself (gmm3, n = m = 2^20): the NFFT solve against the
    GPU direct solve after 10 sweeps from the same start, in the paper's dual
    residual (Table Tab:Accuracy_analysis2), at the NFFT bar 1e-4.  (A full FP64
    oracle at 2^20 is out of reach of host cores; the direct form is held to the
    oracle at 1e-6 elsewhere.)"""
    W = inputs.gmm3(seed=2000)
    args = (dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho)
    bn, gn, _, vn, _ = uotk.uot_sinkhorn(*args, max_sweeps=10, method="nfft")
    bd, gd, _, vd, _ = uotk.uot_sinkhorn(*args, max_sweeps=10, method="direct")
    res = residual(bn.cpu().numpy(), gn.cpu().numpy(), bd.cpu().numpy(), gd.cpu().numpy())
    assert res <= 1e-4, res
    assert abs(vn - vd) <= 1e-4 * abs(vd), (vn, vd)
