"""GPU parity of the batched solver (uotk_uot_sinkhorn_batch) against the FP64
oracle, pair by pair, through the C ABI.

Every pair runs the same Alg. 1 as uotk_uot_sinkhorn with the direct form, so
each is held to the direct form's bar: the paper's dual residual <= 1e-6
(Table Tab:Accuracy_analysis2) after the same number of sweeps, and the dual
value to 1e-6 relative."""
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


def run(uotk, B, **kw):
    return uotk.uot_sinkhorn_batch(dev(B.x), dev(B.a), B.x_off, dev(B.y), dev(B.b), B.y_off,
                                   B.eps, B.rho, **kw)


def check_pairs(B, beta, gamma, sweeps, values, pairs):
    beta, gamma = beta.cpu().numpy(), gamma.cpu().numpy()
    for p in pairs:
        x, a, y, b, eps, rho = B.pair(p)
        X, A, Y, Bw = f64(x), f64(a), f64(y), f64(b)
        rb, rg = oracle.uot_sinkhorn(X, A, Y, Bw, eps, rho, sweeps=int(sweeps[p]))
        gb = beta[B.x_off[p]:B.x_off[p + 1]]
        gg = gamma[B.y_off[p]:B.y_off[p + 1]]
        res = residual(gb, gg, rb, rg)
        assert res <= 1e-6, (p, res, eps, rho)
        v = oracle.dual_value(X, A, Y, Bw, eps, rho, rho, rb, rg)
        assert abs(values[p] - v) <= 1e-6 * abs(v) + 1e-12, (p, values[p], v)


def test_batch_fixed_sweeps_matches_oracle(uotk):
    """32 pairs, n and m log-uniform in [64, 2048] (ragged, some below one
    source tile), eps and rho drawn per pair, 30 sweeps each."""
    B = inputs.pair_batch(seed=4001, npairs=32, nmin=64, nmax=2048)
    beta, gamma, sweeps, values, conv = run(uotk, B, max_sweeps=30)
    assert np.all(sweeps == 30)
    check_pairs(B, beta, gamma, sweeps, values, range(B.npairs))


def test_batch_tolerance_retires_pairs(uotk):
    """tol = 1e-6: pairs with fast contraction (small eta lambda) retire after
    a few tens of sweeps, the others keep going; each pair's duals equal the
    oracle's after exactly its own sweep count."""
    B = inputs.pair_batch(seed=4002, npairs=16, nmin=64, nmax=1024, eps_choices=(0.05,),
                          rho_choices=(0.1, 1.0))
    beta, gamma, sweeps, values, conv = run(uotk, B, max_sweeps=400, tol=1e-6)
    assert conv
    assert len(set(sweeps.tolist())) > 1          # not all at the same count
    # the device loop checks after the first sweep and every two sweeps after it
    assert np.all(sweeps % 2 == 1)
    check_pairs(B, beta, gamma, sweeps, values, range(B.npairs))


def test_batch_workload_sizes_match_oracle(uotk):
    """Pairs of the batched workload's sizes (n, m from 22k to 65k, eps and rho
    drawn per pair): every direction splits its sources over two to four
    groups of 64 tiles, whose FP32 partial sums are combined in FP64 by the
    dual update.  Each pair against the FP64 oracle after 4 sweeps."""
    B = inputs.pair_batch(seed=4012, npairs=4, nmin=20000, nmax=65536)
    beta, gamma, sweeps, values, conv = run(uotk, B, max_sweeps=4)
    assert np.all(sweeps == 4)
    check_pairs(B, beta, gamma, sweeps, values, range(B.npairs))


def test_batch_loop_cap_and_eager_path(uotk):
    """A sweep cap that the device loop's two-sweep body does not divide (the
    last sweep runs after the graph) and the eager path of per-stage profiling
    give the same duals as the oracle at the cap."""
    B = inputs.pair_batch(seed=4004, npairs=6, nmin=64, nmax=1500)
    for prof in (False, True):
        ctx = uotk.Context(0)
        ctx.set_profiling(prof)
        beta, gamma, sweeps, values, conv = uotk.uot_sinkhorn_batch(
            dev(B.x), dev(B.a), B.x_off, dev(B.y), dev(B.b), B.y_off, B.eps, B.rho,
            max_sweeps=12, ctx=ctx)
        ctx.close()
        assert np.all(sweeps == 12)
        check_pairs(B, beta, gamma, sweeps, values, range(B.npairs))


def test_batch_single_pair_equals_single_solver(uotk):
    """One pair through the batch equals uotk_uot_sinkhorn on that pair bit for
    bit in the duals' arithmetic: same kernels, same order of sums."""
    W = inputs.uniform_box(n=700, m=500, d=3)
    beta, gamma, sweeps, values, _ = uotk.uot_sinkhorn_batch(
        dev(W.x), dev(W.a), [0, 700], dev(W.y), dev(W.b), [0, 500], [W.eps], [W.rho],
        max_sweeps=25)
    b1, g1, s1, v1, _ = uotk.uot_sinkhorn(dev(W.x), dev(W.a), dev(W.y), dev(W.b), W.eps, W.rho,
                                          max_sweeps=25)
    rb, rg = oracle.uot_sinkhorn(f64(W.x), f64(W.a), f64(W.y), f64(W.b), W.eps, W.rho, sweeps=25)
    assert residual(beta.cpu().numpy(), gamma.cpu().numpy(), rb, rg) <= 1e-6
    assert residual(b1.cpu().numpy(), g1.cpu().numpy(), rb, rg) <= 1e-6
    assert abs(values[0] - v1) <= 1e-6 * abs(v1)


def test_batch_validation(uotk):
    B = inputs.pair_batch(seed=4003, npairs=3, nmin=16, nmax=64)
    bad_off = B.x_off.copy()
    bad_off[1] = bad_off[0]  # empty first pair
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn_batch(dev(B.x), dev(B.a), bad_off, dev(B.y), dev(B.b), B.y_off,
                                B.eps, B.rho)
    assert e.value.status == 1
    eps = B.eps.copy()
    eps[2] = -1.0
    with pytest.raises(uotk.UotkError) as e:
        run(uotk, inputs.PairBatch(B.x, B.a, B.x_off, B.y, B.b, B.y_off, eps, B.rho))
    assert e.value.status == 1


def test_batch_auto_takes_nfft_for_large_clustered_pairs(uotk):
    """UOTK_AUTO: pairs with at least 16384 points on both sides have their form
    measured (per sum on a built plan); on clustered clouds of about 2e4 points
    the NFFT wins and those pairs are solved by Alg. 2, while the small pairs
    stay in the grouped direct batch.  Every pair against the FP64 Alg. 1 after
    10 sweeps: direct-form pairs at the direct bar (1e-6), NFFT-form pairs at
    the NFFT bar (1e-4, residual and value)."""
    g = inputs.rng(4200)
    sizes = [(2000, 3000), (20000, 18000), (4000, 2500), (19000, 21000), (3000, 3500)]
    eps = [0.02, 0.02, 0.05, 0.02, 0.05]
    rho = [0.5, 0.5, 1.0, 0.5, 1.0]
    xs, ys, As, Bs = [], [], [], []
    for n, m in sizes:
        means = g.uniform(-0.2, 0.2, (5, 3))
        xs.append(inputs.gmm_points(g, n, means, 0.03))
        ys.append(inputs.gmm_points(g, m, means, 0.03))
        As.append((g.uniform(0.5, 1.5, n) / n).astype(np.float32))
        Bs.append((g.uniform(0.5, 1.5, m) / m).astype(np.float32))
    x_off = np.cumsum([0] + [n for n, _ in sizes])
    y_off = np.cumsum([0] + [m for _, m in sizes])
    X, Y = np.concatenate(xs), np.concatenate(ys)
    A, B = np.concatenate(As), np.concatenate(Bs)
    beta, gamma, sw, vals, _ = uotk.uot_sinkhorn_batch(dev(X), dev(A), x_off, dev(Y), dev(B),
                                                       y_off, eps, rho, max_sweeps=10,
                                                       method="auto")
    forms = uotk.batch_forms(len(sizes))
    assert [int(f) for f in forms] == [uotk.DIRECT, uotk.NFFT, uotk.DIRECT, uotk.NFFT,
                                       uotk.DIRECT], forms
    beta, gamma = beta.cpu().numpy(), gamma.cpu().numpy()
    for p in range(len(sizes)):
        rb, rg = oracle.uot_sinkhorn(f64(xs[p]), f64(As[p]), f64(ys[p]), f64(Bs[p]), eps[p],
                                     rho[p], sweeps=10)
        res = residual(beta[x_off[p]:x_off[p + 1]], gamma[y_off[p]:y_off[p + 1]], rb, rg)
        bar = 1e-4 if forms[p] == uotk.NFFT else 1e-6
        assert sw[p] == 10 and res <= bar, (p, res)
        v = oracle.dual_value(f64(xs[p]), f64(As[p]), f64(ys[p]), f64(Bs[p]), eps[p], rho[p],
                              rho[p], rb, rg)
        assert abs(vals[p] - v) <= bar * abs(v) + 1e-12, (p, vals[p], v)
