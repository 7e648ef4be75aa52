"""GPU parity of the gradient operations (uotk_mmd2_grad,
uotk_sinkhorn_divergence_grad) against the FP64 oracle, through the C ABI.

Error model.  Every gradient row is a difference of kernel sums: the weight
gradients subtract two sums, the point gradients form x'_i t_i - s_i with
coordinates shifted to the first point of x.  The bound therefore scales
with the size of the cancelling terms, not with the result:
  * direct form: each FP32 sum has relative error <= delta = 2e-6 with
    respect to the sum of |terms| (the kernel-sum parity bar); a coordinate-
    weighted sum's |terms| are at most R times the plain sum's, R the largest
    coordinate offset from the origin;
  * NFFT form: each sum has absolute error <= E * ||w||_1 with E = 1e-5 (the
    fast-summation bar of the NFFT tests);
  * Sinkhorn divergence: the duals carry the FP32 sum error through the
    iteration, contracted by lambda*q = eta*lambda/(1 + eta*lambda) per
    half-step, so lambda*|beta - beta*| <= delta (1 + eta*lambda); the bound
    adds that to the sums' delta.
Each test computes the scale of the cancelling terms from oracle quantities
and checks |g - g*| <= tol * scale elementwise.  These bounds are worst
cases (measured errors sit at 1-7% of them for the direct sums and far lower
for the duals), so every test also holds the normwise relative error
||g - g*|| / ||g*|| to a bar about ten times the measured value (NORM_*)."""
import numpy as np
import pytest

import oracle
from paper_2306_13618_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DELTA = 2e-6
E_NFFT = 1e-5
NORM_DIRECT = 1e-5     # measured <= 1.3e-6 (MMD^2), 3e-7 (divergence)
NORM_NFFT = 5e-5       # measured <= 1.5e-6 (MMD^2), 4.7e-6 (divergence)


def normwise(got, ref):
    return np.linalg.norm(host(got) - ref) / np.linalg.norm(ref)


@pytest.fixture(scope="module")
def uotk():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f64(a):
    return np.asarray(a, dtype=np.float64)


def host(t):
    return t.cpu().numpy()


def clouds(seed, n, m, d, mass=1.3, lo=-0.3, hi=0.3):
    g = inputs.rng(seed)
    x = g.uniform(lo, hi, (n, d)).astype(np.float32)
    y = g.uniform(lo + 0.05, hi + 0.1, (m, d)).astype(np.float32)
    a = (g.uniform(0.5, 1.5, n) / n).astype(np.float32)
    b = (g.uniform(0.5, 1.5, m) * mass / m).astype(np.float32)
    return x, a, y, b


def offset_radius(x, y):
    """Largest |p_c - x_0c| over both clouds (the shifted-coordinate scale)."""
    o = f64(x[0])
    return max(np.max(np.abs(f64(x) - o)), np.max(np.abs(f64(y) - o)))


def mmd_scales(x, a, y, b, ell, err):
    """Per-row bounds on |g - g*| for MMD^2: err(w) is the error of a sum with
    weights w at every target (array over the targets of that side)."""
    eps = ell * ell
    X, Y, A, B = f64(x), f64(y), f64(a), f64(b)
    R = offset_radius(x, y)
    out = []
    for P, W, Q, V in ((X, A, Y, B), (Y, B, X, A)):
        e1, e2 = err(P, W, P), err(Q, V, P)        # the two plain sums
        ga = 2 * (e1 + e2)
        gp = 4 * W / eps * 2 * R * (e1 + e2)        # |x'| t and s, both sums
        out += [ga, gp[:, None] * np.ones((1, P.shape[1]))]
    return out


def direct_err(src, w, tgt, eps):
    return DELTA * oracle.ksum(src, np.abs(w), tgt, eps)


@pytest.mark.parametrize("d,n,m", [(3, 1537, 999), (1, 700, 1301), (5, 513, 257)])
def test_mmd2_grad_direct(uotk, d, n, m):
    x, a, y, b = clouds(300 + d, n, m, d)
    ell = 0.2
    v, ga, gx, gb, gy = uotk.mmd2_grad(dev(x), dev(a), dev(y), dev(b), ell)
    ra, rx, rb, ry = oracle.mmd2_grad(f64(x), f64(a), f64(y), f64(b), ell)
    rv, rp = oracle.mmd2(f64(x), f64(a), f64(y), f64(b), ell, return_parts=True)
    assert abs(v - rv) <= 1e-6 * (rp[0] + 2 * rp[1] + rp[2])
    sc = mmd_scales(x, a, y, b, ell, lambda s, w, t: direct_err(s, w, t, ell * ell))
    for got, ref, s, name in zip((ga, gx, gb, gy), (ra, rx, rb, ry), sc, "axby"):
        err = np.abs(host(got) - ref)
        assert np.all(err <= 2 * s), (name, np.max(err / s))
        assert normwise(got, ref) <= NORM_DIRECT, (name, normwise(got, ref))


def test_mmd2_grad_nfft(uotk):
    W = inputs.gmm3(seed=2004, n=4096, m=4096)
    x, a, y, b, ell = W.x, W.a, W.y, W.b, W.ell
    v, ga, gx, gb, gy = uotk.mmd2_grad(dev(x), dev(a), dev(y), dev(b), ell, method="nfft")
    ra, rx, rb, ry = oracle.mmd2_grad(f64(x), f64(a), f64(y), f64(b), ell)

    def nfft_err(src, w, tgt):
        return np.full(tgt.shape[0], E_NFFT * np.sum(np.abs(w)))

    sc = mmd_scales(x, a, y, b, ell, nfft_err)
    for got, ref, s, name in zip((ga, gx, gb, gy), (ra, rx, rb, ry), sc, "axby"):
        err = np.abs(host(got) - ref)
        assert np.all(err <= 2 * s), (name, np.max(err / s))
        assert normwise(got, ref) <= NORM_NFFT, (name, normwise(got, ref))


def test_mmd2_grad_large_sampled(uotk):
    """n = m = 2^20, d = 3 Gaussian mixture, NFFT: 64 sampled rows of each side
    against the oracle's row-wise gradient over all 2 x 2^20 points."""
    W = inputs.gmm3(seed=2000)
    ell = W.ell
    v, ga, gx, gb, gy = uotk.mmd2_grad(dev(W.x), dev(W.a), dev(W.y), dev(W.b), ell,
                                       method="nfft")
    R = offset_radius(W.x, W.y)
    mass = float(np.sum(f64(W.a)) + np.sum(f64(W.b)))
    for side, (gw, gp, P, Wt) in enumerate(((ga, gx, W.x, W.a), (gb, gy, W.y, W.b))):
        rows = inputs.subsample_rows(inputs.rng(60 + side), 64, P.shape[0])
        rw, rp = oracle.mmd2_grad_rows(f64(W.x), f64(W.a), f64(W.y), f64(W.b), ell, side, rows)
        e = E_NFFT * mass
        assert np.all(np.abs(host(gw)[rows] - rw) <= 2 * 2 * e)
        bound = 4 * f64(Wt)[rows] / ell**2 * 2 * R * e * 2
        assert np.all(np.abs(host(gp)[rows] - rp) <= bound[:, None])
    # translation invariance over all 2^21 rows
    tot = host(gx).sum(0) + host(gy).sum(0)
    scale = np.abs(host(gx)).sum(0) + np.abs(host(gy)).sum(0)
    assert np.all(np.abs(tot) <= 1e-4 * scale)


def uot_scales(x, a, y, b, eps, rho, sweeps):
    """|cancelling terms| of one UOT problem's gradient rows, both roles, from
    the oracle duals: (s_a, s_x, s_b, s_y) and the R used."""
    X, Y, A, B = f64(x), f64(y), f64(a), f64(b)
    lam = 1.0 / eps
    be, gm = oracle.uot_sinkhorn(X, A, Y, B, eps, rho, rho, sweeps=sweeps)
    T = oracle.ksum(Y, B * np.exp(lam * gm), X, eps)
    Tp = oracle.ksum(X, A * np.exp(lam * be), Y, eps)
    R = offset_radius(x, y)
    ea, eb = np.exp(lam * be) * T, np.exp(lam * gm) * Tp
    s_a = rho * np.exp(-be / rho) + rho + (ea + B.sum()) / lam
    s_b = rho * np.exp(-gm / rho) + rho + (eb + A.sum()) / lam
    s_x = 2 * A * ea * 2 * R
    s_y = 2 * B * eb * 2 * R
    return s_a, s_x, s_b, s_y


def sd_scales(x, a, y, b, eps, rho, sweeps):
    p0 = uot_scales(x, a, y, b, eps, rho, sweeps)
    p1 = uot_scales(x, a, x, a, eps, rho, sweeps)
    p2 = uot_scales(y, b, y, b, eps, rho, sweeps)
    return (p0[0] + 0.5 * (p1[0] + p1[2]), p0[1] + 0.5 * (p1[1] + p1[3]),
            p0[2] + 0.5 * (p2[0] + p2[2]), p0[3] + 0.5 * (p2[1] + p2[3]))


@pytest.mark.parametrize("d,n,m", [(2, 800, 700), (3, 513, 1025)])
def test_sinkhorn_divergence_grad_direct(uotk, d, n, m):
    x, a, y, b = clouds(320 + d, n, m, d)
    eps, rho, S = 0.05, 1.0, 60
    sd, parts, ga, gx, gb, gy = uotk.sinkhorn_divergence_grad(dev(x), dev(a), dev(y), dev(b),
                                                             eps, rho, max_sweeps=S)
    rsd, ra, rx, rb, ry = oracle.sinkhorn_divergence_grad(f64(x), f64(a), f64(y), f64(b), eps,
                                                          rho, S)
    sd_plain, _ = uotk.sinkhorn_divergence(dev(x), dev(a), dev(y), dev(b), eps, rho, max_sweeps=S)
    assert sd == sd_plain
    tol = DELTA * (2 + rho / eps)
    sc = sd_scales(x, a, y, b, eps, rho, S)
    for got, ref, s, name in zip((ga, gx, gb, gy), (ra, rx, rb, ry), sc, "axby"):
        s = s if s.ndim == np.ndim(ref) else s[:, None]
        err = np.abs(host(got) - ref)
        assert np.all(err <= 2 * tol * s), (name, np.max(err / s) / tol)
        assert normwise(got, ref) <= NORM_DIRECT, (name, normwise(got, ref))


def test_sinkhorn_divergence_grad_nfft(uotk):
    W = inputs.gmm3(seed=2005, n=4096, m=4096)
    x, a, y, b = W.x, W.a, W.y, W.b
    eps, rho, S = W.eps, W.rho, 30
    sd, parts, ga, gx, gb, gy = uotk.sinkhorn_divergence_grad(dev(x), dev(a), dev(y), dev(b),
                                                             eps, rho, max_sweeps=S,
                                                             method="nfft")
    rsd, ra, rx, rb, ry = oracle.sinkhorn_divergence_grad(f64(x), f64(a), f64(y), f64(b), eps,
                                                          rho, S)
    # NFFT sums: absolute error E ||w||_1; the duals carry it as in the
    # Sinkhorn NFFT parity test, whose normwise bar this follows.
    assert abs(sd - rsd) <= 1e-4 * sum(abs(p) for p in parts)
    for got, ref, name in zip((ga, gx, gb, gy), (ra, rx, rb, ry), "axby"):
        assert normwise(got, ref) <= NORM_NFFT, (name, normwise(got, ref))


def test_grad_selective_outputs_and_autograd(uotk):
    x, a, y, b = clouds(340, 300, 200, 2)
    ell = 0.3
    full = uotk.mmd2_grad(dev(x), dev(a), dev(y), dev(b), ell)
    part = uotk.mmd2_grad(dev(x), dev(a), dev(y), dev(b), ell, need=(False, True, False, False))
    assert part[1] is None and part[3] is None and part[4] is None
    assert part[0] == full[0] and torch.equal(part[2], full[2])
    # autograd: the loss's backward returns the library gradient times grad_output
    xt, at = dev(x).requires_grad_(), dev(a).requires_grad_()
    yt, bt = dev(y).requires_grad_(), dev(b).requires_grad_()
    loss = uotk.mmd2_loss(xt, at, yt, bt, ell)
    (3.0 * loss).backward()
    assert loss.item() == full[0]
    for t, g in ((at, full[1]), (xt, full[2]), (bt, full[3]), (yt, full[4])):
        assert t.grad.dtype == torch.float32
        assert torch.allclose(t.grad.double(), 3.0 * g, rtol=1e-6, atol=0)
    xs = dev(x).requires_grad_()
    sd = uotk.sinkhorn_divergence_loss(xs, dev(a), dev(y), dev(b), 0.05, 1.0, max_sweeps=40)
    sd.backward()
    ref = uotk.sinkhorn_divergence_grad(dev(x), dev(a), dev(y), dev(b), 0.05, 1.0,
                                        max_sweeps=40)
    assert sd.item() == ref[0]
    assert torch.allclose(xs.grad.double(), ref[3], rtol=1e-6, atol=0)


def test_grad_translation_invariance_direct(uotk):
    """Sum of point gradients = 0 (both quantities depend on the points only
    through differences), for the library's own output at any sweep count."""
    x, a, y, b = clouds(350, 1000, 900, 3)
    _, _, gx, _, gy = uotk.mmd2_grad(dev(x), dev(a), dev(y), dev(b), 0.2)
    tot = host(gx).sum(0) + host(gy).sum(0)
    assert np.all(np.abs(tot) <= 1e-5 * (np.abs(host(gx)).sum(0) + np.abs(host(gy)).sum(0)))
    _, _, _, gx, _, gy = uotk.sinkhorn_divergence_grad(dev(x), dev(a), dev(y), dev(b), 0.05, 1.0,
                                                      max_sweeps=25)
    tot = host(gx).sum(0) + host(gy).sum(0)
    assert np.all(np.abs(tot) <= 1e-5 * (np.abs(host(gx)).sum(0) + np.abs(host(gy)).sum(0)))
