"""GPU parity of the other kernels of Table tab:0 (Laplace, inverse
multiquadric, energy) in the direct FP32 form, through the C ABI.

Error model: every term of a sum with non-negative weights has one sign, so
the relative error of a sum is that of its terms.  A term carries the FP32
squared distance (a few ulp), the approximate sqrt / rsqrt (2^-22 relative) and,
for Laplace, ex2.approx of an exponent r/p computed with that sqrt: relative
error about 2^-22 (r/p) ln2 + a few ulp.  Tested at 2e-6 + 4 * 2^-22 * max r/p
(Laplace) and 2e-6 (IMQ, energy) per output."""
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


@pytest.mark.parametrize("kind,p", [("laplace", 0.2), ("imq", 0.3), ("energy", 1.0)])
@pytest.mark.parametrize("d,n,m", [(1, 1500, 999), (3, 3001, 1777), (7, 513, 600)])
def test_kernel_sum_other_kernels(uotk, kind, p, d, n, m):
    g = inputs.rng(500 + d)
    src = g.uniform(-0.5, 0.5, (n, d)).astype(np.float32)
    tgt = g.uniform(-0.4, 0.6, (m, d)).astype(np.float32)
    w = g.uniform(0.1, 2.0, n).astype(np.float32)
    got = uotk.kernel_sum(dev(src), dev(w), dev(tgt), p, kernel=kind).cpu().numpy()
    ref = oracle.ksum_kernel(kind, p, f64(src), f64(w), f64(tgt))
    err = np.max(np.abs(got - ref) / np.abs(ref))
    if kind == "laplace":
        rmax = np.sqrt(d) * 1.1 / p
        tol = 2e-6 + 4 * 2.0 ** -22 * rmax
    else:
        tol = 2e-6
    assert err <= tol, (kind, d, err, tol)


@pytest.mark.parametrize("kind,p", [("laplace", 0.2), ("imq", 0.3), ("energy", 1.0),
                                    ("gauss", 0.2)])
def test_mmd2_other_kernels(uotk, kind, p):
    W = inputs.uniform_box(n=1500, m=1200)
    v, parts = uotk.mmd2(dev(W.x), dev(W.a), dev(W.y), dev(W.b), p, kernel=kind)
    rv, rp = oracle.mmd2_kernel(kind, p, f64(W.x), f64(W.a), f64(W.y), f64(W.b),
                                return_parts=True)
    tol = 2e-6 + (4 * 2.0 ** -22 * 0.75 / p if kind == "laplace" else 0.0)
    assert np.allclose(parts, rp, rtol=tol, atol=0), (parts, rp)
    kappa = (abs(rp[0]) + 2 * abs(rp[1]) + abs(rp[2])) / abs(rv)
    assert abs(v - rv) <= tol * kappa * abs(rv), (v, rv, kappa)


def test_other_kernels_unsupported_paths(uotk):
    W = inputs.uniform_box(n=200, m=200)
    args = (dev(W.x), dev(W.a), dev(W.y), dev(W.b))
    with pytest.raises(uotk.UotkError) as e:
        uotk.mmd2(*args, 0.2, method="direct_bf16", kernel="laplace")
    assert e.value.status == 4
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(*args, W.eps, W.rho, max_sweeps=3, kernel="imq")
    assert e.value.status == 4
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(args[0], args[1], args[2], 0.2, method="direct_bf16x3", kernel="energy")
    assert e.value.status == 4
