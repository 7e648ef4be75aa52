"""uotk_kernel_sum_noalloc: the direct kernel sum for callers that may not
allocate device memory while they run (memory reserved once at start-up, or a
latency-critical path where an allocation would synchronise the device).  Its
scratch is a fixed array inside the library, shared by every call on a device.

The test calls it through the C ABI twice in a row on different inputs -- the
second call must not see anything the first left in the shared scratch -- and
compares each result with uotk_kernel_sum, the context-based entry point, and
with the FP64 oracle's kernel sum, at the direct form's tolerance (2e-6
relative per output).  With no sources the output must be all zeros.  This file
is collected last, and passes both alone in a fresh process and after the
other tests."""
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


def _case(seed, n, m, d):
    g = inputs.rng(seed)
    src = torch.from_numpy(g.uniform(-0.3, 0.3, (n, d)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(g.uniform(-0.3, 0.3, (m, d)).astype(np.float32)).cuda()
    w = torch.from_numpy(g.uniform(0.1, 2.0, n).astype(np.float32)).cuda()
    return src, w, tgt


def test_noalloc_matches_kernel_sum_twice(uotk):
    cases = [(_case(501, 3001, 1777, 3), 0.05), (_case(502, 20000, 4097, 2), 0.02)]
    for (src, w, tgt), eps in cases:
        out = torch.full((tgt.shape[0],), float("nan"), device="cuda")
        st = uotk.kernel_sum_noalloc(src, w, tgt, eps, out)
        assert st == 0
        ref = uotk.kernel_sum(src, w, tgt, eps)
        torch.cuda.synchronize()
        rel = ((out.double() - ref.double()).abs() / ref.double()).max().item()
        assert rel <= 2e-6, rel
        exact = oracle.ksum(src.cpu().double().numpy(), w.cpu().double().numpy(),
                            tgt.cpu().double().numpy(), eps)
        rel = np.max(np.abs(out.cpu().double().numpy() - exact) / exact)
        assert rel <= 2e-6, rel


def test_noalloc_no_sources_gives_zeros(uotk):
    _, _, tgt = _case(505, 10, 333, 3)
    src = torch.zeros((0, 3), device="cuda")
    out = torch.full((333,), float("nan"), device="cuda")
    assert uotk.kernel_sum_noalloc(src, torch.zeros(0, device="cuda"), tgt, 0.05, out) == 0
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_rejects_oversize_and_bad_weights(uotk):
    src, w, tgt = _case(503, 65537, 16, 3)
    out = torch.empty(16, device="cuda")
    assert uotk.kernel_sum_noalloc(src, w, tgt, 0.05, out) == 4   # UOTK_ERR_UNSUPPORTED
    src, w, tgt = _case(504, 100, 16, 3)
    w[7] = -1.0
    assert uotk.kernel_sum_noalloc(src, w, tgt, 0.05, out) == 1   # UOTK_ERR_INVALID
    q = torch.zeros((10, 4), device="cuda")
    assert uotk.kernel_sum_noalloc(q, torch.ones(10, device="cuda"), q, 0.05,
                                   torch.empty(10, device="cuda")) == 4
