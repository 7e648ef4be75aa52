"""The failure statuses of the C ABI, reached without any device fault.

* UOTK_ERR_NOMEM: the context's workspace limit (uotk_set_workspace_limit) is
  below what the call needs; the call returns before it launches anything.
* UOTK_ERR_TIMEOUT: with uotk_set_wait_timeout_test, the first bounded wait of
  each NFFT spread and gather CTA waits on a barrier that nothing completes and
  runs out after the given cycles; the CTA then waits for its bulk copies in
  flight (normal limit) and leaves, and the host reads the time-out flag.
* In both cases the same context afterwards computes what a fresh context
  computes, bit for bit (the NFFT path is deterministic)."""
import numpy as np
import pytest

from paper_2306_13618_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOMEM, TIMEOUT = 2, 7


@pytest.fixture(scope="module")
def uotk():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk


@pytest.fixture(scope="module")
def clouds():
    W = inputs.gmm3(seed=2020, n=60000, m=50001)
    return tuple(torch.from_numpy(v).cuda() for v in (W.x, W.a, W.y, W.b)) + (W.eps, W.rho)


def test_workspace_limit_gives_nomem_then_recovers(uotk, clouds):
    x, a, y, b, eps, rho = clouds
    ref = uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=uotk.Context(0))
    ctx = uotk.Context(0)
    ctx.set_workspace_limit(1 << 20)
    l0 = ctx.launch_count()
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=ctx)
    assert e.value.status == NOMEM
    assert ctx.launch_count() == l0          # refused before any launch
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(x, a, y, b, eps, rho, max_sweeps=5, method="direct", ctx=ctx)
    assert e.value.status == NOMEM
    ctx.set_workspace_limit(0)
    out = uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=ctx)
    assert torch.equal(out, ref)
    with pytest.raises(uotk.UotkError) as e:
        ctx.set_workspace_limit(-1)
    assert e.value.status == 1
    ctx.close()


def test_wait_timeout_gives_timeout_then_recovers(uotk, clouds):
    x, a, y, b, eps, rho = clouds
    fresh = uotk.Context(0)
    ref = uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=fresh)
    rb, rg, _, rv, _ = uotk.uot_sinkhorn(x, a, y, b, eps, rho, max_sweeps=6, method="nfft",
                                         ctx=fresh)
    fresh.close()
    ctx = uotk.Context(0)
    ctx.set_wait_timeout_test(100000)        # about 50 us per CTA at 2 GHz
    with pytest.raises(uotk.UotkError) as e:
        uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=ctx)
    assert e.value.status == TIMEOUT
    with pytest.raises(uotk.UotkError) as e:
        uotk.uot_sinkhorn(x, a, y, b, eps, rho, max_sweeps=6, method="nfft", ctx=ctx)
    assert e.value.status == TIMEOUT
    ctx.set_wait_timeout_test(0)
    out = uotk.kernel_sum(y, b, x, eps, method="nfft", ctx=ctx)
    assert torch.equal(out, ref)
    gb, gg, _, gv, _ = uotk.uot_sinkhorn(x, a, y, b, eps, rho, max_sweeps=6, method="nfft",
                                         ctx=ctx)
    assert torch.equal(gb, rb) and torch.equal(gg, rg) and gv == rv
    ctx.close()
