"""Failure detection on the device without a fault: a bounded wait that runs out.

The library's kernels bound every wait on an mbarrier; when the limit passes they record
a timeout in the context's status word and unwind.  xpcs_selftest_timeout runs such a
wait that nothing satisfies: the host must see XPCS_ETIMEOUT, after about the limit,
and the context must stay usable for real work, in synchronous and asynchronous mode.
"""
import time

import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, run_raw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


def _still_usable(X, ctx):
    frames = speckle_counts(16, 16, 70, 0.5, 1e-3, 5, np.uint8)
    qmap = ring_qmap(16, 16, 2)
    out = run_raw(X, ctx, frames, qmap, 2)
    for q in range(2):
        assert np.array_equal(lower(out["N"][q]), lower(O.raw_gram(frames, qmap, q)))


def test_expired_wait_reports_timeout_and_context_recovers(X):
    ctx = X.Context(0)
    t0 = time.perf_counter()
    with pytest.raises(X.XpcsError) as ei:
        X.xpcs_selftest_timeout(ctx, 50)
    dt = time.perf_counter() - t0
    assert ei.value.status == X.XPCS_ETIMEOUT
    assert 0.045 < dt < 2.0, dt
    _still_usable(X, ctx)
    ctx.close()


def test_expired_wait_in_async_mode_surfaces_at_synchronize(X):
    ctx = X.Context(0)
    ctx.set_async(True)
    X.xpcs_selftest_timeout(ctx, 20)  # enqueued only
    with pytest.raises(X.XpcsError) as ei:
        ctx.synchronize()
    assert ei.value.status == X.XPCS_ETIMEOUT
    ctx.synchronize()  # the status was consumed: nothing pending
    ctx.set_async(False)
    _still_usable(X, ctx)
    ctx.close()


def test_selftest_rejects_out_of_range_limits(X):
    ctx = X.Context(0)
    for bad in (-5, 1001):  # 0 selects the context's limit
        with pytest.raises(X.XpcsError) as ei:
            X.xpcs_selftest_timeout(ctx, bad)
        assert ei.value.status == X.XPCS_EINVAL
    ctx.close()


def test_context_wait_limit_reaches_the_device_waits(X):
    """xpcs_set_timeout changes the limit of the library's own bounded wait (the one every
    tensor-core kernel uses), read by the kernel from the context's status block."""
    ctx = X.Context(0)
    assert ctx.timeout() == 2000  # the default
    for limit_ms in (60, 400):
        ctx.set_timeout(limit_ms)
        assert ctx.timeout() == limit_ms
        t0 = time.perf_counter()
        with pytest.raises(X.XpcsError) as ei:
            X.xpcs_selftest_timeout(ctx, 0)  # a wait nothing satisfies, with the context's limit
        dt = time.perf_counter() - t0
        assert ei.value.status == X.XPCS_ETIMEOUT
        assert limit_ms / 1000 <= dt < limit_ms / 1000 + 1.0, dt
        _still_usable(X, ctx)  # real work completes well within the shortened limit
    ctx.set_timeout(0)
    assert ctx.timeout() == 2000
    for bad in (-1, 600001):
        with pytest.raises(X.XpcsError) as ei:
            ctx.set_timeout(bad)
        assert ei.value.status == X.XPCS_EINVAL
    ctx.close()
