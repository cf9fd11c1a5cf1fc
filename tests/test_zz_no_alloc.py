"""xpcs_g2_noalloc (g2 over a stored C with fixed scratch) against xpcs_g2.

Both calls go through the C ABI on the same inputs.  The no-allocation call must give
the same g2 (same kernels and row splits: equal within 1e-12 relative, counts exact) on
two calls in a row with different data, must not grow the context's device memory or
take memory from the device, and must reject sizes beyond its fixed scratch.  The file
is collected last so that it also runs after every other test in one process.
"""
import numpy as np
import pytest

from synth import ring_qmap, speckle_counts
from tests.gpu_util import run_raw, torch_cuda

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


def _stored_C(X, ctx, T, n_q, seed, dead=()):
    """A lower-triangle C from the raw path (NaN rows/columns for the dead frames)."""
    torch, dev = torch_cuda()
    frames = speckle_counts(32, 32, T, 0.4, 1e-3, seed, np.uint8)
    frames[list(dead)] = 0
    out = run_raw(X, ctx, frames, ring_qmap(32, 32, n_q), n_q, want_N=False)
    return torch.from_numpy(out["C"]).to(dev)


def _g2_pair(X, ctx, C, n_q, T):
    torch, dev = torch_cuda()
    g_ref = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    c_ref = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_g2(ctx, C, n_q, T, g_ref, c_ref)
    return g_ref.cpu().numpy(), c_ref.cpu().numpy()


def _check(g, c, g_ref, c_ref):
    np.testing.assert_array_equal(c, c_ref)
    assert np.array_equal(np.isnan(g), np.isnan(g_ref))
    ok = ~np.isnan(g_ref)
    np.testing.assert_allclose(g[ok], g_ref[ok], rtol=RTOL, atol=0)


def test_noalloc_matches_g2_on_two_calls_in_a_row(X):
    torch, dev = torch_cuda()
    ctx = X.Context(0)
    cases = [(333, 3, 11, (2, 40)), (517, 5, 12, (0, 300, 516))]  # ragged T, dead frames
    Cs = [_stored_C(X, ctx, T, n_q, seed, dead) for T, n_q, seed, dead in cases]
    # the first call on the device does the set-up; the context's scratch is not touched
    held0 = ctx.device_bytes()
    outs = []
    for i, ((T, n_q, _, _), C) in enumerate(zip(cases, Cs)):
        g = torch.full((n_q, T), -1.0, dtype=torch.float64, device=dev)
        c = torch.full((n_q, T), -1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        X.xpcs_g2_noalloc(ctx, C, n_q, T, g, c)
        torch.cuda.synchronize()
        if i > 0:  # after the set-up call nothing takes device memory
            assert torch.cuda.mem_get_info(dev)[0] == free0
        outs.append((g.cpu().numpy(), c.cpu().numpy()))
    assert ctx.device_bytes() == held0
    for (T, n_q, _, _), C, (g, c) in zip(cases, Cs, outs):
        _check(g, c, *_g2_pair(X, ctx, C, n_q, T))
    ctx.close()


def test_noalloc_repeats_after_a_larger_call(X):
    """A smaller call after a larger one reads none of the larger call's partials."""
    torch, dev = torch_cuda()
    ctx = X.Context(0)
    big = _stored_C(X, ctx, 700, 6, 13)
    small = _stored_C(X, ctx, 150, 2, 14, dead=(7,))
    for C, n_q, T in ((big, 6, 700), (small, 2, 150)):
        g = torch.empty((n_q, T), dtype=torch.float64, device=dev)
        c = torch.empty((n_q, T), dtype=torch.int64, device=dev)
        X.xpcs_g2_noalloc(ctx, C, n_q, T, g, c)
        _check(g.cpu().numpy(), c.cpu().numpy(), *_g2_pair(X, ctx, C, n_q, T))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(X):
    torch, dev = torch_cuda()
    ctx = X.Context(0)
    n_q, T = X.G2_NOALLOC_MAX_CELLS // 128 + 1, 128  # one ring past the limit
    C = torch.zeros((n_q, T, T), dtype=torch.float32, device=dev)  # a real buffer of the stated size
    g = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    launches = ctx.launch_count()
    with pytest.raises(X.XpcsError) as ei:
        X.xpcs_g2_noalloc(ctx, C, n_q, T, g)
    assert ei.value.status == X.XPCS_ERANGE
    assert "exceeds its fixed scratch" in str(ei.value)
    assert ctx.launch_count() == launches
    # more rings than a launch grid takes, though n_q * T is inside the cell limit
    with pytest.raises(X.XpcsError) as ei:
        X.xpcs_g2_noalloc(ctx, C, X.G2_MAX_RINGS + 1, 8, g)
    assert ei.value.status == X.XPCS_ERANGE
    assert ctx.launch_count() == launches
    # at the limit it runs and fills the whole array (partials and the count block at its
    # far end): values in [0.5, 1.5) with scattered NaN (undefined pairs), against xpcs_g2
    n_q = X.G2_NOALLOC_MAX_CELLS // 128
    gen = torch.Generator(device=dev)
    gen.manual_seed(20356)
    Cl = C[:n_q]
    Cl.copy_(torch.rand((n_q, T, T), generator=gen, device=dev) + 0.5)
    Cl[torch.rand((n_q, T, T), generator=gen, device=dev) < 0.05] = float("nan")
    Cl[5] = float("nan")  # one ring with no defined pair: g2 NaN, counts 0
    c = torch.full((n_q, T), -1, dtype=torch.int64, device=dev)
    X.xpcs_g2_noalloc(ctx, Cl, n_q, T, g[:n_q], c)
    g_ref, c_ref = _g2_pair(X, ctx, Cl, n_q, T)
    _check(g[:n_q].cpu().numpy(), c.cpu().numpy(), g_ref, c_ref)
    assert np.all(c_ref[5] == 0)
    ctx.close()
