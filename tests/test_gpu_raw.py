"""GPU parity of the raw exact path (Eq. 1-2, ring g2) against the CPU oracle.

Integer Grams and ring sums must be bit-exact; C (float32) within 1e-6 relative per
element (three float32 roundings of an exact integer ratio); g2 within 2e-6 relative;
pair counts exact.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, run_raw, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def _check_raw(X, ctx, frames, qmap, n_q):
    out = run_raw(X, ctx, frames, qmap, n_q)
    Cref, Nref, Sref, Mq = O.raw_twotime(frames, qmap, n_q)
    assert np.array_equal(lower(out["N"]), lower(Nref)), "integer Gram not bit-exact"
    Cu, Cr = lower(out["C"]), lower(Cref)
    np.testing.assert_array_equal(np.isnan(Cu), np.isnan(Cr))
    ok = ~np.isnan(Cr)
    np.testing.assert_allclose(Cu[ok], Cr[ok], rtol=1e-6, atol=0)
    for q in range(n_q):
        g_ref, c_ref = O.g2_from_twotime(Cref[q])
        np.testing.assert_array_equal(out["count"][q], c_ref)
        g = out["g2"][q]
        np.testing.assert_array_equal(np.isnan(g), np.isnan(g_ref))
        okg = ~np.isnan(g_ref)
        np.testing.assert_allclose(g[okg], g_ref[okg], rtol=2e-6, atol=0)
    return out


def test_raw_64x64_T500_eight_rings(X, ctx):
    # 64x64 detector, T = 500 frames, 8 equal-width rings, uint8 counts of mean 0.1
    frames = speckle_counts(64, 64, 500, 0.1, 1e-3, 20356001, np.uint8)
    _check_raw(X, ctx, frames, ring_qmap(64, 64, 8), 8)


@pytest.mark.parametrize("T", [1, 7, 128, 129, 300])
def test_raw_ragged_frame_counts(X, ctx, T):
    frames = speckle_counts(24, 40, T, 0.8, 2e-3, 11 + T, np.uint8)
    _check_raw(X, ctx, frames, ring_qmap(24, 40, 5), 5)


def test_raw_uint16_dark_frames_and_empty_ring(X, ctx):
    rng = np.random.default_rng(3)
    T, H, W, n_q = 260, 16, 48, 6
    frames = speckle_counts(H, W, T, 0.3, 3e-3, 5, np.uint16)
    frames[[0, 5, 130, 259]] = 0  # undefined frames: NaN pairs, excluded from g2
    qmap = ring_qmap(H, W, n_q)
    qmap[qmap == 4] = -1  # ring 4 is empty
    qmap[rng.random(qmap.size) < 0.1] = -1  # scattered unused pixels
    out = _check_raw(X, ctx, frames, qmap, n_q)
    assert np.all(out["count"][4] == 0) and np.all(np.isnan(out["g2"][4]))


def test_raw_large_counts_near_exact_limit(X, ctx):
    # counts up to 256 stay exact in bf16; the f32 accumulation stays exact below 2^24
    rng = np.random.default_rng(8)
    T, M, n_q = 150, 256, 2
    frames = rng.integers(0, 257, size=(T, M)).astype(np.uint16)
    qmap = (np.arange(M) % n_q).astype(np.int32)  # 128 px per ring: sum of squares < 2^24
    _check_raw(X, ctx, frames, qmap, n_q)


def test_raw_rejects_counts_above_exact_range(X, ctx):
    torch, dev = torch_cuda()
    frames = np.zeros((10, 64), dtype=np.uint16)
    frames[3, 5] = 300
    qmap = np.zeros(64, dtype=np.int32)
    with pytest.raises(X.XpcsError) as e:
        run_raw(X, ctx, frames, qmap, 1)
    assert e.value.status == X.XPCS_ERANGE
    # the context stays usable
    ok = speckle_counts(8, 8, 20, 1.0, 1e-3, 1, np.uint8)
    _check_raw(X, ctx, ok, ring_qmap(8, 8, 2), 2)


def test_ring_sums_exact(X, ctx):
    torch, dev = torch_cuda()
    frames = speckle_counts(32, 32, 77, 2.0, 1e-3, 9, np.uint16)
    qmap = ring_qmap(32, 32, 7)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), 32 * 32, 7)
    S = torch.empty((7, 77), dtype=torch.int64, device=dev)
    X.xpcs_ring_sums(ctx, rings, torch.from_numpy(frames).to(dev), 77, S)
    assert np.array_equal(S.cpu().numpy(), O.ring_sums(frames, qmap, 7))
    assert np.array_equal(rings.sizes(), O.ring_sizes(qmap, 7))


def test_g2_over_stored_twotime(X, ctx):
    torch, dev = torch_cuda()
    frames = speckle_counts(32, 32, 333, 0.4, 1e-3, 21, np.uint8)
    frames[[2, 40]] = 0
    qmap = ring_qmap(32, 32, 3)
    out = run_raw(X, ctx, frames, qmap, 3, want_N=False)
    C = torch.from_numpy(out["C"]).to(dev)
    g2 = torch.empty((3, 333), dtype=torch.float64, device=dev)
    cnt = torch.empty((3, 333), dtype=torch.int64, device=dev)
    X.xpcs_g2(ctx, C, 3, 333, g2, cnt)
    for q in range(3):
        Cq = out["C"][q].astype(np.float64)
        Cq = np.tril(Cq) + np.tril(Cq, -1).T  # the oracle reads a full matrix
        g_ref, c_ref = O.g2_from_twotime(Cq)
        np.testing.assert_array_equal(cnt[q].cpu().numpy(), c_ref)
        g = g2[q].cpu().numpy()
        ok = ~np.isnan(g_ref)
        np.testing.assert_allclose(g[ok], g_ref[ok], rtol=1e-6)


# ---------------------------------------------------------------- the 2^24 bound at its edge
# The raw path promises a bit-exact integer Gram for any ring whose largest per-frame sum
# of squared counts is below 2^24: the f32 accumulator then holds every partial sum of
# N(t1, t2) exactly (all terms are non-negative integers bounded by sqrt(N(t1,t1) N(t2,t2))).
# These cases fill the f32 significand: a frame with 255 pixels at 256 and 65535 pixels
# at 1 has sum of squares 2^24 - 1, so N(t, t) needs all 24 bits, reached by large
# products followed by tens of thousands of unit ones.  A tensor-core adder that kept
# fewer than 24 bits, or dropped small addends next to a large running sum, would lose
# them.

_BIG = 255                    # pixels at count 256: 255 * 2^16 = 2^24 - 2^16
_ONES = (1 << 16) - 1         # pixels at count 1: fills the rest up to 2^24 - 1
_R0 = _BIG + _ONES            # ring 0: 65790 pixels
_R1 = 2050                    # ring 1: mixed magnitudes
_M = _R0 + _R1                # 67840 = 64 x 1060


def _edge_frames(T, seed):
    rng = np.random.default_rng(seed)
    F = np.zeros((T, _M), dtype=np.uint16)
    for t in range(T):
        kind = t % 7
        r0 = F[t, :_R0]
        if kind == 0:    # large products first, then the unit ones: sum of squares 2^24 - 1
            r0[:_BIG] = 256
            r0[_BIG:] = 1
        elif kind == 1:  # unit ones first, large ones last in the ring's pixel order
            r0[:_ONES] = 1
            r0[_ONES:] = 256
        elif kind == 2:  # large ones only: 2^24 - 2^16
            r0[:_BIG] = 256
        elif kind == 3:  # large ones scattered, small counts 1..3 elsewhere
            r0[:] = rng.integers(1, 4, size=_R0)
            big = rng.choice(_R0, size=200, replace=False)
            r0[big] = 256
        elif kind == 4:  # large ones in the last 64-wide chunk positions of the ring
            r0[_R0 - 128:_R0 - 128 + _BIG // 2] = 256
            r0[:30000] = rng.integers(0, 3, size=30000)
        elif kind == 5:  # sparse small counts
            r0[:] = (rng.random(_R0) < 0.3) * rng.integers(1, 4, size=_R0)
        # kind 6: dark in ring 0 (undefined pairs)
        r1 = F[t, _R0:]
        nb = int(rng.integers(0, 251))         # a few pixels at 256, the rest 1..3
        r1[:] = rng.integers(1, 4, size=_R1)
        if nb:
            r1[rng.choice(_R1, size=nb, replace=False)] = 256
    return F


def _edge_qmap():
    q = np.zeros(_M, dtype=np.int32)
    q[_R0:] = 1
    return q


def test_raw_exact_at_sum_of_squares_edge(X, ctx):
    T = 140  # two tile rows, the second ragged
    frames = _edge_frames(T, 24)
    S2 = (frames[:, :_R0].astype(np.int64) ** 2).sum(1)
    assert S2.max() == (1 << 24) - 1  # the largest value the bound admits is reached
    S2b = (frames[:, _R0:].astype(np.int64) ** 2).sum(1)
    assert S2b.max() < (1 << 24)
    out = _check_raw(X, ctx, frames, _edge_qmap(), 2)
    # the diagonal of the frames at the edge needs all 24 bits of the f32 significand
    assert out["N"][0, 0, 0] == (1 << 24) - 1 and out["N"][0, 1, 1] == (1 << 24) - 1


def test_raw_exact_edge_reversed_pixel_order(X, ctx):
    # the same frames with the pixel order of each ring reversed: the small terms now come
    # first in the chunk order and the large ones last
    T = 140
    frames = _edge_frames(T, 25)
    frames = np.concatenate([frames[:, :_R0][:, ::-1], frames[:, _R0:][:, ::-1]], axis=1).copy()
    _check_raw(X, ctx, frames, _edge_qmap(), 2)


def test_raw_rejects_sum_of_squares_at_two_to_24(X, ctx):
    # one frame of ring 0 with 256 pixels at 256: sum of squares exactly 2^24
    frames = np.zeros((9, 512), dtype=np.uint16)
    frames[:, :64] = 1
    frames[4, 100:356] = 256
    qmap = np.zeros(512, dtype=np.int32)
    qmap[400:] = 1
    with pytest.raises(X.XpcsError) as e:
        run_raw(X, ctx, frames, qmap, 2)
    assert e.value.status == X.XPCS_ERANGE
    # one count less is inside the bound and exact
    frames[4, 100] = 255
    _check_raw(X, ctx, frames, qmap, 2)
