"""Parity of every two-time kernel configuration against the oracle.

The two-time kernel runs in one of two schedules (single tiles, one N = 128 MMA per tile,
or tile pairs: one N = 256 MMA for tiles (I, J) and (I, J + 1)),
with a caller-chosen number of tiles per work item, and, for compressed g2-only calls,
with all tiles of a work item accumulated into one accumulator.  Each configuration is
forced with xpcs_twotime_config and checked against the oracle: the raw integer Gram
bit-exact, C and g2 within the tolerances of the raw and compressed parity tests, pair
counts exact.  Frame counts give odd and even numbers of 128-frame tile blocks, so the
last tile pair of a row is cut in half, and single-tile work items occur.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, rel_errors, run_raw, torch_cuda

pytestmark = pytest.mark.gpu

CONFIGS = [(8, "tiles"), (1, "tiles"), (8, "tile_pairs"), (1, "tile_pairs"), (3, "tile_pairs"),
           (16, "tile_pairs"), (4, "tiles"), (5, "tiles")]
TOL = {"fp16": 1e-3, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    c = X.Context(0)
    yield c
    c.twotime_config(0)


@pytest.mark.parametrize("T", [129, 300, 777])
def test_raw_every_schedule(X, ctx, T):
    frames = speckle_counts(24, 32, T, 0.7, 2e-3, 20356070 + T, np.uint8)
    frames[[3, T // 2]] = 0  # undefined frames
    n_q = 4
    qmap = ring_qmap(24, 32, n_q)
    Cref, Nref, _, _ = O.raw_twotime(frames, qmap, n_q)
    refs = [O.g2_from_twotime(Cref[q]) for q in range(n_q)]
    for tiles, sched in CONFIGS:
        ctx.twotime_config(tiles, sched)
        out = run_raw(X, ctx, frames, qmap, n_q)
        assert np.array_equal(lower(out["N"]), lower(Nref)), (tiles, sched)
        Cu, Cr = lower(out["C"]), lower(Cref)
        np.testing.assert_array_equal(np.isnan(Cu), np.isnan(Cr))
        ok = ~np.isnan(Cr)
        np.testing.assert_allclose(Cu[ok], Cr[ok], rtol=1e-6, atol=0)
        for q in range(n_q):
            g_ref, c_ref = refs[q]
            np.testing.assert_array_equal(out["count"][q], c_ref)
            okg = ~np.isnan(g_ref)
            assert np.array_equal(np.isnan(out["g2"][q]), np.isnan(g_ref))
            np.testing.assert_allclose(out["g2"][q][okg], g_ref[okg], rtol=2e-6, atol=0)
    ctx.twotime_config(0)


def _compressed_case(T, seed, n_q=5, k=40):
    H = W = 32
    frames = speckle_counts(H, W, T + 150, 0.6, 2e-3, seed, np.uint16)
    B, _ = O.fit_basis(frames[:150], k)
    Xs = frames[150:].copy()
    Xs[[0, T - 1]] = 0  # dark frames: S~ = 0, undefined pairs
    qmap = ring_qmap(H, W, n_q)
    A = O.encode(Xs, B).astype(np.float32).astype(np.float64)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cref, _ = O.compressed_twotime(A, G, s, Mq)
    return B, A, qmap, n_q, Cref


@pytest.mark.parametrize("T,prec", [(129, "bf16x3"), (300, "fp16"), (777, "bf16x3"), (777, "fp16")])
def test_compressed_every_schedule_with_and_without_C(X, ctx, T, prec):
    torch, dev = torch_cuda()
    B, A, qmap, n_q, Cref = _compressed_case(T, 20356080 + T)
    M = B.shape[0]
    refs = [O.g2_from_twotime(Cref[q]) for q in range(n_q)]
    rings = X.Rings(ctx, torch.from_numpy(qmap.astype(np.int32)).to(dev), M, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).to(dev)
    C = torch.empty((n_q, T, T), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    for tiles, sched in CONFIGS:
        ctx.twotime_config(tiles, sched)
        for with_C in (True, False):  # without C: the g2-only form, one diagonal pass per item
            C.fill_(float("nan"))
            g2.fill_(0.0)
            X.xpcs_twotime(ctx, basis, Ad, T, prec, C_out=C if with_C else None, g2_out=g2, count_out=cnt)
            if with_C:
                rm, _ = rel_errors(lower(C.cpu().numpy()), lower(Cref))
                assert rm < TOL[prec], (tiles, sched, rm)
            gh, ch = g2.cpu().numpy(), cnt.cpu().numpy()
            for q in range(n_q):
                g_ref, c_ref = refs[q]
                np.testing.assert_array_equal(ch[q], c_ref)
                gm, _ = rel_errors(gh[q], g_ref)
                assert gm < TOL[prec], (tiles, sched, with_C, q, gm)
    ctx.twotime_config(0)


def test_config_rejects_out_of_range(X, ctx):
    for tiles, sched in ((-1, 0), (65, 0), (8, 3), (8, -1)):
        with pytest.raises(X.XpcsError) as e:
            ctx.twotime_config(tiles, sched)
        assert e.value.status == X.XPCS_EINVAL
