"""GPU parity of the compressed path (Eq. 7-10 with per-ring factors) against the oracle.

Reference: the FP64 oracle of the compressed computation from the same FP64 basis and
coefficients, so the tensor-core input rounding counts as error.  Error metric over
defined pairs: rel_max = max|dC| / max|C_ref| (same for g2).  Bounds per precision mode,
derived from the operand unit roundoff u (each C entry is a k-term dot product of two
rounded operands, |error| <~ 2u |C| plus accumulation): fp16 u = 2^-11 -> 1e-3, bf16
u = 2^-8 -> 1e-2, bf16x3 (hi/lo split, dropped lo*lo term ~ u^2) -> 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, rel_errors, torch_cuda

pytestmark = pytest.mark.gpu

TOL = {"fp16": 1e-3, "bf16": 1e-2, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def run_compressed(X, ctx, B, A, qmap, n_q, prec, want_C=True):
    torch, dev = torch_cuda()
    T = A.shape[0]
    M = B.shape[0]
    rings = X.Rings(ctx, torch.from_numpy(qmap.astype(np.int32)).to(dev), M, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).to(dev)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev) if want_C else None
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime(ctx, basis, Ad, T, prec, C_out=C, g2_out=g2, count_out=cnt)
    out = dict(g2=g2.cpu().numpy(), count=cnt.cpu().numpy(), basis=basis, rings=rings)
    if want_C:
        out["C"] = C.cpu().numpy()
    return out


def _check(out, Cref, n_q, prec):
    rm, rr = rel_errors(lower(out["C"]), lower(Cref))
    assert rm < TOL[prec], (prec, rm, rr)
    for q in range(n_q):
        g_ref, c_ref = O.g2_from_twotime(Cref[q])
        np.testing.assert_array_equal(out["count"][q], c_ref)
        gm, _ = rel_errors(out["g2"][q], g_ref)
        assert gm < TOL[prec], (prec, q, gm)
    return rm


@pytest.mark.parametrize("prec", ["fp16", "bf16", "bf16x3"])
def test_compressed_lossy_basis(X, ctx, prec):
    # lossy online-style setting: basis fit on earlier frames, k = 24 < rank
    H = W = 40
    n_q, k, T = 6, 24, 300
    frames = speckle_counts(H, W, T + 200, 0.5, 2e-3, 20356002, np.uint16)
    B, _ = O.fit_basis(frames[:200], k)
    Xs = frames[200:]
    qmap = ring_qmap(H, W, n_q)
    A = O.encode(Xs, B).astype(np.float32).astype(np.float64)  # the GPU consumes float32 A
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cref, _ = O.compressed_twotime(A, G, s, Mq)
    out = run_compressed(X, ctx, B, A, qmap, n_q, prec)
    _check(out, Cref, n_q, prec)
    # ring factors computed on the device match the oracle's
    _, Gd, sd = out["basis"].export()
    np.testing.assert_allclose(Gd, G, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(sd, s, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
def test_identity_basis_equals_raw(X, ctx, prec):
    # Eq. 11: with a full basis (B = I) the compressed correlation is the raw one
    H, W, n_q, T = 16, 16, 4, 200
    frames = speckle_counts(H, W, T, 1.0, 3e-3, 4, np.uint8)
    qmap = ring_qmap(H, W, n_q)
    B = np.eye(H * W)
    A = frames.astype(np.float64)
    Craw = O.raw_twotime(frames, qmap, n_q)[0]
    out = run_compressed(X, ctx, B, A, qmap, n_q, prec)
    _check(out, Craw, n_q, prec)


@pytest.mark.parametrize("T", [1, 100, 257])
def test_compressed_ragged_T_and_k(X, ctx, T):
    H, W, n_q, k = 20, 20, 3, 70  # k not a multiple of 64: padded K
    frames = speckle_counts(H, W, T + 150, 1.0, 2e-3, 33 + T, np.uint8)
    B, _ = O.fit_basis(frames[:150], k)
    A = O.encode(frames[150:], B).astype(np.float32).astype(np.float64)
    qmap = ring_qmap(H, W, n_q)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cref, _ = O.compressed_twotime(A, G, s, Mq)
    out = run_compressed(X, ctx, B, A, qmap, n_q, "bf16x3")
    _check(out, Cref, n_q, "bf16x3")


def test_compressed_undefined_frames(X, ctx):
    # lossy ring sums can be <= 0: those pairs are NaN and excluded from g2
    H, W, n_q, k, T = 16, 16, 4, 8, 180
    frames = speckle_counts(H, W, T + 100, 0.2, 2e-3, 77, np.uint8)
    B, _ = O.fit_basis(frames[:100], k)
    A = O.encode(frames[100:], B)
    A[[3, 90]] = 0.0
    A[50] = -A[50]
    A = A.astype(np.float32).astype(np.float64)
    qmap = ring_qmap(H, W, n_q)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cref, St = O.compressed_twotime(A, G, s, Mq)
    assert (St <= 0).any()
    out = run_compressed(X, ctx, B, A, qmap, n_q, "bf16x3")
    np.testing.assert_array_equal(np.isnan(lower(out["C"])), np.isnan(lower(Cref)))
    _check(out, Cref, n_q, "bf16x3")


def test_grouped_sector_masks_uneven_sizes(X, ctx):
    # ring-plus-sector masks with log-spaced, uneven pixel counts (20 .. 1500 px, 16
    # masks, pixels outside every mask unused), all in one launch: the compressed path
    # against the FP64 oracle, and the exact raw path's integer Gram bit for bit
    from synth import sector_qmap
    from tests.gpu_util import run_raw

    H, W, T, k = 96, 96, 300, 40
    qmap = sector_qmap(H, W, n_annuli=4, n_sectors=4, min_px=20, max_px=1500, seed=7)
    n_q = int(qmap.max()) + 1
    assert n_q == 16 and (qmap < 0).any()
    frames = speckle_counts(H, W, T + 200, 0.5, 2e-3, 20356003, np.uint16)
    B, _ = O.fit_basis(frames[:200], k)
    Xs = frames[200:]
    A = O.encode(Xs, B).astype(np.float32).astype(np.float64)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cref, _ = O.compressed_twotime(A, G, s, Mq)
    out = run_compressed(X, ctx, B, A, qmap, n_q, "bf16x3")
    _check(out, Cref, n_q, "bf16x3")
    raw = run_raw(X, ctx, Xs, qmap, n_q)
    for q in range(n_q):
        Nref = O.raw_gram(Xs, qmap, q)
        assert np.array_equal(lower(raw["N"][q]), lower(Nref)), q
