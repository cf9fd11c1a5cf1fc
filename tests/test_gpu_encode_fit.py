"""GPU parity of the encode (Eq. 7) and the basis fit (Eq. 3-6) against the oracle.

Encode: counts up to 1023 are exact in f16, the basis enters as a scaled hi/lo f16 pair
(about 2^-22 relative per element) and the products accumulate in f32, so A matches the
FP64 oracle to 1e-4 of max|A|.  Fit: both sides eigendecompose the same FP64 Gram (LAPACK on the
host, cuSOLVER on the device); singular values agree to 1e-9 and, after the sign
convention, basis columns to 1e-7.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, rel_errors, run_raw, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def _rings(X, ctx, qmap, n_q):
    torch, dev = torch_cuda()
    return X.Rings(ctx, torch.from_numpy(qmap.astype(np.int32)).to(dev), qmap.size, n_q)


@pytest.mark.parametrize("dtype,k,T", [(np.uint16, 64, 300), (np.uint8, 24, 129), (np.uint16, 70, 77),
                                       (np.uint8, 128, 256), (np.uint16, 256, 140)])
def test_encode_matches_oracle(X, ctx, dtype, k, T):
    torch, dev = torch_cuda()
    H, W, n_q = 32, 40, 5
    frames = speckle_counts(H, W, T + 300, 0.7, 2e-3, 1000 + k, dtype)
    B, _ = O.fit_basis(frames[:300], k)
    qmap = ring_qmap(H, W, n_q)
    rings = _rings(X, ctx, qmap, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    Xs = np.ascontiguousarray(frames[300:])
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, torch.from_numpy(Xs).to(dev), T, A)
    Aref = O.encode(Xs, B)
    rm, rr = rel_errors(A.cpu().numpy().astype(np.float64), Aref)
    assert rm < 1e-4 and rr < 1e-4, (rm, rr)


def test_encode_rejects_counts_above_exact_range(X, ctx):
    torch, dev = torch_cuda()
    M, k, T = 64, 8, 20
    rng = np.random.default_rng(0)
    B, _ = np.linalg.qr(rng.standard_normal((M, k)))
    rings = _rings(X, ctx, np.zeros(M, dtype=np.int32), 1)
    basis = X.xpcs_basis_import(ctx, rings, B)
    frames = np.zeros((T, M), dtype=np.uint16)
    frames[4, 9] = 2000  # counts up to 1023 are exact in the f16 encode
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    with pytest.raises(X.XpcsError) as e:
        X.xpcs_encode(ctx, basis, torch.from_numpy(frames).to(dev), T, A)
    assert e.value.status == X.XPCS_ERANGE


def _align_signs(B, Bref):
    sgn = np.sign((B * Bref).sum(axis=0))
    sgn[sgn == 0] = 1
    return B * sgn


@pytest.mark.parametrize("dtype,n_fit,k", [(np.uint16, 200, 32), (np.uint8, 150, 64)])
def test_fit_basis_matches_oracle(X, ctx, dtype, n_fit, k):
    torch, dev = torch_cuda()
    H, W, n_q = 32, 32, 4
    frames = speckle_counts(H, W, n_fit, 1.0, 2e-3, 77 + k, dtype)
    frames[7] = 0  # a dark frame is dropped by the fit
    qmap = ring_qmap(H, W, n_q)
    rings = _rings(X, ctx, qmap, n_q)
    sig = np.empty(n_fit)
    basis = X.xpcs_fit_basis(ctx, rings, torch.from_numpy(frames).to(dev), n_fit, k, sigma_host=sig)
    Bref, sref = O.fit_basis(frames, k)
    np.testing.assert_allclose(sig[: len(sref)][:k], sref[:k], rtol=1e-9)
    Bd, Gd, sd = basis.export()
    np.testing.assert_allclose(Bd.T @ Bd, np.eye(k), atol=1e-10)
    Ba = _align_signs(Bd, Bref)
    np.testing.assert_allclose(Ba, Bref, atol=1e-7)
    Gref, s_ref, _ = O.ring_factors(Ba, qmap, n_q)
    Gd2, sd2, _ = O.ring_factors(Bd, qmap, n_q)
    np.testing.assert_allclose(Gd, Gd2, atol=1e-12)
    np.testing.assert_allclose(sd, sd2, atol=1e-12)


def test_spectrum_rank_rule_matches_oracle(X, ctx):
    # Sec. 3.1 rank choice (values >= 2x the smallest) on the device fit's spectrum equals
    # the same rule on the oracle's own fit of the same frames
    torch, dev = torch_cuda()
    H, W, n_q, n_fit = 40, 40, 5, 300
    frames = speckle_counts(H, W, n_fit, 0.5, 1e-3, 20356005, np.uint16)
    rings = _rings(X, ctx, ring_qmap(H, W, n_q), n_q)
    sig = np.empty(n_fit)
    X.xpcs_fit_basis(ctx, rings, torch.from_numpy(frames).to(dev), n_fit, 8, sigma_host=sig)
    _, sref = O.fit_basis(frames, 8)
    K = X.xpcs_rank_from_spectrum(sig)
    assert K == O.rank_from_spectrum(sref)
    assert 1 <= K < n_fit


def test_fit_on_calibration_run_then_another_series(X, ctx):
    # online variant (Sec. 2.3): the basis comes from an earlier run on the same sample and
    # every frame of the new series is encoded with it; compared with the oracle doing the
    # same (its own fit of the calibration run, encode of the new series)
    torch, dev = torch_cuda()
    H = W = 40
    n_q, k, T, n_fit = 6, 32, 300, 200
    calib = speckle_counts(H, W, n_fit, 0.2, 1e-3, 20356105, np.uint16)
    series = speckle_counts(H, W, T, 0.2, 1e-3, 20356005, np.uint16)
    qmap = ring_qmap(H, W, n_q)
    rings = _rings(X, ctx, qmap, n_q)
    basis = X.xpcs_fit_basis(ctx, rings, torch.from_numpy(calib).to(dev), n_fit, k)
    Xd = torch.from_numpy(series).to(dev)
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, Xd, T, A)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime(ctx, basis, A, T, "bf16x3", C_out=C, g2_out=g2, count_out=cnt)
    Bref, _ = O.fit_basis(calib, k)
    G, s, Mq = O.ring_factors(Bref, qmap, n_q)
    Cref, _ = O.compressed_twotime(O.encode(series, Bref), G, s, Mq)
    Ch = C.cpu().numpy()
    assert np.array_equal(np.isnan(lower(Ch)), np.isnan(lower(Cref)))
    rm, _ = rel_errors(lower(Ch), lower(Cref))
    assert rm < 1e-4, rm
    for q in range(n_q):
        gref, cref = O.g2_from_twotime(Cref[q])
        np.testing.assert_array_equal(cnt[q].cpu().numpy(), cref)
        gm, _ = rel_errors(g2[q].cpu().numpy(), gref)
        assert gm < 1e-4, (q, gm)


def test_fit_rejects_k_above_rank(X, ctx):
    torch, dev = torch_cuda()
    frames = np.zeros((20, 64), dtype=np.uint8)
    frames[:, :3] = np.arange(20)[:, None] % 4 + 1  # rank 1 up to dark rows
    frames[::5, 10] = 7  # rank 2
    rings = _rings(X, ctx, np.zeros(64, dtype=np.int32), 1)
    with pytest.raises(X.XpcsError) as e:
        X.xpcs_fit_basis(ctx, rings, torch.from_numpy(frames).to(dev), 20, 5)
    assert e.value.status == X.XPCS_EINVAL


def test_end_to_end_fit_encode_twotime(X, ctx):
    # offline lossy pipeline on the device: fit -> encode -> compressed two-time + g2
    torch, dev = torch_cuda()
    H = W = 48
    n_q, k, T, n_fit = 8, 48, 400, 120
    frames = speckle_counts(H, W, T, 0.2, 1e-3, 20356003, np.uint16)
    qmap = ring_qmap(H, W, n_q)
    rings = _rings(X, ctx, qmap, n_q)
    Xd = torch.from_numpy(frames).to(dev)
    basis = X.xpcs_fit_basis(ctx, rings, Xd, n_fit, k)
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, Xd, T, A)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    X.xpcs_twotime(ctx, basis, A, T, "fp16", C_out=C, g2_out=g2)
    Bref, _ = O.fit_basis(frames[:n_fit], k)
    G, s, Mq = O.ring_factors(Bref, qmap, n_q)
    Cref, _ = O.compressed_twotime(O.encode(frames, Bref), G, s, Mq)
    rm, _ = rel_errors(lower(C.cpu().numpy()), lower(Cref))
    assert rm < 1e-3, rm
    for q in range(n_q):
        gref, _ = O.g2_from_twotime(Cref[q])
        gm, _ = rel_errors(g2[q].cpu().numpy(), gref)
        assert gm < 1e-3, (q, gm)


def test_fitted_full_rank_compressed_equals_raw(X, ctx):
    # Eq. 11 on the device: offline lossless compression reproduces the raw two-time
    torch, dev = torch_cuda()
    H, W, n_q, T = 16, 16, 4, 60
    frames = speckle_counts(H, W, T, 2.0, 2e-3, 5, np.uint8)
    qmap = ring_qmap(H, W, n_q)
    r = int(np.linalg.matrix_rank(frames.astype(np.float64)))
    rings = _rings(X, ctx, qmap, n_q)
    Xd = torch.from_numpy(frames).to(dev)
    basis = X.xpcs_fit_basis(ctx, rings, Xd, T, r)
    A = torch.empty((T, r), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, Xd, T, A)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    X.xpcs_twotime(ctx, basis, A, T, "bf16x3", C_out=C)
    raw = run_raw(X, ctx, frames, qmap, n_q, want_N=False)
    rm, _ = rel_errors(lower(C.cpu().numpy()), lower(raw["C"]))
    assert rm < 1e-4, rm
