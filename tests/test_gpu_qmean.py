"""GPU parity of the exact ring sums option (XPCS_QMEAN_EXACT_RAW) against the oracle.

With this option the denominators of Eq. 1 on the compressed path are the exact ring sums
of the raw frames, captured when the frames are encoded, instead of a_t s_q.  Reference:
the oracle's compressed_twotime_exact_sums (and twotime_eq12 over the same sums for the
Eq. 12 normalisation) from the same FP64 basis and coefficients.  Tolerances are those of
the default compressed path per precision; the exact sums themselves are bit-exact.  A
stream opened with the option is checked against the windowed g2 of the same definition
(1e-4 of max|g2|, counts exact).
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import lower, rel_errors, torch_cuda

pytestmark = pytest.mark.gpu

TOL = {"fp16": 1e-3, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def _lossy_case(X, ctx, T=260, H=32, W=32, n_q=5, k=24, seed=20356091):
    torch, dev = torch_cuda()
    frames = speckle_counts(H, W, T + 200, 0.4, 2e-3, seed, np.uint16)
    B, _ = O.fit_basis(frames[:200], k)
    Xs = frames[200:].copy()
    Xs[[0, 77 % T]] = 0  # dark frames: S = 0, undefined pairs
    qmap = ring_qmap(H, W, n_q)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    return Xs, B, qmap, n_q, rings, basis


def test_encode_sums_gives_the_exact_ring_sums_and_the_same_coefficients(X, ctx):
    torch, dev = torch_cuda()
    Xs, B, qmap, n_q, rings, basis = _lossy_case(X, ctx)
    T, k = Xs.shape[0], B.shape[1]
    Xd = torch.from_numpy(Xs).to(dev)
    A1 = torch.empty((T, k), dtype=torch.float32, device=dev)
    A2 = torch.empty_like(A1)
    S = torch.full((n_q, T), -1, dtype=torch.int64, device=dev)
    X.xpcs_encode_sums(ctx, basis, Xd, T, A1, S)
    X.xpcs_encode(ctx, basis, Xd, T, A2)
    assert np.array_equal(S.cpu().numpy(), O.ring_sums(Xs, qmap, n_q))
    assert torch.equal(A1, A2)


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
@pytest.mark.parametrize("norm", ["mean", "eq12"])
def test_exact_ring_sums_lossy_basis(X, ctx, prec, norm):
    torch, dev = torch_cuda()
    Xs, B, qmap, n_q, rings, basis = _lossy_case(X, ctx, seed=20356092)
    T = Xs.shape[0]
    A = O.encode(Xs, B).astype(np.float32).astype(np.float64)  # the GPU consumes float32 A
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    S = O.ring_sums(Xs, qmap, n_q)
    if norm == "mean":
        Cref = O.compressed_twotime_exact_sums(A, G, S, Mq)
    else:
        Cref = np.array([O.twotime_eq12(O.compressed_ring_gram(A, G[q]), S[q], Mq[q]) for q in range(n_q)])
    Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).to(dev)
    Sd = torch.from_numpy(S).to(dev)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime_opts(ctx, basis, Ad, T, prec, norm, "exact_raw", S_raw=Sd, C_out=C, g2_out=g2, count_out=cnt)
    Ch = C.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(lower(Ch)), np.isnan(lower(Cref)))
    rm, _ = rel_errors(lower(Ch), lower(Cref))
    assert rm < TOL[prec], rm
    gh, ch = g2.cpu().numpy(), cnt.cpu().numpy()
    for q in range(n_q):
        g_ref, c_ref = O.g2_from_twotime(Cref[q])
        np.testing.assert_array_equal(ch[q], c_ref)
        gm, _ = rel_errors(gh[q], g_ref)
        assert gm < TOL[prec], (q, gm)


def test_exact_ring_sums_with_a_lossless_basis_reproduce_the_raw_path(X, ctx):
    # B = I: coefficients are the counts, and the exact ring sums are those of the raw path
    torch, dev = torch_cuda()
    H = W = 12
    n_q, T = 3, 150
    Xs = speckle_counts(H, W, T, 0.8, 2e-3, 20356093, np.uint16)
    Xs[[3, 90]] = 0
    qmap = ring_qmap(H, W, n_q)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(ctx, rings, np.eye(H * W))
    Xd = torch.from_numpy(Xs).to(dev)
    A = torch.empty((T, H * W), dtype=torch.float32, device=dev)
    S = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_encode_sums(ctx, basis, Xd, T, A, S)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    X.xpcs_twotime_opts(ctx, basis, A, T, "bf16x3", "mean", "exact_raw", S_raw=S, C_out=C)
    Craw = O.raw_twotime(Xs, qmap, n_q)[0]
    Ch = C.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(lower(Ch)), np.isnan(lower(Craw)))
    rm, _ = rel_errors(lower(Ch), lower(Craw))
    assert rm < 1e-4, rm


def test_exact_ring_sums_option_checks(X, ctx):
    torch, dev = torch_cuda()
    Xs, B, qmap, n_q, rings, basis = _lossy_case(X, ctx, T=64)
    T, k = Xs.shape[0], B.shape[1]
    Ad = torch.from_numpy(O.encode(Xs, B).astype(np.float32)).to(dev)
    Sd = torch.from_numpy(O.ring_sums(Xs, qmap, n_q)).to(dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    with pytest.raises(X.XpcsError) as e:  # the exact sums are required
        X.xpcs_twotime_opts(ctx, basis, Ad, T, "fp16", "mean", "exact_raw", S_raw=None, g2_out=g2)
    assert e.value.status == X.XPCS_EINVAL
    with pytest.raises(X.XpcsError) as e:  # the Frobenius rows use no ring sums
        X.xpcs_twotime_opts(ctx, basis, Ad, T, "fp16", "frob", "exact_raw", S_raw=Sd, g2_out=g2)
    assert e.value.status == X.XPCS_EINVAL
    with pytest.raises(X.XpcsError) as e:
        X.xpcs_twotime_opts(ctx, basis, Ad, T, "fp16", "mean", 2, S_raw=Sd, g2_out=g2)
    assert e.value.status == X.XPCS_EINVAL
    # the default ring sums ignore S_raw
    X.xpcs_twotime_opts(ctx, basis, Ad, T, "fp16", "mean", "compressed", S_raw=None, g2_out=g2)


@pytest.mark.parametrize("sizes", [(1, 3, 8), (64, 13)])
def test_stream_with_exact_ring_sums(X, ctx, sizes):
    Xs, B, qmap, n_q, rings, basis = _lossy_case(X, ctx, T=200, H=24, W=40, n_q=4, k=20, seed=20356094)
    T, Wl = Xs.shape[0], 60
    st = X.Stream(ctx, basis, Wl, 64, dtype="uint16", qmean="exact_raw")
    i, j = 0, 0
    ticket = 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    g2, cnt = st.read_g2()
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    C = O.compressed_twotime_exact_sums(O.encode(Xs, B), G, O.ring_sums(Xs, qmap, n_q), Mq)
    for q in range(n_q):
        g_ref, c_ref = O.windowed_g2(C[q], Wl)
        np.testing.assert_array_equal(cnt[q], c_ref[:Wl])
        rm, _ = rel_errors(g2[q], g_ref[:Wl])
        assert rm < 1e-4, (q, rm)
    st.close()
