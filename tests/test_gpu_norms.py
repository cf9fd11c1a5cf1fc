"""GPU parity of the two other normalisations of the two-time correlation.

* Frobenius rows (Eq. 2 with the rows of the data normalised by their Frobenius norm,
  Sec. 2.1): C = N(t1,t2) / sqrt(N(t1,t1) N(t2,t2)), the cosine similarity of a ring's
  frames; frames with N(t,t) = 0 are undefined.
* Literal Eq. 12: C = M_q N(t1,t2) / Sbar^2 with Sbar the ring sum averaged over all
  frames, so the diagonal means are <I(t) I(t+tau)> / <I>^2 over frames and ring pixels;
  every pair counts.

Raw path: the integer Gram is exact and the scales are FP64 rounded to f32, so C agrees
with the oracle to f32 rounding (bound 1e-6) and the pair counts exactly.  Compressed
path: the oracle's FP64 basis and coefficients are imported, bounds per precision as in
the other compressed tests (fp16 1e-3, bf16x3 1e-4).
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


def _outputs(torch, dev, n_q, T):
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    return C, g2, cnt


def _compare(C, g2, cnt, Cref, tol, n_q):
    Ch = C.cpu().numpy()
    assert np.array_equal(np.isnan(lower(Ch)), np.isnan(lower(Cref)))
    rm, rr = rel_errors(lower(Ch), lower(Cref))
    assert rm < tol, (rm, rr)
    g2h, ch = g2.cpu().numpy(), cnt.cpu().numpy()
    for q in range(n_q):
        g_ref, c_ref = O.g2_from_twotime(Cref[q])
        np.testing.assert_array_equal(ch[q], c_ref)
        gm, _ = rel_errors(g2h[q], g_ref)
        assert gm < tol, (q, gm)


@pytest.fixture(scope="module")
def raw_case():
    H = W = 24
    n_q, T = 5, 300  # three tiles with a ragged tail
    frames = speckle_counts(H, W, T, 0.3, 2e-3, 20356021, np.uint16)
    qmap = ring_qmap(H, W, n_q)
    frames[[5, 140, 299]] = 0  # dark frames: undefined under both Eq. 1 and Frobenius rows
    N = np.stack([O.raw_gram(frames, qmap, q) for q in range(n_q)])
    S = O.ring_sums(frames, qmap, n_q)
    Mq = O.ring_sizes(qmap, n_q)
    return dict(frames=frames, qmap=qmap, n_q=n_q, T=T, N=N, S=S, Mq=Mq)


def _run_raw(X, ctx, case, norm):
    torch, dev = torch_cuda()
    n_q, T = case["n_q"], case["T"]
    rings = X.Rings(ctx, torch.from_numpy(case["qmap"]).to(dev), case["qmap"].size, n_q)
    C, g2, cnt = _outputs(torch, dev, n_q, T)
    Nd = torch.zeros((n_q, T, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime_raw_norm(ctx, rings, torch.from_numpy(case["frames"]).to(dev), T, norm, C_out=C, N_out=Nd,
                            g2_out=g2, count_out=cnt)
    np.testing.assert_array_equal(lower(Nd.cpu().numpy()), lower(case["N"]))  # exact in every mode
    return C, g2, cnt


def test_raw_frobenius_rows(X, ctx, raw_case):
    C, g2, cnt = _run_raw(X, ctx, raw_case, "frob")
    Cref = np.stack([O.frobenius_twotime(raw_case["N"][q]) for q in range(raw_case["n_q"])])
    _compare(C, g2, cnt, Cref, 1e-6, raw_case["n_q"])


def test_raw_literal_eq12(X, ctx, raw_case):
    C, g2, cnt = _run_raw(X, ctx, raw_case, "eq12")
    n_q, T = raw_case["n_q"], raw_case["T"]
    Cref = np.stack([O.twotime_eq12(raw_case["N"][q], raw_case["S"][q], raw_case["Mq"][q]) for q in range(n_q)])
    _compare(C, g2, cnt, Cref, 1e-6, n_q)
    np.testing.assert_array_equal(cnt.cpu().numpy(), np.broadcast_to(T - np.arange(T), (n_q, T)))
    g2h = g2.cpu().numpy()
    for q in (0, n_q - 1):  # against the pixel-level definition as well
        for tau in (1, 128, 250):
            ref = O.g2_eq12(raw_case["frames"], raw_case["qmap"], q, tau)
            assert abs(g2h[q, tau] - ref) <= 1e-6 * abs(ref), (q, tau)


@pytest.fixture(scope="module")
def comp_case():
    H = W = 40
    n_q, k, T = 6, 40, 280
    frames = speckle_counts(H, W, T + 200, 0.5, 2e-3, 20356022, np.uint16)
    B, _ = O.fit_basis(frames[:200], k)
    qmap = ring_qmap(H, W, n_q)
    A = O.encode(frames[200:], B).astype(np.float32).astype(np.float64)  # the GPU consumes float32 A
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    return dict(B=B, A=A, qmap=qmap, n_q=n_q, T=T, G=G, s=s, Mq=Mq)


def _run_comp(X, ctx, case, prec, norm):
    torch, dev = torch_cuda()
    n_q, T = case["n_q"], case["T"]
    rings = X.Rings(ctx, torch.from_numpy(case["qmap"]).to(dev), case["qmap"].size, n_q)
    basis = X.xpcs_basis_import(ctx, rings, case["B"])
    Ad = torch.from_numpy(np.ascontiguousarray(case["A"], dtype=np.float32)).to(dev)
    C, g2, cnt = _outputs(torch, dev, n_q, T)
    X.xpcs_twotime_norm(ctx, basis, Ad, T, prec, norm, C_out=C, g2_out=g2, count_out=cnt)
    return C, g2, cnt


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
def test_compressed_frobenius_rows(X, ctx, comp_case, prec):
    A, G = comp_case["A"], comp_case["G"]
    Cref = np.stack([O.frobenius_twotime(O.compressed_ring_gram(A, G[q])) for q in range(comp_case["n_q"])])
    C, g2, cnt = _run_comp(X, ctx, comp_case, prec, "frob")
    _compare(C, g2, cnt, Cref, TOL[prec], comp_case["n_q"])


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
def test_compressed_literal_eq12(X, ctx, comp_case, prec):
    A, G, s, Mq = comp_case["A"], comp_case["G"], comp_case["s"], comp_case["Mq"]
    Cref = np.stack([O.twotime_eq12(O.compressed_ring_gram(A, G[q]), A @ s[q], Mq[q])
                     for q in range(comp_case["n_q"])])
    C, g2, cnt = _run_comp(X, ctx, comp_case, prec, "eq12")
    _compare(C, g2, cnt, Cref, TOL[prec], comp_case["n_q"])


def test_bad_normalisation_is_rejected(X, ctx, comp_case):
    with pytest.raises(X.XpcsError) as e:
        _run_comp(X, ctx, comp_case, "bf16x3", 3)
    assert e.value.status == X.XPCS_EINVAL
