"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these retypes the oracle's formula: each compares it with a hand-derived
fixture, brute force, a closed form, an identity of the method (Eq. 8-11), an
independent library routine, or speckle statistics of known decay.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from synth import rate_of_pixels, ring_qmap, speckle_counts

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frac(v):
    return None if v is None else float(Fraction(v[0], v[1]))


# ---------------------------------------------------------------- hand-derived fixture

def test_golden_tiny_twotime():
    g = json.load(open(os.path.join(GOLD, "tiny_twotime.json")))
    X = np.array(g["X"], dtype=np.uint8)
    qmap = np.array(g["qmap"], dtype=np.int32)
    C, N, S, Mq = O.raw_twotime(X, qmap, 2)
    assert S.tolist() == g["S"]
    for q in range(2):
        for i in range(3):
            for j in range(i, 3):
                assert N[q, i, j] == g["N_upper"][q][i][j]
                want = _frac(g["C_num_den"][q][i][j])
                if want is None:
                    assert np.isnan(C[q, i, j])
                else:
                    assert C[q, i, j] == pytest.approx(want, rel=1e-15)
        g2, cnt = O.g2_from_twotime(C[q])
        assert cnt.tolist() == g["count"][q]
        for tau in range(3):
            want = _frac(g["g2_num_den"][q][tau])
            if want is None:
                assert np.isnan(g2[tau])
            else:
                assert g2[tau] == pytest.approx(want, rel=1e-15)


# ---------------------------------------------------------------- brute force

def _brute(X, qmap, n_q):
    T, M = X.shape
    out = []
    for q in range(n_q):
        pix = [p for p in range(M) if qmap[p] == q]
        S = [sum(int(X[t, p]) for p in pix) for t in range(T)]
        C = [[None] * T for _ in range(T)]
        for a in range(T):
            for b in range(T):
                n = sum(int(X[a, p]) * int(X[b, p]) for p in pix)
                C[a][b] = Fraction(len(pix) * n, S[a] * S[b]) if S[a] > 0 and S[b] > 0 else None
        g2 = []
        for tau in range(T):
            vals = [C[t][t + tau] for t in range(T - tau) if C[t][t + tau] is not None]
            g2.append((sum(vals, Fraction(0)) / len(vals)) if vals else None)
        out.append((S, C, g2))
    return out


def test_raw_path_matches_brute_force_rationals():
    rng = np.random.default_rng(5)
    T, M, n_q = 7, 13, 3
    X = rng.poisson(0.8, size=(T, M)).astype(np.uint8)
    X[3, :] = 0  # an all-dark frame: undefined pairs
    qmap = rng.integers(-1, n_q, size=M).astype(np.int32)
    C, N, S, Mq = O.raw_twotime(X, qmap, n_q)
    for q, (Sb, Cb, g2b) in enumerate(_brute(X, qmap, n_q)):
        assert S[q].tolist() == Sb
        for a in range(T):
            for b in range(T):
                if Cb[a][b] is None:
                    assert np.isnan(C[q, a, b])
                else:
                    assert C[q, a, b] == pytest.approx(float(Cb[a][b]), rel=1e-14)
        g2, _ = O.g2_from_twotime(C[q])
        for tau in range(T):
            if g2b[tau] is None:
                assert np.isnan(g2[tau])
            else:
                assert g2[tau] == pytest.approx(float(g2b[tau]), rel=1e-13)


# ---------------------------------------------------------------- closed forms and invariances

def test_constant_frames_correlate_to_one():
    # a frame constant over a ring: N = c1 c2 M, S = c M, so C = 1 exactly (Eq. 1)
    T, M, n_q = 5, 40, 4
    qmap = (np.arange(M) % n_q).astype(np.int32)
    c = np.array([1, 3, 2, 7, 5])
    X = np.repeat(c[:, None], M, axis=1).astype(np.uint8)
    C, _, _, _ = O.raw_twotime(X, qmap, n_q)
    assert np.all(C == 1.0)


def test_per_frame_scale_and_permutation():
    rng = np.random.default_rng(1)
    T, M, n_q = 9, 30, 3
    X = rng.poisson(2.0, size=(T, M)).astype(np.float64) + 1
    qmap = rng.integers(0, n_q, size=M).astype(np.int32)
    alpha = rng.uniform(0.5, 3.0, size=T)
    G, s, Mq = O.ring_factors(np.eye(M), qmap, n_q)
    C1, _ = O.compressed_twotime(X, G, s, Mq)
    C2, _ = O.compressed_twotime(alpha[:, None] * X, G, s, Mq)
    np.testing.assert_allclose(C1, C2, rtol=1e-12)  # Eq. 1 is scale-free per frame
    perm = rng.permutation(T)
    C3, _ = O.compressed_twotime(X[perm], G, s, Mq)
    np.testing.assert_allclose(C3, C1[:, perm][:, :, perm], rtol=1e-12)
    pix = rng.permutation(M)
    G4, s4, M4 = O.ring_factors(np.eye(M), qmap[pix], n_q)
    C4, _ = O.compressed_twotime(X[:, pix], G4, s4, M4)
    np.testing.assert_allclose(C4, C1, rtol=1e-12)


# ---------------------------------------------------------------- identities of the method

def _small_speckle(T=40, H=12, W=12, n_q=3, mean=1.5, seed=3):
    X = speckle_counts(H, W, T, mean, 2e-3, seed, np.uint8)
    return X, ring_qmap(H, W, n_q), n_q


def test_eq11_identity_basis_reduces_to_raw_exactly():
    # B = I_M: the coefficients are the counts themselves and every step is exact
    X, qmap, n_q = _small_speckle()
    Craw, N, S, Mq = O.raw_twotime(X, qmap, n_q)
    G, s, M2 = O.ring_factors(np.eye(X.shape[1]), qmap, n_q)
    A = O.encode(X, np.eye(X.shape[1]))
    Cc, St = O.compressed_twotime(A, G, s, M2)
    assert np.array_equal(St, S.astype(np.float64))
    np.testing.assert_array_equal(np.isnan(Cc), np.isnan(Craw))
    ok = ~np.isnan(Craw)
    np.testing.assert_allclose(Cc[ok], Craw[ok], rtol=1e-15)


def test_eq11_any_orthogonal_full_basis_is_lossless():
    X, qmap, n_q = _small_speckle()
    M = X.shape[1]
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((M, M)))
    Craw = O.raw_twotime(X, qmap, n_q)[0]
    G, s, Mq = O.ring_factors(Q, qmap, n_q)
    Cc, _ = O.compressed_twotime(O.encode(X, Q), G, s, Mq)
    ok = ~np.isnan(Craw)
    np.testing.assert_allclose(Cc[ok], Craw[ok], rtol=1e-10, atol=1e-12)


def test_fitted_basis_at_full_rank_is_lossless():
    # offline lossless compression (Sec. 3.1, Eq. 11): K = rank(X) reproduces the raw TTC
    X, qmap, n_q = _small_speckle(T=30)
    r = np.linalg.matrix_rank(X.astype(np.float64))
    B, sigma = O.fit_basis(X, r)
    Craw = O.raw_twotime(X, qmap, n_q)[0]
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    Cc, _ = O.compressed_twotime(O.encode(X, B), G, s, Mq)
    ok = ~np.isnan(Craw)
    np.testing.assert_allclose(Cc[ok], Craw[ok], rtol=1e-9, atol=1e-9)
    with pytest.raises(ValueError):
        O.fit_basis(X, r + 1)


def test_eq10_homomorphic_equals_decompress_then_correlate():
    # Eq. 8-10: the ring Gram of the decompressed frames equals a G_q a^T
    X, qmap, n_q = _small_speckle(T=30)
    B, _ = O.fit_basis(X[:20], 6)
    A = O.encode(X, B)
    Xt = O.decompress(A, B)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    for q in range(n_q):
        idx = O.ring_index(qmap, q)
        np.testing.assert_allclose(O.compressed_ring_gram(A, G[q]), Xt[:, idx] @ Xt[:, idx].T,
                                   rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(O.compressed_ring_sums(A, s)[q], Xt[:, idx].sum(axis=1),
                                   rtol=1e-10, atol=1e-10)


def test_exact_ring_sums_reduce_to_raw_with_a_lossless_basis():
    # with B = I the coefficients are the counts: the compressed Gram with the exact ring
    # sums is the raw two-time correlation, and a s_q equals the exact sums
    X, qmap, n_q = _small_speckle()
    X[[4, 17]] = 0  # dark frames: undefined pairs
    Craw, N, S, Mq = O.raw_twotime(X, qmap, n_q)
    G, s, M2 = O.ring_factors(np.eye(X.shape[1]), qmap, n_q)
    Ce = O.compressed_twotime_exact_sums(O.encode(X, np.eye(X.shape[1])), G, S, M2)
    np.testing.assert_array_equal(np.isnan(Ce), np.isnan(Craw))
    ok = ~np.isnan(Craw)
    np.testing.assert_allclose(Ce[ok], Craw[ok], rtol=1e-15)


def test_exact_ring_sums_with_a_lossy_basis_from_pixel_definitions():
    # lossy basis: numerator = ring Gram of the decompressed frames (Eq. 8), denominators =
    # the raw frames' ring sums, each summed pixel by pixel for a few pairs
    X, qmap, n_q = _small_speckle(T=30)
    X[5] = 0
    B, _ = O.fit_basis(X[:20], 5)
    A = O.encode(X, B)
    Xt = O.decompress(A, B)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    S = O.ring_sums(X, qmap, n_q)
    Ce = O.compressed_twotime_exact_sums(A, G, S, Mq)
    rng = np.random.default_rng(9)
    for q in range(n_q):
        idx = [p for p in range(X.shape[1]) if qmap[p] == q]
        for t1, t2 in list(rng.integers(0, 30, size=(12, 2))) + [(5, 3), (7, 7)]:
            num = sum(Xt[t1, p] * Xt[t2, p] for p in idx)
            s1 = sum(int(X[t1, p]) for p in idx)
            s2 = sum(int(X[t2, p]) for p in idx)
            if s1 > 0 and s2 > 0:
                assert Ce[q, t1, t2] == pytest.approx(len(idx) * num / (s1 * s2), rel=1e-10, abs=1e-12)
            else:
                assert np.isnan(Ce[q, t1, t2])
    # lossy: the exact sums differ from a s_q, so the two forms differ
    Cc, St = O.compressed_twotime(A, G, s, Mq)
    assert not np.allclose(St, S)


def test_basis_orthonormal_eckart_young_and_svd():
    X, _, _ = _small_speckle(T=50)
    k = 7
    B, sigma = O.fit_basis(X, k)
    np.testing.assert_allclose(B.T @ B, np.eye(k), atol=1e-12)
    Fn = X.astype(np.float64)
    Fn = Fn / np.sqrt((Fn * Fn).sum(1, keepdims=True))
    sv = np.linalg.svd(Fn, compute_uv=False)  # independent LAPACK routine (gesdd)
    np.testing.assert_allclose(sigma[: len(sv)], sv, rtol=1e-9, atol=1e-12)
    resid = Fn - Fn @ B @ B.T
    np.testing.assert_allclose((resid ** 2).sum(), (sv[k:] ** 2).sum(), rtol=1e-9)
    # the top right singular vectors span the same space
    _, _, Vt = np.linalg.svd(Fn, full_matrices=False)
    P1 = B @ B.T
    P2 = Vt[:k].T @ Vt[:k]
    np.testing.assert_allclose(P1, P2, atol=1e-9)


def test_per_ring_basis_has_identity_ring_factor():
    # the paper's per-q-subset compression (Sec. 2.2) is the block-diagonal special case
    rng = np.random.default_rng(4)
    M, n_q, kq = 24, 3, 4
    qmap = np.repeat(np.arange(n_q), M // n_q).astype(np.int32)
    B = np.zeros((M, n_q * kq))
    for q in range(n_q):
        Q, _ = np.linalg.qr(rng.standard_normal((M // n_q, kq)))
        B[q * (M // n_q):(q + 1) * (M // n_q), q * kq:(q + 1) * kq] = Q
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    for q in range(n_q):
        blk = G[q][q * kq:(q + 1) * kq, q * kq:(q + 1) * kq]
        np.testing.assert_allclose(blk, np.eye(kq), atol=1e-12)
        G[q][q * kq:(q + 1) * kq, q * kq:(q + 1) * kq] = 0
        assert np.abs(G[q]).max() == 0


# ---------------------------------------------------------------- speckle statistics (Eq. 13 form)

def test_speckle_g2_follows_siegert_decay():
    # one complex-Gaussian mode per pixel: g2(tau) = 1 + mean_p exp(-2 Gamma_p tau)
    H = W = 64
    T, n_q, D = 800, 8, 4e-4
    X = speckle_counts(H, W, T, 2.0, D, 12, np.uint8)
    qmap = ring_qmap(H, W, n_q)
    gam = rate_of_pixels(H, W, D)
    C, _, _, _ = O.raw_twotime(X, qmap, n_q)
    for q in (1, 2, 4, 7):
        g2, _ = O.g2_from_twotime(C[q])
        idx = O.ring_index(qmap, q)
        for tau in (1, 2, 5, 20):
            want = 1.0 + np.exp(-2 * gam[idx] * tau).mean()
            assert abs(g2[tau] - want) < 0.03 * want, (q, tau, g2[tau], want)
    # outer rings at long lags: decorrelated, g2 -> 1
    for q in range(2, n_q):
        g2, _ = O.g2_from_twotime(C[q])
        assert abs(np.nanmean(g2[100:400]) - 1.0) < 0.01


def test_literal_eq12_agrees_with_diagonal_average_on_stationary_speckle():
    H = W = 40
    X = speckle_counts(H, W, 300, 3.0, 5e-4, 13, np.uint8)
    qmap = ring_qmap(H, W, 4)
    C, _, _, _ = O.raw_twotime(X, qmap, 4)
    for q in range(4):
        g2, _ = O.g2_from_twotime(C[q])
        for tau in (1, 10, 50):
            assert abs(O.g2_eq12(X, qmap, q, tau) - g2[tau]) < 0.03 * g2[tau]


def test_frobenius_twotime_is_cosine_similarity():
    rng = np.random.default_rng(9)
    X = rng.poisson(1.0, size=(6, 20)).astype(np.uint8) + 1
    qmap = np.zeros(20, dtype=np.int32)
    Cf = O.frobenius_twotime(O.raw_gram(X, qmap, 0))
    Xf = X.astype(np.float64)
    for a in range(6):
        for b in range(6):
            cos = Xf[a] @ Xf[b] / (np.linalg.norm(Xf[a]) * np.linalg.norm(Xf[b]))
            assert Cf[a, b] == pytest.approx(cos, rel=1e-14)


def test_windowed_g2_drops_long_lags():
    X, qmap, n_q = _small_speckle(T=20)
    C = O.raw_twotime(X, qmap, n_q)[0]
    g2w, cw = O.windowed_g2(C[0], 5)
    g2, c = O.g2_from_twotime(C[0])
    np.testing.assert_array_equal(g2w[:5], g2[:5])
    assert np.all(cw[5:] == 0) and np.all(np.isnan(g2w[5:]))


# ---------------------------------------------------------------- the paper's printed numbers

def test_paper_compression_ratios_and_speedup():
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    off = g["offline_cr"]
    for K, cr in zip(off["K"], off["CR"]):
        assert O.compression_ratio_offline(off["N"], K) == cr
    on = g["online_cr"]
    for K, cr in zip(on["K"], on["CR"]):
        assert abs(O.compression_ratio_online(on["M"], K) - cr) / cr < 0.01  # printed rounded
    ls = g["lossless_speedup"]
    assert abs(O.lossless_speedup(ls["N"], ls["M"]) - ls["factor"]) / ls["factor"] < 0.01


# ---------------------------------------------------------------- rank rule of Sec. 3.1

def test_rank_rule_hand_spectra():
    # hand-counted: values >= 2 x the smallest (1.0) are 8, 4, 2.5 and 2 (equality counts)
    assert O.rank_from_spectrum([8.0, 4.0, 2.5, 2.0, 1.5, 1.0]) == 4
    assert O.rank_from_spectrum([8.0, 4.0, 2.5, 2.0, 1.5, 1.0], factor=3.0) == 2
    # a rank-deficient tail is not the minimum: the smallest kept value is 1.0
    assert O.rank_from_spectrum([3.0, 1.0, 0.0, 0.0]) == 1
    # a flat spectrum has no component that stands out
    assert O.rank_from_spectrum([1.0, 1.0, 1.0]) == 0


@pytest.mark.parametrize("seed", [0, 3])
def test_rank_rule_finds_planted_components(seed):
    # five equal-weight patterns plus white noise: after the fit's row normalisation the
    # noise singular values spread by about 1.5x (Marchenko-Pastur edges at n/M = 0.05), so
    # the rule on singular values returns the five planted components, while the same
    # rule applied to squared values (eigenvalues, spread about 2.3x) would count noise too
    rng = np.random.default_rng(seed)
    n, M, r = 60, 1200, 5
    P = np.linalg.qr(rng.standard_normal((M, r)))[0].T
    u = rng.standard_normal((n, r))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    F = 50 * u @ P + 0.5 * rng.standard_normal((n, M))
    _, s = O.fit_basis(F, r)
    assert O.rank_from_spectrum(s) == r
    assert int((s * s >= 2 * (s * s).min()).sum()) > r


def test_eq12_twotime_diagonals_equal_the_pixel_level_literal_eq12():
    # Eq. 12 two ways: diagonal means of M_q N / Sbar^2 (Gram form) against the oracle's
    # pixel-level average of I(t) I(t+tau) over frames and ring pixels divided by <I>^2
    X, qmap, n_q = _small_speckle(T=40)
    S = O.ring_sums(X, qmap, n_q)
    Mq = O.ring_sizes(qmap, n_q)
    for q in range(n_q):
        g2, cnt = O.g2_from_twotime(O.twotime_eq12(O.raw_gram(X, qmap, q), S[q], Mq[q]))
        np.testing.assert_array_equal(cnt, 40 - np.arange(40))
        for tau in (0, 1, 7, 39):
            assert abs(g2[tau] - O.g2_eq12(X, qmap, q, tau)) < 1e-12 * abs(g2[tau])


# ---------------------------------------------------------------- downstream analysis (Sec. 3)

def test_relaxation_fit_recovers_a_noiseless_eq13_curve():
    tau = np.arange(400, dtype=np.float64)
    g2 = 1.0 + 0.3 * np.exp(-2.0 * tau / 50.0)
    g2[[3, 77, 200]] = np.nan  # undefined lags are skipped
    B, C, t0, rms = O.relaxation_fit(g2, 1, 399, 1.0, 1e4)
    assert abs(B - 1.0) < 1e-7 and abs(C - 0.3) < 1e-7 and abs(t0 - 50.0) < 1e-5 and rms < 1e-8


def test_relaxation_fit_on_speckle_gives_the_decay_time():
    # one mode per pixel: g2 - 1 = mean_p exp(-2 Gamma_p tau), so the fitted t0 lies between
    # the ring's extreme 1/Gamma and near 1/mean(Gamma), with baseline 1 and contrast 1
    H = W = 64
    T, n_q, D = 800, 8, 4e-4
    X = speckle_counts(H, W, T, 2.0, D, 12, np.uint8)
    qmap = ring_qmap(H, W, n_q)
    gam = rate_of_pixels(H, W, D)
    C, _, _, _ = O.raw_twotime(X, qmap, n_q)
    for q in (1, 2, 3):
        g2, _ = O.g2_from_twotime(C[q])
        B, Cc, t0, _ = O.relaxation_fit(g2, 1, 300, 0.5, 1e4)
        g = gam[O.ring_index(qmap, q)]
        assert 1 / g.max() < t0 < 1 / g.min(), (q, t0)
        assert abs(t0 * g.mean() - 1.0) < 0.15, (q, t0)
        assert abs(B - 1.0) < 0.02 and abs(Cc - 1.0) < 0.05, (q, B, Cc)


def test_peak_visibility_and_detectability_hand_example():
    g2 = np.array([2.0, 1.1, 1.0, 1.02, 0.98, 1.5, 1.3, 1.0, np.nan, 1.0])
    # peak over lags 4..6 is 1.5; background over lags 7..9 (NaN skipped) is 1.0
    assert abs(O.peak_visibility(g2, 4, 6, 7, 9) - 0.5) < 1e-15
    assert O.detectable(0.5, 0.2) and not O.detectable(0.5, 0.3)


def test_twotime_stats_hand_example():
    nan = np.nan
    C = np.array([[9.0, 1.0, 3.0], [1.0, 9.0, nan], [3.0, nan, 9.0]])
    # off-diagonal defined pairs: (1,0) = 1 and (2,0) = 3 -> mean 2, std 1
    m, s = O.twotime_stats(C)
    assert m == 2.0 and s == 1.0


# ---------------------------------------------------------------- per-pair values (sampled parity)

def test_raw_pair_values_hand_example():
    # ring 0 = pixels {0, 2, 3} (M_q = 3), ring 1 = pixel {1}, pixel 4 outside every ring;
    # ring 0's rows: (2, 0, 1), (1, 3, 2), (0, 0, 0) with sums 3, 6, 0
    qmap = np.array([0, 1, 0, 0, -1], dtype=np.int32)
    X = np.array([[2, 7, 0, 1, 9],
                  [1, 0, 3, 2, 9],
                  [0, 5, 0, 0, 9]], dtype=np.uint16)
    N, C = O.raw_pair_values(X, qmap, 0, np.array([0, 0, 1, 2]), np.array([1, 0, 1, 0]))
    assert N.tolist() == [4, 5, 14, 0]
    np.testing.assert_allclose(C[:3], [3 * 4 / (3 * 6), 3 * 5 / (3 * 3), 3 * 14 / (6 * 6)], rtol=1e-15)
    assert np.isnan(C[3])  # a dark frame: the pair is undefined
    # a one-pixel ring: C = x_a x_b / (x_a x_b) = 1 whenever both counts are nonzero
    N1, C1 = O.raw_pair_values(X, qmap, 1, np.array([0, 0]), np.array([2, 1]))
    assert N1.tolist() == [35, 0] and C1[0] == 1.0 and np.isnan(C1[1])


def test_pair_values_agree_with_the_whole_matrix_and_reduce_to_raw_with_a_lossless_basis():
    # per-pair values against the whole-matrix oracle (raw) and, with the identity as a
    # lossless basis (A = X, G_q = diag(ring mask), s_q = ring mask), compressed = raw
    rng = np.random.default_rng(20356041)
    T, M, n_q = 12, 20, 3
    X = rng.poisson(1.5, (T, M)).astype(np.uint16)
    X[4] = 0
    qmap = (np.arange(M) % n_q).astype(np.int32)
    qmap[M - 1] = -1
    t1 = rng.integers(0, T, 40)
    t2 = rng.integers(0, T, 40)
    Cm = O.raw_twotime(X, qmap, n_q)[0]
    B = np.eye(M)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    A = O.encode(X, B)
    for q in range(n_q):
        _, Cr = O.raw_pair_values(X, qmap, q, t1, t2)
        np.testing.assert_array_equal(np.isnan(Cr), np.isnan(Cm[q][t1, t2]))
        ok = ~np.isnan(Cr)
        np.testing.assert_allclose(Cr[ok], Cm[q][t1, t2][ok], rtol=1e-14)
        Cc = O.compressed_pair_values(A, G[q], s[q], Mq[q], t1, t2)
        np.testing.assert_array_equal(np.isnan(Cc), np.isnan(Cr))
        np.testing.assert_allclose(Cc[ok], Cr[ok], rtol=1e-13)
    assert np.isnan(Cr[(t1 == 4) | (t2 == 4)]).all()
