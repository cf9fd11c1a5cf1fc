"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

This shows the pins are strong enough: a dropped term, a wrong ring, a wrong lag index
or a skipped normalisation each fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import oracle.xpcs_oracle as OX
import tests.test_oracle_pins as P


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(OX, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _fails(*pins):
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


ALL_PINS = (
    P.test_golden_tiny_twotime,
    P.test_raw_path_matches_brute_force_rationals,
    P.test_constant_frames_correlate_to_one,
    P.test_eq11_identity_basis_reduces_to_raw_exactly,
    P.test_eq10_homomorphic_equals_decompress_then_correlate,
    P.test_basis_orthonormal_eckart_young_and_svd,
    P.test_fitted_basis_at_full_rank_is_lossless,
)


def test_dropped_ring_size_factor_is_caught(monkeypatch):
    orig = OX.twotime_from_gram
    _patch(monkeypatch, "twotime_from_gram", lambda N, S1, S2, Mq: orig(N, S1, S2, 1.0))
    assert _fails(*ALL_PINS)


def test_ring_sum_over_all_pixels_is_caught(monkeypatch):
    orig = OX.ring_factors

    def bad_factors(B, qmap, n_q):
        G, s, Mq = orig(B, qmap, n_q)
        s[:] = np.asarray(B, dtype=np.float64).sum(axis=0)
        return G, s, Mq

    _patch(monkeypatch, "ring_factors", bad_factors)
    assert _fails(*ALL_PINS)


def test_gram_without_ring_factor_is_caught(monkeypatch):
    _patch(monkeypatch, "compressed_ring_gram", lambda A, Gq: np.asarray(A, float) @ np.asarray(A, float).T)
    assert _fails(*ALL_PINS)


def test_lag_off_by_one_is_caught(monkeypatch):
    def bad_g2(C):
        T = C.shape[0]
        g2 = np.full(T, np.nan)
        cnt = np.zeros(T, dtype=np.int64)
        for tau in range(T - 1):
            d = np.diagonal(C, offset=tau + 1)
            ok = ~np.isnan(d)
            cnt[tau] = ok.sum()
            if cnt[tau]:
                g2[tau] = d[ok].mean()
        return g2, cnt

    _patch(monkeypatch, "g2_from_twotime", bad_g2)
    assert _fails(*ALL_PINS)


def test_unnormalised_fit_frames_are_caught(monkeypatch):
    def bad_fit(F, k):
        F = np.asarray(F, dtype=np.float64)
        lam, U = np.linalg.eigh(F @ F.T)
        o = np.argsort(lam)[::-1]
        lam, U = lam[o], U[:, o]
        sig = np.sqrt(np.maximum(lam, 0))
        if k > int((lam > 1e-9 * lam[0]).sum()):
            raise ValueError("rank")
        return (F.T @ U[:, :k]) / sig[:k], sig

    _patch(monkeypatch, "fit_basis", bad_fit)
    assert _fails(*ALL_PINS)


def test_transposed_pixel_axis_in_encode_is_caught(monkeypatch):
    # a_t built from the wrong axis of the basis (B^T B instead of X B) on square inputs
    def bad_encode(X, B):
        X = np.asarray(X, dtype=np.float64)
        B = np.asarray(B, dtype=np.float64)
        return X @ B[::-1]

    _patch(monkeypatch, "encode", bad_encode)
    assert _fails(*ALL_PINS)


@pytest.mark.parametrize("scale", [0.5, 2.0])
def test_scaled_ring_sums_are_caught(monkeypatch, scale):
    orig = OX.ring_sums
    _patch(monkeypatch, "ring_sums", lambda X, qmap, n_q: (orig(X, qmap, n_q) * scale).astype(np.int64))
    assert _fails(*ALL_PINS)


PAIR_PINS = (
    P.test_raw_pair_values_hand_example,
    P.test_pair_values_agree_with_the_whole_matrix_and_reduce_to_raw_with_a_lossless_basis,
)


def test_pair_values_without_ring_size_are_caught(monkeypatch):
    orig = OX.raw_pair_values

    def bad(X, qmap, q, t1, t2):
        N, C = orig(X, qmap, q, t1, t2)
        return N, C / max(1, OX.ring_index(qmap, q).size)  # M_q dropped

    _patch(monkeypatch, "raw_pair_values", bad)
    assert _fails(*PAIR_PINS)


def test_compressed_pair_values_with_swapped_frames_in_one_sum_are_caught(monkeypatch):
    def bad(A, Gq, sq, Mq, t1, t2):
        A = np.asarray(A, dtype=np.float64)
        out = np.empty(len(t1))
        for i, (a, b) in enumerate(zip(t1, t2)):
            n = A[a] @ Gq @ A[b]
            sa, sb = A[a] @ sq, A[a] @ sq  # the second frame's ring sum taken from the first
            out[i] = Mq * n / (sa * sb) if (sa > 0 and sb > 0) else np.nan
        return out

    _patch(monkeypatch, "compressed_pair_values", bad)
    assert _fails(*PAIR_PINS)


EXACT_SUM_PINS = (
    P.test_exact_ring_sums_reduce_to_raw_with_a_lossless_basis,
    P.test_exact_ring_sums_with_a_lossy_basis_from_pixel_definitions,
)


def test_exact_sums_of_the_wrong_ring_are_caught(monkeypatch):
    orig = OX.compressed_twotime_exact_sums
    _patch(monkeypatch, "compressed_twotime_exact_sums",
           lambda A, G, S, Mq: orig(A, G, np.roll(np.asarray(S), 1, axis=0), Mq))
    assert _fails(*EXACT_SUM_PINS)


def test_exact_sums_as_pixel_means_are_caught(monkeypatch):
    orig = OX.compressed_twotime_exact_sums
    _patch(monkeypatch, "compressed_twotime_exact_sums",
           lambda A, G, S, Mq: orig(A, G, np.asarray(S, float) / np.asarray(Mq, float)[:, None], Mq))
    assert _fails(*EXACT_SUM_PINS)


def test_exact_sums_without_the_ring_factor_are_caught(monkeypatch):
    orig = OX.compressed_twotime_exact_sums

    def bad(A, G, S, Mq):
        eye = np.broadcast_to(np.eye(np.asarray(A).shape[1]), np.asarray(G).shape)
        return orig(A, eye, S, Mq)  # N~ = a a^T: the ring factor G_q dropped

    _patch(monkeypatch, "compressed_twotime_exact_sums", bad)
    assert _fails(*EXACT_SUM_PINS)
