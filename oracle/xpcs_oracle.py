"""Plain FP64/int64 oracle of the XPCS correlation path of arXiv 2407.20356.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU-baseline legs
of the benchmark, never by the CUDA library.

Notation follows the paper: X (N x M, rows = flattened frames, Sec. 2.1), V / V_K the
encoding matrix (Eq. 3, 6), Y_K = X V_K the compressed data (Eq. 7), G the two-time
correlation (Eq. 1, 2, 10).  Per q-ring quantities carry a ring index q: M_q pixels,
B_q the rows of the basis B (= V_K) for those pixels.

Readings of the paper taken here (each listed in the design notes):
* Two-time correlation per ring (Eq. 1): the overlines are averages over the ring's
  pixels at a fixed time, so C_q(t1,t2) = M_q N_q(t1,t2) / (S_q(t1) S_q(t2)) with
  N_q = X_q X_q^T (Eq. 2 restricted to the ring) and S_q(t) the ring's photon sum.
  A pair whose denominator factor is <= 0 is undefined (NaN) and excluded from g2.
* g2(tau) is the average of C_q along the tau-th diagonal over the valid pairs;
  index tau runs over 0..T-1 (tau = 0 includes shot noise and is reported as is).
* Basis fit (Eq. 3-6): rows of the fit frames are divided by their Frobenius norm
  (Sec. 2.1), all-zero rows are dropped, no centring; V_K spans the top-K right
  singular vectors, obtained from the eigendecomposition of F F^T:
  B[:, i] = F^T u_i / sigma_i, sigma_i = sqrt(lambda_i).  Column signs: the entry of
  largest magnitude is made positive.
* Compressed path (Eq. 8-10 restricted to a ring): with a_t = x_t B (Eq. 7),
  G_q = B_q^T B_q and s_q = B_q^T 1, the ring Gram of the decompressed frames
  x~ = x B B^T is N~_q(t1,t2) = a_t1 G_q a_t2^T and the ring sum is S~_q(t) = a_t s_q.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "ring_index", "ring_sizes", "ring_sums", "raw_gram", "twotime_from_gram",
    "g2_from_twotime", "raw_twotime", "fit_basis", "encode", "ring_factors",
    "compressed_ring_gram", "compressed_ring_sums", "compressed_twotime", "compressed_twotime_exact_sums",
    "decompress", "raw_pair_values", "compressed_pair_values", "g2_eq12",
    "frobenius_twotime", "windowed_g2", "compression_ratio_offline",
    "compression_ratio_online", "lossless_speedup", "rank_from_spectrum", "twotime_eq12",
    "relaxation_fit", "peak_visibility", "twotime_stats", "detectable",
]


# ---------------------------------------------------------------- rings (Sec. 2.2)

def ring_index(qmap: np.ndarray, q: int) -> np.ndarray:
    """Pixel indices of ring q (a q-range subset of the detector, Sec. 2.2)."""
    return np.flatnonzero(np.asarray(qmap) == q)


def ring_sizes(qmap: np.ndarray, n_q: int) -> np.ndarray:
    """M_q: number of pixels labelled q."""
    return np.array([ring_index(qmap, q).size for q in range(n_q)], dtype=np.int64)


# ---------------------------------------------------------------- raw path (Eq. 1, 2)

def ring_sums(X: np.ndarray, qmap: np.ndarray, n_q: int) -> np.ndarray:
    """S_q(t) = sum over pixels p in ring q of x_{t,p}, int64, shape (n_q, T).

    M_q times the overline of I_t in Eq. 1.
    """
    X = np.asarray(X)
    S = np.zeros((n_q, X.shape[0]), dtype=np.int64)
    for q in range(n_q):
        idx = ring_index(qmap, q)
        if idx.size:
            S[q] = X[:, idx].astype(np.int64).sum(axis=1)
    return S


def raw_gram(X: np.ndarray, qmap: np.ndarray, q: int) -> np.ndarray:
    """N_q = X_q X_q^T in int64 (Eq. 2 on the ring's pixels), shape (T, T)."""
    Xq = np.asarray(X)[:, ring_index(qmap, q)].astype(np.int64)
    return Xq @ Xq.T


def twotime_from_gram(Nq: np.ndarray, S1: np.ndarray, S2: np.ndarray, Mq: float) -> np.ndarray:
    """C(t1,t2) = M_q N(t1,t2) / (S(t1) S(t2)) in float64 (Eq. 1).

    Pairs where either ring sum is <= 0 are NaN.
    """
    S1 = np.asarray(S1, dtype=np.float64)
    S2 = np.asarray(S2, dtype=np.float64)
    den = np.outer(S1, S2)
    ok = np.outer(S1 > 0, S2 > 0)
    C = np.full(den.shape, np.nan)
    C[ok] = float(Mq) * np.asarray(Nq, dtype=np.float64)[ok] / den[ok]
    return C


def g2_from_twotime(C: np.ndarray):
    """g2(tau) = mean over t of C(t, t+tau) over defined pairs, tau = 0..T-1.

    Returns (g2 float64[T], count int64[T]); g2 is NaN where count is 0.
    """
    T = C.shape[0]
    g2 = np.full(T, np.nan)
    cnt = np.zeros(T, dtype=np.int64)
    for tau in range(T):
        d = np.diagonal(C, offset=tau)
        ok = ~np.isnan(d)
        cnt[tau] = int(ok.sum())
        if cnt[tau]:
            g2[tau] = float(d[ok].sum()) / cnt[tau]
    return g2, cnt


def raw_twotime(X: np.ndarray, qmap: np.ndarray, n_q: int):
    """Raw two-time correlation of every ring: (C [n_q,T,T], N [n_q,T,T] int64, S, Mq)."""
    S = ring_sums(X, qmap, n_q)
    Mq = ring_sizes(qmap, n_q)
    T = np.asarray(X).shape[0]
    C = np.empty((n_q, T, T))
    N = np.empty((n_q, T, T), dtype=np.int64)
    for q in range(n_q):
        N[q] = raw_gram(X, qmap, q)
        C[q] = twotime_from_gram(N[q], S[q], S[q], Mq[q])
    return C, N, S, Mq


# ---------------------------------------------------------------- basis fit (Eq. 3-6)

def fit_basis(F: np.ndarray, k: int):
    """Encoding matrix V_K (M x k) of the fit frames F, plus all singular values.

    Rows of F are divided by their Frobenius norm (Sec. 2.1); zero rows are dropped.
    The columns of V are eigenvectors of F^T F (Eq. 3); they are formed from the
    eigenvectors u_i of the small Gram F F^T as F^T u_i / sigma_i.  The K largest are
    kept (Eq. 6).  Raises ValueError if k exceeds the numerical rank.
    """
    F = np.asarray(F, dtype=np.float64)
    nrm = np.sqrt((F * F).sum(axis=1))
    keep = nrm > 0
    Fn = F[keep] / nrm[keep, None]
    Gf = Fn @ Fn.T
    lam, U = np.linalg.eigh(Gf)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    U = U[:, order]
    tol = max(Gf.shape) * np.finfo(np.float64).eps * max(lam[0], 0.0)
    rank = int((lam > tol).sum())
    if k < 1 or k > rank:
        raise ValueError(f"k={k} outside [1, rank={rank}]")
    sigma = np.sqrt(np.maximum(lam, 0.0))
    B = (Fn.T @ U[:, :k]) / sigma[:k]
    for i in range(k):
        j = int(np.argmax(np.abs(B[:, i])))
        if B[j, i] < 0:
            B[:, i] = -B[:, i]
    return B, sigma


def rank_from_spectrum(sigma: np.ndarray, factor: float = 2.0) -> int:
    """Rank choice of Sec. 3.1: how many values of the spectrum are at least `factor`
    times its smallest value (the paper's count uses a factor of two).

    The spectrum is the descending list of singular values returned by fit_basis.  Values
    at or below the numerical-rank cutoff (sigma^2 <= n eps sigma_max^2, the cutoff
    fit_basis applies to the eigenvalues) are not part of it, so a rank-deficient fit
    does not make the minimum zero.
    """
    s = np.asarray(sigma, dtype=np.float64)
    n = s.size
    tol = n * np.finfo(np.float64).eps * max(s[0], 0.0) ** 2
    kept = s[(s > 0) & (s * s > tol)]
    if kept.size == 0:
        return 0
    return int((kept >= factor * kept.min()).sum())


# ---------------------------------------------------------------- compressed path (Eq. 7-10)

def encode(X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Y_K = X V_K (Eq. 7): coefficients a_t = x_t B, float64 (T x k)."""
    return np.asarray(X, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def decompress(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X~ = Y_K V_K^T = X V_K V_K^T (Eq. 5, 8)."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64).T


def ring_factors(B: np.ndarray, qmap: np.ndarray, n_q: int):
    """Per-ring factors of the basis: G_q = B_q^T B_q (k x k), s_q = B_q^T 1, M_q.

    With these, the ring Gram and ring sums of the decompressed frames follow from
    the coefficients alone (Eq. 9-10 restricted to the ring's pixels).
    """
    B = np.asarray(B, dtype=np.float64)
    k = B.shape[1]
    G = np.zeros((n_q, k, k))
    s = np.zeros((n_q, k))
    Mq = np.zeros(n_q, dtype=np.int64)
    for q in range(n_q):
        Bq = B[ring_index(qmap, q)]
        G[q] = Bq.T @ Bq
        s[q] = Bq.sum(axis=0)
        Mq[q] = Bq.shape[0]
    return G, s, Mq


def compressed_ring_gram(A: np.ndarray, Gq: np.ndarray) -> np.ndarray:
    """N~_q = A G_q A^T (Eq. 10 with the ring factor between the coefficient rows)."""
    A = np.asarray(A, dtype=np.float64)
    return A @ Gq @ A.T


def compressed_ring_sums(A: np.ndarray, s: np.ndarray) -> np.ndarray:
    """S~_q(t) = a_t s_q for every ring, shape (n_q, T)."""
    return np.asarray(s, dtype=np.float64) @ np.asarray(A, dtype=np.float64).T


def compressed_twotime(A: np.ndarray, G: np.ndarray, s: np.ndarray, Mq: np.ndarray):
    """Two-time correlation of every ring from coefficients only: (C~ [n_q,T,T], S~)."""
    n_q = G.shape[0]
    T = np.asarray(A).shape[0]
    St = compressed_ring_sums(A, s)
    C = np.empty((n_q, T, T))
    for q in range(n_q):
        C[q] = twotime_from_gram(compressed_ring_gram(A, G[q]), St[q], St[q], Mq[q])
    return C, St


def compressed_twotime_exact_sums(A: np.ndarray, G: np.ndarray, S: np.ndarray, Mq: np.ndarray) -> np.ndarray:
    """Compressed two-time correlation with the exact ring sums of the raw frames in the
    denominators: C_q = M_q N~_q(t1,t2) / (S_q(t1) S_q(t2)), with N~_q = a G_q a^T (Eq. 10)
    and S_q(t) = sum of the ring's raw counts (the Eq. 1 means, captured when the frames are
    encoded) instead of S~_q = a s_q.  Shape [n_q, T, T]; pairs with S <= 0 are NaN."""
    n_q = G.shape[0]
    T = np.asarray(A).shape[0]
    C = np.empty((n_q, T, T))
    for q in range(n_q):
        C[q] = twotime_from_gram(compressed_ring_gram(A, G[q]), S[q], S[q], Mq[q])
    return C


# ---------------------------------------------------------------- sampled values (large sizes)

def raw_pair_values(X: np.ndarray, qmap: np.ndarray, q: int, t1: np.ndarray, t2: np.ndarray):
    """N_q(t1,t2) and C_q(t1,t2) for listed pairs only, computed one pair at a time."""
    idx = ring_index(qmap, q)
    Mq = idx.size
    N = np.empty(len(t1), dtype=np.int64)
    C = np.empty(len(t1))
    for i, (a, b) in enumerate(zip(t1, t2)):
        xa = np.asarray(X[a, idx], dtype=np.int64)
        xb = np.asarray(X[b, idx], dtype=np.int64)
        N[i] = int(xa @ xb)
        sa, sb = int(xa.sum()), int(xb.sum())
        C[i] = Mq * N[i] / (sa * sb) if (sa > 0 and sb > 0) else np.nan
    return N, C


def compressed_pair_values(A: np.ndarray, Gq: np.ndarray, sq: np.ndarray, Mq: int,
                           t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
    """C~_q(t1,t2) for listed pairs only."""
    A = np.asarray(A, dtype=np.float64)
    out = np.empty(len(t1))
    for i, (a, b) in enumerate(zip(t1, t2)):
        n = A[a] @ Gq @ A[b]
        sa, sb = A[a] @ sq, A[b] @ sq
        out[i] = Mq * n / (sa * sb) if (sa > 0 and sb > 0) else np.nan
    return out


# ---------------------------------------------------------------- variants and reporting

def g2_eq12(X: np.ndarray, qmap: np.ndarray, q: int, tau: int) -> float:
    """Literal Eq. 12: <I(q,t) I(q,t+tau)> / <I(q)>^2, averages over t and ring pixels."""
    Xq = np.asarray(X)[:, ring_index(qmap, q)].astype(np.float64)
    T = Xq.shape[0]
    num = (Xq[: T - tau] * Xq[tau:]).mean()
    den = Xq.mean() ** 2
    return float(num / den)


def frobenius_twotime(Nq: np.ndarray) -> np.ndarray:
    """Eq. 2 with rows normalised by their Frobenius norm: N(t1,t2)/sqrt(N(t1,t1) N(t2,t2))."""
    d = np.sqrt(np.diagonal(np.asarray(Nq, dtype=np.float64)))
    den = np.outer(d, d)
    out = np.full(den.shape, np.nan)
    ok = den > 0
    out[ok] = np.asarray(Nq, dtype=np.float64)[ok] / den[ok]
    return out


def twotime_eq12(Nq: np.ndarray, S: np.ndarray, Mq: float) -> np.ndarray:
    """Two-time form of the literal Eq. 12: M_q N(t1,t2) / Sbar^2, Sbar the ring sum averaged
    over all T frames.  Its mean along the tau-th diagonal (every pair counts) is
    <I(q,t) I(q,t+tau)> / <I(q)>^2 with both averages over frames and the ring's pixels.
    NaN everywhere if Sbar <= 0.
    """
    Sbar = float(np.mean(np.asarray(S, dtype=np.float64)))
    N = np.asarray(Nq, dtype=np.float64)
    if Sbar <= 0:
        return np.full(N.shape, np.nan)
    return float(Mq) * N / (Sbar * Sbar)


# ---------------------------------------------------------------- downstream analysis (Sec. 3)

def relaxation_fit(g2: np.ndarray, tau_lo: int, tau_hi: int, t0_min: float, t0_max: float):
    """Least-squares fit of Eq. 13, g2(tau) = B + C exp(-2 tau / t0), over the defined lags
    tau_lo..tau_hi (unweighted).

    For a fixed t0 the model is linear in (B, C), solved by lstsq; the residual is then a
    function of t0 alone, minimised over log t0 in [t0_min, t0_max]: a 2001-point grid, then
    a bounded scalar minimisation between the grid neighbours of the best point.  Returns
    (B, C, t0, rms residual); NaNs if fewer than three lags are defined.
    """
    from scipy.optimize import minimize_scalar

    tau = np.arange(tau_lo, tau_hi + 1, dtype=np.float64)
    g = np.asarray(g2, dtype=np.float64)[tau_lo:tau_hi + 1]
    ok = ~np.isnan(g)
    tau, g = tau[ok], g[ok]
    if g.size < 3:
        return (np.nan,) * 4

    def solve(lt0):
        e = np.exp(-2.0 * tau / np.exp(lt0))
        M = np.stack([np.ones_like(e), e], axis=1)
        coef = np.linalg.lstsq(M, g, rcond=None)[0]
        r = g - M @ coef
        return float(r @ r), coef

    grid = np.linspace(np.log(t0_min), np.log(t0_max), 2001)
    res = np.array([solve(x)[0] for x in grid])
    i = int(np.argmin(res))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, grid.size - 1)]
    best = minimize_scalar(lambda x: solve(x)[0], bounds=(lo, hi), method="bounded",
                           options={"xatol": 1e-12})
    lt0 = best.x if best.fun <= res[i] else grid[i]
    rss, (B, C) = solve(lt0)
    return float(B), float(C), float(np.exp(lt0)), float(np.sqrt(rss / g.size))


def peak_visibility(g2: np.ndarray, pa: int, pb: int, ba: int, bb: int) -> float:
    """Sec. 3.1: the peak of g2 over lags pa..pb minus its background level, read as the
    mean of g2 over the lags ba..bb (defined lags only)."""
    g = np.asarray(g2, dtype=np.float64)
    return float(np.nanmax(g[pa:pb + 1]) - np.nanmean(g[ba:bb + 1]))


def twotime_stats(C: np.ndarray):
    """Mean and (population) standard deviation of the two-time values C(t1, t2), t1 != t2,
    over the defined pairs (each unordered pair once), the spread Sec. 3.2 calls the
    background level of the TTC."""
    C = np.asarray(C, dtype=np.float64)
    il = np.tril_indices(C.shape[0], -1)
    v = C[il]
    v = v[~np.isnan(v)]
    if v.size == 0:
        return np.nan, np.nan
    m = v.sum() / v.size
    return float(m), float(np.sqrt(((v - m) ** 2).sum() / v.size))


def detectable(visibility: float, ttc_std: float, factor: float = 2.0) -> bool:
    """Sec. 3.2: a correlation peak counts as detectable when its visibility exceeds
    `factor` (two) times the standard deviation of the TTC."""
    return bool(visibility > factor * ttc_std)


def windowed_g2(C: np.ndarray, W: int):
    """g2 over pairs with tau < W only (a history that keeps the last W frames)."""
    g2, cnt = g2_from_twotime(C)
    g2 = g2.copy()
    cnt = cnt.copy()
    g2[W:] = np.nan
    cnt[W:] = 0
    return g2, cnt


def compression_ratio_offline(N: int, K: int) -> float:
    """Offline CR ~ N / K (Sec. 3.1): raw N x M versus the M x K encoding matrix."""
    return N / K


def compression_ratio_online(M: int, K: int) -> float:
    """Online CR ~ M / K (Sec. 3.2): raw N x M versus the N x K coefficients."""
    return M / K


def lossless_speedup(N: int, M: int) -> float:
    """Lossless compute ratio O(n^2 M) / O(n^2 N) = M / N (Sec. 4 complexity)."""
    return M / N
