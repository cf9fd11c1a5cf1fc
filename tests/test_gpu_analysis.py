"""GPU parity of the downstream analysis (Sec. 3) against the oracle.

* Eq. 13 fit: on the same g2 bytes both sides minimise the same least-squares residual
  (the device sums f32 terms in FP64, the oracle works in FP64 throughout), so B and C
  agree to 1e-5 and t0 to 1e-4 relative; end to end (each side's own g2 of the same
  frames) the parameters agree to 1e-3 relative.
* TTC statistics: the device reads the f32 two-time values (relative rounding 2^-24) and
  sums in FP64, so mean and standard deviation agree to 1e-5 relative.
* Peak visibility and the detectability flag: plain max / mean of the same bytes.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import run_raw, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def _synthetic_g2(n_q, T, seed):
    rng = np.random.default_rng(seed)
    tau = np.arange(T, dtype=np.float64)
    B = 1.0 + 0.01 * rng.standard_normal(n_q)
    C = rng.uniform(0.1, 0.5, n_q)
    t0 = np.exp(rng.uniform(np.log(20.0), np.log(800.0), n_q))
    g2 = B[:, None] + C[:, None] * np.exp(-2.0 * tau[None, :] / t0[:, None])
    g2 += 0.002 * rng.standard_normal((n_q, T))
    g2[:, 0] += 1.0  # shot-noise spike at tau = 0, outside the fitted lags
    g2[rng.random((n_q, T)) < 0.01] = np.nan
    return g2, (B, C, t0)


def test_fit_matches_oracle_on_the_same_curves(X, ctx):
    torch, dev = torch_cuda()
    n_q, T = 5, 3000
    g2, truth = _synthetic_g2(n_q, T, 20356031)
    out = torch.empty((n_q, 4), dtype=torch.float64, device=dev)
    X.xpcs_fit_relaxation(ctx, torch.from_numpy(g2).to(dev), n_q, T, 1, T - 1, 1.0, 1e5, out)
    got = out.cpu().numpy()
    for q in range(n_q):
        B, C, t0, rms = O.relaxation_fit(g2[q], 1, T - 1, 1.0, 1e5)
        assert abs(got[q, 0] - B) < 1e-5 and abs(got[q, 1] - C) < 1e-5, (q, got[q], (B, C))
        assert abs(got[q, 2] / t0 - 1.0) < 1e-4, (q, got[q, 2], t0)
        assert abs(got[q, 3] / rms - 1.0) < 1e-4
        assert abs(t0 / truth[2][q] - 1.0) < 0.05  # and the fit finds the planted decay


def test_fit_end_to_end_on_speckle(X, ctx):
    torch, dev = torch_cuda()
    H = W = 48
    T, n_q, D = 600, 6, 4e-4
    frames = speckle_counts(H, W, T, 2.0, D, 20356032, np.uint8)
    qmap = ring_qmap(H, W, n_q)
    raw = run_raw(X, ctx, frames, qmap, n_q, want_C=False, want_N=False)
    out = torch.empty((n_q, 4), dtype=torch.float64, device=dev)
    X.xpcs_fit_relaxation(ctx, torch.from_numpy(raw["g2"]).to(dev), n_q, T, 1, 300, 0.5, 1e4, out)
    got = out.cpu().numpy()
    C = O.raw_twotime(frames, qmap, n_q)[0]
    for q in range(1, n_q):
        g_ref, _ = O.g2_from_twotime(C[q])
        ref = O.relaxation_fit(g_ref, 1, 300, 0.5, 1e4)
        np.testing.assert_allclose(got[q, :3], ref[:3], rtol=1e-3)


def test_fit_with_too_few_lags_gives_nan(X, ctx):
    torch, dev = torch_cuda()
    g2 = np.full((2, 50), np.nan)
    g2[0, 1:3] = 1.2  # two defined lags: too few
    g2[1, 1:40] = 1.0 + 0.2 * np.exp(-2.0 * np.arange(1, 40) / 10.0)
    out = torch.empty((2, 4), dtype=torch.float64, device=dev)
    X.xpcs_fit_relaxation(ctx, torch.from_numpy(g2).to(dev), 2, 50, 1, 49, 1.0, 1e3, out)
    got = out.cpu().numpy()
    assert np.isnan(got[0]).all()
    assert abs(got[1, 2] - 10.0) < 1e-3


def test_twotime_stats_match_oracle(X, ctx):
    torch, dev = torch_cuda()
    H = W = 32
    T, n_q = 300, 4
    frames = speckle_counts(H, W, T, 0.5, 1e-3, 20356033, np.uint16)
    frames[[10, 200]] = 0  # undefined frames: NaN rows and columns are skipped
    qmap = ring_qmap(H, W, n_q)
    torch, dev = torch_cuda()
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    Cd = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    X.xpcs_twotime_raw(ctx, rings, torch.from_numpy(frames).to(dev), T, C_out=Cd)
    mean = torch.empty(n_q, dtype=torch.float64, device=dev)
    sd = torch.empty(n_q, dtype=torch.float64, device=dev)
    X.xpcs_twotime_stats(ctx, Cd, n_q, T, mean, sd)
    Cref = O.raw_twotime(frames, qmap, n_q)[0]
    for q in range(n_q):
        m, s = O.twotime_stats(Cref[q])
        assert abs(mean[q].item() / m - 1.0) < 1e-5 and abs(sd[q].item() / s - 1.0) < 1e-5, (q, m, s)


def test_peak_visibility_and_detectability(X, ctx):
    torch, dev = torch_cuda()
    n_q, T = 3, 400
    rng = np.random.default_rng(20356034)
    g2 = 1.0 + 0.002 * rng.standard_normal((n_q, T))
    g2[:, 118:123] += np.array([0.02, 0.05, 0.08])[:, None]  # planted peak near lag 120
    g2[1, 300] = np.nan
    ttc_sd = np.array([0.02, 0.02, 0.02])
    dg2 = torch.from_numpy(g2).to(dev)
    vis = torch.empty(n_q, dtype=torch.float64, device=dev)
    flag = torch.empty(n_q, dtype=torch.int32, device=dev)
    X.xpcs_peak_visibility(ctx, dg2, n_q, T, 100, 140, 250, 399, vis, torch.from_numpy(ttc_sd).to(dev), 2.0, flag)
    for q in range(n_q):
        v = O.peak_visibility(g2[q], 100, 140, 250, 399)
        assert abs(vis[q].item() - v) < 1e-12
        assert bool(flag[q].item()) == O.detectable(v, ttc_sd[q])
    assert flag.cpu().numpy().tolist() == [0, 1, 1]


def test_analysis_rejects_bad_windows(X, ctx):
    torch, dev = torch_cuda()
    g2 = torch.ones((1, 10), dtype=torch.float64, device=dev)
    out = torch.empty((1, 4), dtype=torch.float64, device=dev)
    for args in ((1, 10, 1.0, 10.0), (5, 4, 1.0, 10.0), (1, 9, 10.0, 1.0)):
        with pytest.raises(X.XpcsError) as e:
            X.xpcs_fit_relaxation(ctx, g2, 1, 10, *args, out)
        assert e.value.status == X.XPCS_EINVAL
    vis = torch.empty(1, dtype=torch.float64, device=dev)
    with pytest.raises(X.XpcsError):
        X.xpcs_peak_visibility(ctx, g2, 1, 10, 0, 10, 0, 3, vis)
