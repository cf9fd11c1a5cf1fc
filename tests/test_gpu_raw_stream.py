"""GPU parity of the online stream on raw frames (xpcs_raw_stream) against the oracle.

Every pushed frame's exact raw two-time row against the last W frames is folded into g2
sums.  Reference: the oracle's raw two-time matrix of the same frames (Eq. 1-2, int64
Gram, FP64), averaged along its diagonals with lags >= W dropped.  The Gram is exact on
the tensor cores; C is three f32 roundings of an exact ratio and the sums run in FP64
over f32 per-tile diagonal sums, so g2 agrees to 2e-6 relative; pair counts are exact.
Step sizes mix single frames, steps cut at 128-frame blocks and 64-frame steps, and the
frames outrun the history ring several times.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.mark.parametrize("W,T,sizes,dtype", [(300, 1100, (1, 3, 64, 13, 100), np.uint8),
                                             (129, 700, (64,), np.uint16),
                                             (40, 260, (1,), np.uint8)])
def test_raw_stream_matches_windowed_oracle(X, W, T, sizes, dtype):
    torch, dev = torch_cuda()
    H, Wd, n_q = 24, 32, 4
    frames = speckle_counts(H, Wd, T, 0.6, 2e-3, 20356100 + W, dtype)
    frames[[5, T // 2]] = 0  # undefined frames
    qmap = ring_qmap(H, Wd, n_q)
    ctx = X.Context(0)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * Wd, n_q)
    rs = X.RawStream(ctx, rings, W, dtype=np.dtype(dtype).name)
    Xd = torch.from_numpy(frames).to(dev)
    i, j = 0, 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        rs.push(Xd[i:i + n])
        i += n
        j += 1
    assert rs.frames() == T
    g2, cnt = rs.read_g2()
    C = O.raw_twotime(frames, qmap, n_q)[0]
    for q in range(n_q):
        g_ref, c_ref = O.windowed_g2(C[q], W)
        np.testing.assert_array_equal(cnt[q], c_ref[:W])
        ok = ~np.isnan(g_ref[:W])
        assert np.array_equal(np.isnan(g2[q]), ~ok)
        np.testing.assert_allclose(g2[q][ok], g_ref[:W][ok], rtol=2e-6, atol=0)
    ctx.close()


def test_raw_stream_rejects_counts_outside_the_exact_range(X):
    torch, dev = torch_cuda()
    ctx = X.Context(0)
    qmap = np.zeros(64, dtype=np.int32)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), 64, 1)
    rs = X.RawStream(ctx, rings, 50, dtype="uint16")
    f = np.zeros((3, 64), dtype=np.uint16)
    f[1, 7] = 300
    with pytest.raises(X.XpcsError) as e:
        rs.push(torch.from_numpy(f).to(dev))
    assert e.value.status == X.XPCS_ERANGE
    ctx.close()
