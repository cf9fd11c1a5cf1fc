"""The overlapped host-frame encode (xpcs_encode_host) against the device-frame encode.

The frames of a 256x256 uint16 detector go from pinned host memory through the staging
buffers in blocks of about 256 MB (2048 frames), here three blocks with a ragged last one.
Each block's encode sums its pixel splits in its own order, so A agrees with xpcs_encode
on the same frames to f32 rounding (1e-6 of max|A|), and with the FP64 oracle to the
encode's tolerance (1e-4 of max|A|).
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap
from synth.speckle import TorchSpeckle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


def test_encode_host_matches_device_encode_over_several_blocks(X):
    torch, dev = torch_cuda()
    H = W = 256
    M, T, k, n_q = H * W, 4500, 32, 8
    ctx = X.Context(0)
    Xd = TorchSpeckle(H, W, 0.1, 2e-3, 20356095, dtype="uint16", device=str(dev)).next(T)
    rng = np.random.default_rng(5)
    B, _ = np.linalg.qr(rng.standard_normal((M, k)))
    qmap = ring_qmap(H, W, n_q)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), M, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    Xh = torch.empty((T, M), dtype=Xd.dtype, pin_memory=True)
    Xh.copy_(Xd)
    A_dev = torch.empty((T, k), dtype=torch.float32, device=dev)
    A_host = torch.full((T, k), float("nan"), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, Xd, T, A_dev, dtype="uint16")
    X.xpcs_encode_host(ctx, basis, Xh, T, A_host, dtype="uint16")
    a, b = A_host.cpu().numpy().astype(np.float64), A_dev.cpu().numpy().astype(np.float64)
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()
    # a few frames of every block against the FP64 oracle
    rows = np.array([0, 1, 2047, 2048, 3000, 4095, 4096, 4499])
    ref = O.encode(Xh.numpy()[rows], B)
    assert np.abs(a[rows] - ref).max() <= 1e-4 * np.abs(ref).max()
    # a second call reuses the staging buffers and events
    A_host.fill_(float("nan"))
    X.xpcs_encode_host(ctx, basis, Xh, T, A_host, dtype="uint16")
    assert torch.equal(A_host, torch.from_numpy(a.astype(np.float32)).to(dev))
    ctx.close()
