"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding."""
import numpy as np

UPPER_NAN = np.nan


def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch, torch.device("cuda:0")


def rel_errors(got, ref):
    """(rel_max, rel_rms) over entries defined in both: max|d|/max|ref|, ||d||/||ref||."""
    ok = ~np.isnan(ref) & ~np.isnan(got)
    d = np.abs(got[ok] - ref[ok])
    if d.size == 0:
        return 0.0, 0.0
    return float(d.max() / np.abs(ref[ok]).max()), float(np.sqrt((d ** 2).sum() / (ref[ok] ** 2).sum()))


def lower(a):
    """Lower triangle (t1 >= t2) of the last two axes as a flat array per leading index."""
    T = a.shape[-1]
    il = np.tril_indices(T)
    return a[..., il[0], il[1]]


def run_raw(X, ctx, frames, qmap, n_q, want_C=True, want_N=True):
    torch, dev = torch_cuda()
    T, M = frames.shape
    rings = X.Rings(ctx, torch.from_numpy(qmap.astype(np.int32)).to(dev), M, n_q)
    Xd = torch.from_numpy(frames).to(dev)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev) if want_C else None
    N = torch.zeros((n_q, T, T), dtype=torch.int64, device=dev) if want_N else None
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime_raw(ctx, rings, Xd, T, C_out=C, N_out=N, g2_out=g2, count_out=cnt)
    out = dict(g2=g2.cpu().numpy(), count=cnt.cpu().numpy(), rings=rings)
    if want_C:
        out["C"] = C.cpu().numpy()
    if want_N:
        out["N"] = N.cpu().numpy()
    return out
