"""CUDA-graph capture of library calls: a captured encode + two-time step replays to the
same bytes as the direct calls (every kernel of the step sums in a fixed order), counts its
kernels, and the context refuses what would move buffers a live graph refers to."""
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


def _setup(X, T=300, H=32, W=32, n_q=4, k=24):
    torch, dev = torch_cuda()
    ctx = X.Context(0)
    frames = speckle_counts(H, W, T + 100, 0.5, 2e-3, 20356041, np.uint16)
    B, _ = O.fit_basis(frames[:100], k)
    qmap = ring_qmap(H, W, n_q)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    Xd = torch.from_numpy(frames[100:]).to(dev)
    return torch, dev, ctx, rings, basis, Xd


def test_captured_step_replays_to_the_same_bytes(X):
    torch, dev, ctx, rings, basis, Xd = _setup(X)
    T, n_q, k = Xd.shape[0], 4, 24
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)

    def step():
        X.xpcs_encode(ctx, basis, Xd, T, A)
        X.xpcs_twotime(ctx, basis, A, T, "bf16x3", C_out=C, g2_out=g2, count_out=cnt)

    step()  # direct run: sizes the scratch and makes the first-use pieces
    ctx.synchronize()
    C0, g0, c0 = C.clone(), g2.clone(), cnt.clone()
    C.fill_(float("nan"))  # the library writes the lower triangle only
    g2.fill_(0.0)
    cnt.fill_(0)
    X.xpcs_capture_begin(ctx)
    step()
    graph = X.xpcs_capture_end(ctx)
    assert graph.kernels() >= 4
    assert torch.equal(g2, torch.zeros_like(g2))  # recorded, not run
    n0 = ctx.launch_count()
    for _ in range(2):
        graph.launch()
    ctx.synchronize()
    assert ctx.launch_count() - n0 == 2 * graph.kernels()
    assert torch.equal(C.isnan(), C0.isnan())
    ok = ~C0.isnan()
    assert torch.equal(C[ok], C0[ok])
    assert torch.equal(g2.isnan(), g0.isnan()) and torch.equal(g2[~g0.isnan()], g0[~g0.isnan()])
    assert torch.equal(cnt, c0)
    # while the graph exists, work of a larger shape would move the scratch it uses
    T2 = T + 200
    X2 = torch.zeros((T2, Xd.shape[1]), dtype=Xd.dtype, device=dev)
    X2[:T] = Xd
    A2 = torch.empty((T2, k), dtype=torch.float32, device=dev)
    with pytest.raises(X.XpcsError) as e:
        X.xpcs_encode(ctx, basis, X2, T2, A2)
        X.xpcs_twotime(ctx, basis, A2, T2, "bf16x3", g2_out=torch.empty((n_q, T2), dtype=torch.float64,
                                                                        device=dev))
    assert e.value.status == X.XPCS_EBUSY
    graph.close()
    X.xpcs_encode(ctx, basis, X2, T2, A2)  # fine again once the graph is gone
    ctx.synchronize()
    ctx.close()


def test_capture_refuses_profiling(X):
    torch, dev, ctx, rings, basis, Xd = _setup(X, T=64)
    ctx.profile_enable(True)
    with pytest.raises(X.XpcsError) as e:
        X.xpcs_capture_begin(ctx)
    assert e.value.status == X.XPCS_EINVAL
    ctx.profile_enable(False)
    ctx.close()


def test_autotuned_configuration_gives_the_same_results(X):
    # the tuned configuration only changes how the work is split and scheduled: C is
    # bit-identical, counts exact, g2 equal up to the order of its f32 partial sums
    torch, dev, ctx, rings, basis, Xd = _setup(X, T=700)
    T, n_q, k = Xd.shape[0], 4, 24
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, Xd, T, A)
    outs = []
    for tune in (False, True):
        C = torch.full((n_q, T, T), float("nan"), dtype=torch.float32, device=dev)
        g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
        cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
        if tune:
            got = X.xpcs_autotune_twotime(ctx, basis, A, T, "bf16x3", C_out=C, g2_out=g2, count_out=cnt, reps=1)
            assert got["tiles_per_item"] in (1, 2, 4, 8, 16, 32) and got["ms"] > 0
        else:
            X.xpcs_twotime(ctx, basis, A, T, "bf16x3", C_out=C, g2_out=g2, count_out=cnt)
        ctx.synchronize()
        outs.append((C, g2, cnt))
    (C0, g0, c0), (C1, g1, c1) = outs
    assert torch.equal(C0.isnan(), C1.isnan()) and torch.equal(C0[~C0.isnan()], C1[~C1.isnan()])
    assert torch.equal(c0, c1)
    ok = ~g0.isnan()
    assert torch.allclose(g1[ok], g0[ok], rtol=1e-5, atol=0)
    ctx.close()
