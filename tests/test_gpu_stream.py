"""GPU parity of the online stream (Sec. 2.2, Fig. 1c) against the oracle.

The stream folds every pushed frame's two-time row into g2 sums over lags < W.  The
reference is the FP64 oracle of the compressed two-time matrix of the same frames from
the same FP64 basis, averaged along diagonals with lags >= W dropped.  The stream works in
f32 (sparse encode, k-term dot products) with bf16x3 products, so g2 agrees to 1e-4 of
max|g2|; a stream opened in f16 (one product of f16 rows) is held to 1e-3.  Pair counts are
exact, including the counts that single-frame steps defer to 64-frame blocks.
"""
import numpy as np
import pytest

import oracle as O
from synth import ring_qmap, speckle_counts
from tests.gpu_util import rel_errors, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2407_20356_gb300 import xpcs

    return xpcs


@pytest.fixture(scope="module")
def ctx(X):
    return X.Context(0)


def _setup(X, ctx, H, W, n_q, k, T, n_fit, dtype, seed, mean=0.3):
    torch, dev = torch_cuda()
    frames = speckle_counts(H, W, n_fit + T, mean, 2e-3, seed, dtype)
    B, _ = O.fit_basis(frames[:n_fit], k)  # calibration run before acquisition
    qmap = ring_qmap(H, W, n_q)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    return frames[n_fit:], B, qmap, rings, basis


def _oracle_window_g2(Xs, B, qmap, n_q, Wl):
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    C, _ = O.compressed_twotime(O.encode(Xs, B), G, s, Mq)
    out_g, out_c = [], []
    for q in range(n_q):
        g, c = O.windowed_g2(C[q], Wl)
        out_g.append(g[:Wl])
        out_c.append(c[:Wl])
    return np.array(out_g), np.array(out_c)


@pytest.mark.parametrize("dtype,k,Wl,sizes", [(np.uint16, 20, 50, (1, 3, 8, 13, 5)),
                                              (np.uint8, 64, 120, (8,)),
                                              (np.uint16, 150, 64, (2, 7))])
def test_stream_g2_matches_oracle(X, ctx, dtype, k, Wl, sizes):
    H, W, n_q, T = 24, 40, 4, 200
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 250, dtype, 300 + k)
    st = X.Stream(ctx, basis, Wl, 8, dtype=np.dtype(dtype).name)
    i, j = 0, 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    assert st.frames() == T
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    lat = st.latency()
    assert lat["batches"] > 0 and lat["p99_us"] >= lat["p50_us"] > 0
    st.close()


def test_stream_small_and_large_steps_mixed(X, ctx):
    # steps of at most 8 frames and larger steps lay out their (frame, ring) pairs
    # differently; mixing them in one stream, in both orders, must not change g2
    H, W, n_q, k, T, Wl = 20, 20, 5, 32, 160, 70
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 150, np.uint16, 515)
    st = X.Stream(ctx, basis, Wl, 12)
    i, j, sizes = 0, 0, (4, 12, 9, 1, 12, 5)
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    st.close()


def test_stream_many_rings_and_lag_tiles(X, ctx):
    # more rings than one row-update ring group (36) and several 128-lag tiles, batches
    # longer than one window shift (16 frames)
    H, W, n_q, k, T, Wl = 24, 24, 40, 24, 300, 260
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 200, np.uint16, 404, mean=1.0)
    st = X.Stream(ctx, basis, Wl, 40)
    for i, n in ((0, 37), (37, 1), (38, 40), (78, 222)):
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
    assert st.poll(ticket, 10000)
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    st.close()


@pytest.mark.parametrize("k,sizes", [(128, (9, 1, 12, 40, 3)), (256, (1, 9, 64, 5))])
def test_stream_lag_tiles_and_epilogues(X, ctx, k, sizes):
    # the row update picks its lag tile from the step size (128 lags for one frame, 120 up
    # to 9, 96 up to 33, else 64 or 32) and its epilogue from what fits shared memory: at
    # 36 rings these steps reach the small-step, rotated-block and skewed-buffer epilogues
    # at k = 128 and k = 256; a window of 300 lags leaves a ragged last tile at every size.
    # 1600 pixels and a 600-frame calibration keep k = 256 well below the data's rank, so
    # no ring's compressed sum S~ comes near zero (on a 576-pixel detector one ring's
    # S~ nearly cancels and its lag-0 g2 reaches 4e5, amplifying f32 rounding the same way
    # for every batching)
    H, W, n_q, T, Wl = 40, 40, 36, 420, 300
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 600, np.uint16, 606 + k, mean=1.0)
    st = X.Stream(ctx, basis, Wl, 64)
    i, j = 0, 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    st.close()


def test_stream_batching_and_device_push_agree(X, ctx):
    torch, dev = torch_cuda()
    H, W, n_q, k, T, Wl = 16, 32, 3, 24, 150, 40
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 120, np.uint16, 77)
    a = X.Stream(ctx, basis, Wl, 1)
    for t in range(T):
        a.push(Xs[t:t + 1])
    b = X.Stream(ctx, basis, Wl, 16)
    b.push(torch.from_numpy(Xs).to(dev))  # device frames, batches of 16
    ga, ca = a.read_g2()
    gb, cb = b.read_g2()
    np.testing.assert_array_equal(ca, cb)
    ok = ~np.isnan(ga)
    np.testing.assert_allclose(gb[ok], ga[ok], rtol=1e-6)


def test_stream_push_at_counts_latency_from_arrival(X, ctx):
    # frames stamped 20 ms in the past: every latency includes those 20 ms; results are
    # those of an unstamped device push
    torch, dev = torch_cuda()
    H, W, n_q, k, T, Wl = 16, 16, 2, 16, 64, 32
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 80, np.uint16, 55)
    Xd = torch.from_numpy(Xs).to(dev)
    a = X.Stream(ctx, basis, Wl, 8)
    b = X.Stream(ctx, basis, Wl, 8)
    a.push(Xd)
    t0 = X.clock_ns()
    arrive = t0 - 20_000_000 + np.arange(T, dtype=np.int64) * 1000
    ticket = b.push_at(Xd, arrive)
    assert b.poll(ticket, 10000)
    lat = b.latency(reset=True)
    assert lat["batches"] == T
    assert 20_000 - T < lat["p50_us"] <= lat["p99_us"] <= lat["max_us"]
    assert lat["max_us"] < 20_000 + 10_000_000  # bounded by the poll timeout
    ga, ca = a.read_g2()
    gb, cb = b.read_g2()
    np.testing.assert_array_equal(ca, cb)
    ok = ~np.isnan(ga)
    np.testing.assert_array_equal(gb[ok], ga[ok])
    a.close()
    b.close()


def test_stream_matches_offline_twotime(X, ctx):
    # streamed g2 == offline compressed two-time g2 on the same frames (lags < W)
    torch, dev = torch_cuda()
    H, W, n_q, k, T, Wl = 20, 20, 4, 32, 256, 256
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 150, np.uint16, 91)
    st = X.Stream(ctx, basis, Wl, 32)
    st.push(Xs)
    g2s, cs = st.read_g2()
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    X.xpcs_encode(ctx, basis, torch.from_numpy(Xs).to(dev), T, A)
    g2o = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    co = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    X.xpcs_twotime(ctx, basis, A, T, "bf16x3", g2_out=g2o, count_out=co)
    np.testing.assert_array_equal(cs, co.cpu().numpy())
    for q in range(n_q):
        rm, _ = rel_errors(g2s[q], g2o[q].cpu().numpy())
        assert rm < 1e-4, (q, rm)


def test_stream_admission_by_budget(X):
    # a context whose budget holds one stream: the second open is refused until the
    # first closes
    torch, dev = torch_cuda()
    H, W, n_q, k = 32, 32, 4, 16
    frames = speckle_counts(H, W, 100, 0.5, 2e-3, 5, np.uint16)
    B, _ = O.fit_basis(frames, k)
    probe = X.Context(0)
    rings = X.Rings(probe, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(probe, rings, B)
    s1 = X.Stream(probe, basis, 20000, 8)
    one = probe.device_bytes()
    s1.close()
    base = probe.device_bytes()
    probe.close()
    ctx = X.Context(0, hbm_budget=base + (one - base) + (one - base) // 2)
    rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
    basis = X.xpcs_basis_import(ctx, rings, B)
    a = X.Stream(ctx, basis, 20000, 8)
    with pytest.raises(X.XpcsError) as e:
        X.Stream(ctx, basis, 20000, 8)
    assert e.value.status == X.XPCS_EBUSY
    a.close()
    b = X.Stream(ctx, basis, 20000, 8)  # admitted once memory is free
    b.push(frames[:10])
    g2, cnt = b.read_g2()
    assert cnt[:, 0].max() > 0


def test_stream_checkpoint_and_resume(X, ctx):
    # a stream checkpointed mid-series and resumed in a fresh stream ends with the same
    # bytes as one that ran through (same batches), and both match the oracle
    H, W, n_q, k, T, Wl = 16, 32, 3, 24, 200, 60
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 120, np.uint16, 88)
    full = X.Stream(ctx, basis, Wl, 8)
    for i in range(0, T, 8):
        full.push(Xs[i:i + 8])
    first = X.Stream(ctx, basis, Wl, 8)
    for i in range(0, 96, 8):
        first.push(Xs[i:i + 8])
    ck = first.checkpoint()
    first.close()
    resumed = X.Stream(ctx, basis, Wl, 8)
    resumed.restore(ck)
    assert resumed.frames() == 96
    for i in range(96, T, 8):
        resumed.push(Xs[i:i + 8])
    gf, cf = full.read_g2()
    gr, cr = resumed.read_g2()
    np.testing.assert_array_equal(cr, cf)
    assert np.array_equal(np.isnan(gr), np.isnan(gf)) and np.array_equal(gr[~np.isnan(gr)], gf[~np.isnan(gf)])
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cr, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(gr[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    # a checkpoint only goes into a fresh stream of the same shape
    with pytest.raises(X.XpcsError) as e:
        resumed.restore(ck)
    assert e.value.status == X.XPCS_EINVAL
    other = X.Stream(ctx, basis, Wl + 1, 8)
    with pytest.raises(X.XpcsError) as e:
        other.restore(ck)
    assert e.value.status == X.XPCS_EINVAL


@pytest.mark.parametrize("dtype,k,n_q,Wl,T,sizes,mb", [(np.uint16, 20, 4, 300, 900, (64, 40, 33, 100, 1, 64), 64),
                                                       (np.uint8, 64, 40, 60, 500, (64, 32, 7), 64),
                                                       (np.uint16, 150, 5, 200, 700, (64,), 64),
                                                       (np.uint16, 24, 6, 400, 1000, (128, 100, 130, 5), 128)])
def test_stream_large_steps_on_the_twotime_kernel(X, ctx, dtype, k, n_q, Wl, T, sizes, mb):
    # steps of 32 frames or more run on the two-time kernel (history blocks x the step's
    # 128-frame block); pushes are cut at block boundaries, the history ring wraps, and
    # small steps on the row update kernel are mixed in
    H, W = 24, 40
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 250, dtype, 700 + k)
    st = X.Stream(ctx, basis, Wl, mb, dtype=np.dtype(dtype).name)
    i, j = 0, 0
    ticket = 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    assert st.frames() == T
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-4, (q, rm)
    st.close()


# f16 streams: the coefficient history and the w_q(t) rows as one f16 piece (one product,
# unit roundoff 2^-11), so g2 agrees to 1e-3 of max|g2| (as the offline f16 path); pair
# counts stay exact.  Single frames (the single-frame kernel, up to k = 256 in f16), small
# steps (the row update kernel), large steps (the two-time kernel) and the ring buffer's
# wrap are all covered.
@pytest.mark.parametrize("dtype,k,n_q,Wl,T,sizes,mb,mean", [(np.uint16, 20, 4, 50, 200, (1, 3, 8, 13, 1, 5), 16, 0.3),
                                                            (np.uint16, 200, 5, 130, 300, (1, 1, 7, 1, 64), 64, 0.3),
                                                            (np.uint8, 64, 40, 60, 400, (64, 32, 7, 1), 64, 0.3),
                                                            (np.uint16, 24, 6, 400, 1000, (128, 100, 130, 5), 128, 0.3),
                                                            (np.uint16, 48, 3, 90, 300, (1, 9, 20, 3), 32, 5000.0)])
def test_stream_fp16_matches_oracle(X, ctx, dtype, k, n_q, Wl, T, sizes, mb, mean):
    # the last case has about 5000 photons per pixel (steps below 32 frames: the sparse
    # encode takes counts of any size): leading coefficients near 1.5e5, above the f16
    # range unless each history row carries its scale
    H, W = 24, 40
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 250, dtype, 900 + k, mean=mean)
    st = X.Stream(ctx, basis, Wl, mb, dtype=np.dtype(dtype).name, prec="fp16")
    i, j = 0, 0
    ticket = 0
    while i < T:
        n = min(sizes[j % len(sizes)], T - i)
        ticket = st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        j += 1
    assert st.poll(ticket, 10000)
    g2, cnt = st.read_g2()
    g_ref, c_ref = _oracle_window_g2(Xs, B, qmap, n_q, Wl)
    np.testing.assert_array_equal(cnt, c_ref)
    for q in range(n_q):
        rm, _ = rel_errors(g2[q], g_ref[q])
        assert rm < 1e-3, (q, rm)
    st.close()


def test_stream_precision_options_and_checkpoints(X, ctx):
    # bf16 is not a stream precision; a checkpoint goes only into a stream of its own
    # precision, and an f16 stream resumes from its checkpoint bit for bit
    H, W, n_q, k, T, Wl = 16, 32, 3, 24, 160, 40
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 120, np.uint16, 91)
    with pytest.raises(X.XpcsError) as e:
        X.Stream(ctx, basis, Wl, 8, prec="bf16")
    assert e.value.status == X.XPCS_EINVAL
    full = X.Stream(ctx, basis, Wl, 8, prec="fp16")
    first = X.Stream(ctx, basis, Wl, 8, prec="fp16")
    for i in range(0, T, 8):
        full.push(Xs[i:i + 8])
        if i < 80:
            first.push(Xs[i:i + 8])
    ck = first.checkpoint()
    first.close()
    wrong = X.Stream(ctx, basis, Wl, 8)  # bf16x3
    with pytest.raises(X.XpcsError) as e:
        wrong.restore(ck)
    assert e.value.status == X.XPCS_EINVAL
    wrong.close()
    resumed = X.Stream(ctx, basis, Wl, 8, prec="fp16")
    resumed.restore(ck)
    for i in range(80, T, 8):
        resumed.push(Xs[i:i + 8])
    gf, cf = full.read_g2()
    gr, cr = resumed.read_g2()
    np.testing.assert_array_equal(cr, cf)
    assert np.array_equal(np.isnan(gr), np.isnan(gf)) and np.array_equal(gr[~np.isnan(gr)], gf[~np.isnan(gf)])
    full.close()
    resumed.close()


def test_stream_deferred_pair_counts(X, ctx):
    # single-frame steps defer their pair counts to blocks of 64 frames, added one 64th of
    # the lag range per later single-frame step (or at a read, a checkpoint, or a larger
    # step): exact counts at reads in mid-block, around larger steps and across a
    # checkpoint, with about a third of the frames undefined in a ring (exact ring sums of
    # sparse frames: a ring without photons has S = 0)
    H, W, n_q, k, T, Wl = 24, 40, 4, 20, 560, 150
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 250, np.uint16, 4242, mean=0.004)
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    A = O.encode(Xs, B)
    S = O.ring_sums(Xs, qmap, n_q)
    assert (S == 0).mean() > 0.1

    def check(st, Tr, tol):
        g2, cnt = st.read_g2()
        C = O.compressed_twotime_exact_sums(A[:Tr], G, S[:, :Tr], Mq)
        m = min(Tr, Wl)  # lags beyond the frames so far have no pairs
        for q in range(n_q):
            g_ref, c_ref = O.windowed_g2(C[q], Wl)
            np.testing.assert_array_equal(cnt[q][:m], c_ref[:m])
            assert not cnt[q][m:].any() and np.isnan(g2[q][m:]).all()
            rm, _ = rel_errors(g2[q][:m], g_ref[:m])
            assert rm < tol, (Tr, q, rm)

    # one frame at a time, a 5-frame step at frame 100, a 40-frame step at 180, reads at
    # 131 (mid-block) and 300, a checkpoint at 400 (mid-block) resumed in a fresh stream
    plan = [1] * 100 + [5] + [1] * 75 + [40] + [1] * 180 + [1] * 160
    st = X.Stream(ctx, basis, Wl, 64, qmean="exact_raw")
    i = 0
    for n in plan:
        st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
        if i in (131, 300):
            check(st, i, 1e-4)
        if i == 400:
            ck = st.checkpoint()
            st.close()
            st = X.Stream(ctx, basis, Wl, 64, qmean="exact_raw")
            st.restore(ck)
    assert i == T
    check(st, T, 1e-4)
    st.close()
    # the same in f16
    st = X.Stream(ctx, basis, Wl, 64, qmean="exact_raw", prec="fp16")
    i = 0
    for n in plan:
        st.push(np.ascontiguousarray(Xs[i:i + n]))
        i += n
    check(st, T, 1e-3)
    st.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16"])
def test_stream_single_frames_at_long_history(X, ctx, prec):
    # 36 rings and k = 128: one frame at a time takes the single-frame kernel with each
    # tile's running sums staged in shared memory (one slice for bf16x3 rows, two for f16),
    # and with 157 lag tiles over at most 152 CTAs some fold two tiles, so the slices'
    # phases turn over.  The same frames in steps of two (the row update kernel, which
    # counts its pairs itself) give the same counts and g2 up to the products' summation
    # order.
    H, W, n_q, k, T, Wl = 48, 48, 36, 128, 20200, 20000
    Xs, B, qmap, rings, basis = _setup(X, ctx, H, W, n_q, k, T, 400, np.uint16, 1571, mean=0.3)
    a = X.Stream(ctx, basis, Wl, 2, prec=prec)
    b = X.Stream(ctx, basis, Wl, 2, prec=prec)
    t = 0
    for i in range(T):
        t = a.push(Xs[i:i + 1])
    assert a.poll(t, 60000)
    for i in range(0, T, 2):
        t = b.push(Xs[i:i + 2])
    assert b.poll(t, 60000)
    ga, ca = a.read_g2()
    gb, cb = b.read_g2()
    np.testing.assert_array_equal(ca, cb)
    assert ca[:, 0].min() > 0 and ca[:, Wl - 1].min() > 0
    ok = ~np.isnan(ga)
    assert np.array_equal(ok, ~np.isnan(gb))
    np.testing.assert_allclose(ga[ok], gb[ok], rtol=1e-5)
    a.close()
    b.close()
