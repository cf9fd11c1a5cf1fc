"""The C-ABI library loads and exports every entry point include/xpcs.h declares.

CPU-only: loads the shared library and resolves symbols; no compute call is made.
"""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xpcs.h")
LIB = os.path.join(ROOT, "paper_2407_20356_gb300", "lib", "libxpcs.so")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xpcs_[a-z0-9_]+)\s*\(", src)))


def _ensure_built():
    if not os.path.exists(LIB):
        from paper_2407_20356_gb300 import _build

        _build.build_library()


def test_library_exports_every_declared_symbol():
    _ensure_built()
    names = header_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(LIB)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (xpcs_[a-z0-9_]+)\b", out))
    assert set(names) <= exported, set(names) - exported


def test_binding_declares_the_header_functions():
    _ensure_built()
    from paper_2407_20356_gb300 import xpcs

    assert sorted(xpcs.declared_symbols()) == header_functions()
    assert xpcs.xpcs_version() >= 100


def test_binding_constants_match_the_header():
    _ensure_built()
    from paper_2407_20356_gb300 import xpcs

    src = open(HEADER).read()
    m = re.search(r"#define\s+XPCS_G2_NOALLOC_MAX_CELLS\s+\(1 << (\d+)\)", src)
    assert m and xpcs.G2_NOALLOC_MAX_CELLS == 1 << int(m.group(1))
    m = re.search(r"#define\s+XPCS_G2_MAX_RINGS\s+(\d+)", src)
    assert m and xpcs.G2_MAX_RINGS == int(m.group(1))
    for name, val in re.findall(r"\b(XPCS_NORM_[A-Z0-9]+)\s*=\s*(\d+)", src):
        assert getattr(xpcs, name) == int(val), name


def test_rank_rule_host_function_matches_the_oracle():
    # host-side logic behind the ABI (no device work): the rank rule of Sec. 3.1
    _ensure_built()
    import numpy as np

    import oracle as O
    from paper_2407_20356_gb300 import xpcs

    rng = np.random.default_rng(11)
    spectra = [[8.0, 4.0, 2.5, 2.0, 1.5, 1.0], [3.0, 1.0, 0.0, 0.0], [1.0, 1.0, 1.0], [5.0], [0.0, 0.0]]
    spectra += [np.sort(rng.exponential(1.0, size=n))[::-1] for n in (2, 17, 300)]
    for s in spectra:
        for f in (1.5, 2.0, 3.0):
            assert xpcs.xpcs_rank_from_spectrum(s, f) == O.rank_from_spectrum(s, f), (s, f)
    for bad, f in (([1.0, 2.0], 2.0), ([2.0, 1.0], 0.0), ([float("nan"), 1.0], 2.0)):
        try:
            xpcs.xpcs_rank_from_spectrum(bad, f)
        except xpcs.XpcsError:
            continue
        raise AssertionError(("accepted", bad, f))


def test_context_closes_handles_before_the_handles_they_use(monkeypatch):
    # Host logic only: a context built without the device, fake handles named like the
    # binding's classes, and a stub in place of the library's context destroy.  Each
    # handle must be closed before the ones it was made from (server and graph before
    # stream, stream before basis, basis before ring plan), whatever order they were
    # created in, and the context itself last.
    _ensure_built()
    import weakref

    from paper_2407_20356_gb300 import xpcs as X

    order = []

    class _Lib:
        def xpcs_destroy(self, h):
            order.append("Context")

    monkeypatch.setattr(X, "_lib", _Lib())

    def fake(name):
        def close(self):
            order.append(name)

        return type(name, (), {"close": close})()

    ctx = X.Context.__new__(X.Context)
    ctx.h = object()
    ctx._children = weakref.WeakSet()
    kids = [fake(n) for n in ("Rings", "Basis", "Stream", "Graph", "Server", "Stream", "Rings")]
    for k in kids:
        ctx._adopt(k)
    ctx.close()
    rank = {"Server": 0, "Graph": 1, "Stream": 2, "Basis": 3, "Rings": 4}
    assert order[-1] == "Context" and len(order) == len(kids) + 1
    assert [rank[n] for n in order[:-1]] == sorted(rank[n] for n in order[:-1])
    assert ctx.h is None


def test_stream_row_tile_choice_by_step_size():
    # Host-side selection of the stream row update's lag tile and epilogue: every step of
    # 1..64 frames gets a tile whose history rows fit one 128-row operand and a layout that
    # fits 227 KB of shared memory, the small-step epilogue exactly for steps of <= 8
    # frames, and the longest listed tile for the shapes the benchmarks run.
    _ensure_built()
    from paper_2407_20356_gb300 import xpcs as X

    for n_q, k in ((36, 128), (100, 256), (100, 128), (100, 64), (4, 20), (40, 24), (5, 150), (36, 150)):
        for b in range(1, 65):
            t = X.xpcs_stream_row_tile(n_q, k, b)
            assert 0 < t["smem_bytes"] <= 227 * 1024, (n_q, k, b, t)
            if b >= 32:  # steps of 32 frames or more run on the two-time kernel
                assert t["epilogue"] == 3 and t["lags"] == 128 and t["w_stages"] == 0, (n_q, k, b, t)
                continue
            assert t["lags"] in (128, 120, 96, 64, 32) and t["lags"] + b - 1 <= 128, (n_q, k, b, t)
            assert t["w_stages"] in (1, 2), (n_q, k, b, t)
            assert (t["epilogue"] == 2) == (b <= 8), (n_q, k, b, t)
    expect = {(36, 128, 1): 128, (36, 128, 8): 120, (36, 128, 9): 120, (36, 128, 31): 96,
              (100, 256, 1): 64, (100, 256, 9): 32, (100, 64, 1): 128, (100, 64, 31): 96}
    for (n_q, k, b), lags in expect.items():
        assert X.xpcs_stream_row_tile(n_q, k, b)["lags"] == lags, (n_q, k, b)
    for bad in ((0, 128, 1), (36, 0, 1), (36, 257, 1), (36, 128, 0), (36, 128, 65), (1025, 64, 1)):
        try:
            X.xpcs_stream_row_tile(*bad)
        except X.XpcsError as e:
            assert e.status == X.XPCS_EINVAL
        else:
            raise AssertionError(bad)
