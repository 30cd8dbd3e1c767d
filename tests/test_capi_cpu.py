"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/rsc.h declares, and rejects bad arguments on
the host before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2603_02402_gb300 import build as build_lib
from paper_2603_02402_gb300 import rsc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_lib()
    return rsc.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rsc_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert "rsc_knn" in declared and "rsc_connectivities" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(rsc.SIGNATURES) == declared


def test_version(L):
    assert "sm_103a" in rsc.rsc_version()


def test_workspace_size_is_host_only_and_grows(L):
    a = rsc.rsc_knn_workspace_size(10_000, 50, 15)
    b = rsc.rsc_knn_workspace_size(20_000, 50, 15)
    assert 0 < a < b
    c = rsc.rsc_connectivities_workspace_size(10_000, 15)
    assert c > 10_000 * 15 * 12
    assert rsc.rsc_connectivities_max_nnz(10, 15) == 2 * 10 * 14


@pytest.mark.parametrize("args,code", [
    ((0, 50, 15, 0), rsc.RSC_ERR_INVALID_ARG),        # n = 0
    ((100, 0, 15, 0), rsc.RSC_ERR_INVALID_ARG),       # d = 0
    ((100, 65, 15, 0), rsc.RSC_ERR_INVALID_ARG),      # d too large
    ((100, 64, 15, 1), rsc.RSC_ERR_INVALID_ARG),      # cosine needs d <= 63
    ((100, 50, 0, 0), rsc.RSC_ERR_INVALID_ARG),       # k = 0
    ((10, 50, 11, 0), rsc.RSC_ERR_INVALID_ARG),       # k > n
    ((100, 50, 65, 0), rsc.RSC_ERR_INVALID_ARG),      # k > 64
    ((100, 50, 15, 7), rsc.RSC_ERR_INVALID_ARG),      # metric
])
def test_knn_argument_errors(L, args, code):
    n, d, k, m = args
    out = ctypes.c_size_t(0)
    o = rsc.rsc_knn_opts(0, 0, 0, 0, None, None)
    st = L.rsc_knn_workspace_size(n, d, k, m, ctypes.byref(o), ctypes.byref(out))
    assert st == code
    assert L.rsc_last_error()


def test_knn_rejects_missing_workspace_before_launch(L):
    o = rsc.rsc_knn_opts(0, 0, 0, 0, None, None)
    fake = ctypes.c_void_p(256)   # never dereferenced: the workspace check fails first
    st = L.rsc_knn(fake, 1000, 50, 15, 0, fake, fake, ctypes.byref(o), None, 0)
    assert st == rsc.RSC_ERR_WORKSPACE
    st = L.rsc_knn(fake, 1000, 50, 15, 0, fake, fake, ctypes.byref(o), ctypes.c_void_p(512), 16)
    assert st == rsc.RSC_ERR_WORKSPACE
    st = L.rsc_knn(fake, 1000, 50, 15, 0, fake, fake, ctypes.byref(o), ctypes.c_void_p(100), 1 << 40)
    assert st == rsc.RSC_ERR_INVALID_ARG   # misaligned


def test_candidate_option_errors(L):
    out = ctypes.c_size_t(0)
    o = rsc.rsc_knn_opts(0, 10, 0, 0, None, None)      # fewer candidates than k
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(0, 80, 0, 0, None, None)      # above the widest list
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(9, 0, 0, 0, None, None)       # unknown precision
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(1, 0, 0, 3, None, None)       # tc_parts must be 0, 2 or 4
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(1, 0, 0, 0, None, None, 3)    # locality must be 0, 1 or 2
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(1, 0, 0, 0, None, None, 0, 5)  # prune must be 0, 1 or 2
    assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(1, 0, 0, 0, None, None, 1, 2)  # pruning needs the locality ordering
    assert L.rsc_knn_workspace_size(100_000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_UNSUPPORTED
    for stages in (1, 7):                                 # 0 or 2 .. 6 pipeline stages
        o = rsc.rsc_knn_opts(1, 0, 0, 0, None, None, 0, 0, stages)
        assert L.rsc_knn_workspace_size(1000, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_INVALID_ARG
    o = rsc.rsc_knn_opts(3, 0, 0, 0, None, None)          # FP8 folds the norm into 5 columns: d <= 59
    assert L.rsc_knn_workspace_size(1000, 60, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_ERR_UNSUPPORTED
    assert L.rsc_knn_workspace_size(1000, 59, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_OK


def _ws(L, n, precision, locality, prune=1):
    out = ctypes.c_size_t(0)
    o = rsc.rsc_knn_opts(precision, 0, 0, 0, None, None, locality, prune)
    assert L.rsc_knn_workspace_size(n, 50, 15, 0, ctypes.byref(o), ctypes.byref(out)) == rsc.RSC_OK
    return out.value


def test_locality_workspace(L):
    # the ordering adds a permutation (4 bytes per row) and its k-means scratch
    # to the BF16 workspace; automatic from 16,384 rows; no effect on FP32
    n = 100_000
    off, on, auto = (_ws(L, n, 1, v) for v in (1, 2, 0))
    assert on >= off + 4 * n and auto == on
    assert _ws(L, 10_000, 1, 0) == _ws(L, 10_000, 1, 1) < _ws(L, 10_000, 1, 2)
    assert _ws(L, n, 0, 2) == _ws(L, n, 0, 1)


def test_prune_workspace(L):
    # pruning saves every (row, part) list (keys and ids: 8 bytes per candidate;
    # k = 15 keeps 2 parts x 16 = 32 candidates per row) and the kept-tile
    # lists on top of the ordered workspace
    n = 100_000
    base, pruned, auto = _ws(L, n, 1, 2, 1), _ws(L, n, 1, 2, 2), _ws(L, n, 1, 2, 0)
    assert pruned >= base + 8 * n * 32 and auto == pruned
    assert _ws(L, n, 1, 1, 0) == _ws(L, n, 1, 1, 1)      # no ordering: automatic pruning stays off


def test_connectivities_argument_errors(L):
    fake = ctypes.c_void_p(256)
    assert L.rsc_connectivities(None, fake, 10, 5, fake, fake, fake, 100, None, None, fake, 1 << 30, None) \
        == rsc.RSC_ERR_INVALID_ARG
    assert L.rsc_connectivities(fake, fake, 10, 0, fake, fake, fake, 100, None, None, fake, 1 << 30, None) \
        == rsc.RSC_ERR_INVALID_ARG
    assert L.rsc_connectivities(fake, fake, 10, 5, fake, fake, fake, 100, None, None, None, 0, None) \
        == rsc.RSC_ERR_WORKSPACE


def test_autotune_table_save_load_roundtrip(L, tmp_path):
    rsc.rsc_autotune_clear()
    src = tmp_path / "tuned.txt"
    src.write_text("# kind precision metric d k k_cross log2n db_splits candidates tc_parts\n"
                   "0 1 0 50 15 0 19 2 0 4\n"
                   "1 1 0 50 15 3 21 0 0 2\n")
    rsc.rsc_autotune_load(str(src))
    # an automatic rsc_knn request of that key now plans with 2 database splits
    auto = rsc.rsc_knn_workspace_size(600_000, 50, 15, "euclidean", "bf16")
    explicit = ctypes.c_size_t(0)
    o = rsc.rsc_knn_opts(1, 0, 2, 4, None, None)
    assert L.rsc_knn_workspace_size(600_000, 50, 15, 0, ctypes.byref(o), ctypes.byref(explicit)) == 0
    assert auto == explicit.value
    out = tmp_path / "saved.txt"
    rsc.rsc_autotune_save(str(out))
    rows = [l.split() for l in out.read_text().splitlines() if not l.startswith("#")]
    # the saved table carries the pipeline stages as an 11th column (0: automatic)
    assert sorted(rows) == sorted([l.split() + ["0"] for l in src.read_text().splitlines() if not l.startswith("#")])
    v2 = tmp_path / "v2.txt"
    v2.write_text("0 1 0 50 15 0 18 1 0 2 4\n")
    rsc.rsc_autotune_load(str(v2))
    rsc.rsc_autotune_save(str(out))
    assert ["0", "1", "0", "50", "15", "0", "18", "1", "0", "2", "4"] in \
        [l.split() for l in out.read_text().splitlines() if not l.startswith("#")]
    for line in ("0 1 0 50 15 0 19 2 0 3\n",       # tc_parts 3 is not a valid choice
                 "0 1 0 50 15 0 19 2 0 2 7\n"):    # at most 6 stages
        bad = tmp_path / "bad.txt"
        bad.write_text(line)
        with pytest.raises(rsc.RscError):
            rsc.rsc_autotune_load(str(bad))
    rsc.rsc_autotune_clear()


def _static_limit(k):
    """Largest n whose connectivities workspace fits the 32 MiB static scratch."""
    lo, hi = 1, 10 ** 7
    while lo < hi:
        m = (lo + hi + 1) // 2
        if rsc.rsc_connectivities_workspace_size(m, k) <= 32 << 20:
            lo = m
        else:
            hi = m - 1
    return lo


@pytest.mark.parametrize("k", [15, 30])
def test_static_connectivities_rejects_before_any_gpu_work(L, k):
    # argument and size checks return before the scratch address is looked
    # up; the pointers are never dereferenced
    fake = ctypes.c_void_p(256)
    n = _static_limit(k) + 1
    cap = rsc.rsc_connectivities_max_nnz(n, k)
    st = L.rsc_connectivities_static(fake, fake, n, k, fake, fake, fake, cap, None, None, None)
    assert st == rsc.RSC_ERR_WORKSPACE
    assert b"32 MiB" in L.rsc_last_error()
    for bad_k in (0, 257):
        assert L.rsc_connectivities_static(fake, fake, 100, bad_k, fake, fake, fake, 10 ** 6, None, None,
                                           None) == rsc.RSC_ERR_INVALID_ARG
    # a capacity below the 2 n (k - 1) bound is refused (the call never synchronises)
    assert L.rsc_connectivities_static(fake, fake, 100, k, fake, fake, fake, rsc.rsc_connectivities_max_nnz(100, k) - 1,
                                       None, None, None) == rsc.RSC_ERR_INVALID_ARG


def test_connectivities_k_range(L):
    fake = ctypes.c_void_p(256)
    for bad_k in (0, 257):
        assert L.rsc_connectivities(fake, fake, 10, bad_k, fake, fake, fake, 100, None, None, fake, 1 << 30,
                                    None) == rsc.RSC_ERR_INVALID_ARG
    assert rsc.rsc_connectivities_max_nnz(10, 1) == 0     # k = 1: every row lists only itself


@pytest.mark.parametrize("spread,min_dist", [(1.0, 0.5), (1.0, 0.1), (2.0, 0.3), (1.0, 0.0), (0.5, 1.0)])
def test_umap_find_ab_matches_scipy_curve_fit(L, spread, min_dist):
    optimize = pytest.importorskip("scipy.optimize")
    import numpy as np
    x = np.linspace(0, 3 * spread, 300)
    y = np.where(x < min_dist, 1.0, np.exp(-(x - min_dist) / spread))
    (sa, sb), _ = optimize.curve_fit(lambda x, a, b: 1.0 / (1.0 + a * x ** (2 * b)), x, y)
    a, b = rsc.rsc_umap_find_ab(spread, min_dist)
    assert a == pytest.approx(sa, rel=1e-4) and b == pytest.approx(sb, rel=1e-4)
    if (spread, min_dist) == (1.0, 0.5):
        assert a == pytest.approx(0.583, abs=5e-4) and b == pytest.approx(1.334, abs=5e-4)


def test_umap_argument_errors(L):
    import ctypes
    with pytest.raises(rsc.RscError):
        rsc.rsc_umap_find_ab(0.0, 0.5)
    with pytest.raises(rsc.RscError):
        rsc.rsc_umap_find_ab(1.0, -0.1)
    assert rsc.rsc_umap_workspace_size(1000, 20000, 2) > 20000 * 4 + 2 * 1000 * 2 * 4
    assert rsc.rsc_umap_workspace_size(1000, 0, 3) >= 2 * 1000 * 4 * 4
    for args in ((0, 10, 2), (10, -1, 2), (10, 10, 0), (10, 10, 5), (2**31, 10, 2)):
        with pytest.raises(rsc.RscError):
            rsc.rsc_umap_workspace_size(*args)
    fake = ctypes.c_void_p(4096)
    def call(n=10, nnz=10, dim=2, ws=1 << 20, **kw):
        o = rsc.rsc_umap_opts(kw.get("a", 0.58), kw.get("b", 1.33), kw.get("gamma", 1.0), kw.get("lr", 1.0),
                              kw.get("r", 5), kw.get("N", 200), kw.get("first", 0), kw.get("last", 0), 0, None)
        return L.rsc_umap_layout(fake, fake, fake, n, nnz, dim, fake, ctypes.byref(o), kw.get("wsp", fake), ws)
    bad = [dict(n=0), dict(dim=5), dict(nnz=-1), dict(N=0), dict(N=100001), dict(first=5, last=4),
           dict(last=201), dict(first=-1), dict(r=-1), dict(r=65), dict(a=float("nan")), dict(lr=float("inf"))]
    for kw in bad:
        assert call(**kw) == rsc.RSC_ERR_INVALID_ARG, kw
    assert call(ws=16) == rsc.RSC_ERR_WORKSPACE
    assert call(wsp=None) == rsc.RSC_ERR_WORKSPACE


def test_edistance_argument_errors(L):
    import numpy as np
    off = np.array([0, 10, 25, 40], np.int64)
    assert rsc.rsc_edistance_workspace_size(40, 50, off) > 40 * 2 * 384
    pairs = np.array([[0, 0], [0, 2]], np.int32)
    assert rsc.rsc_edistance_workspace_size(40, 50, off, pairs) > rsc.rsc_edistance_workspace_size(40, 50, off) - 1
    bad = [
        (40, 0, off, None, rsc.RSC_ERR_INVALID_ARG),                                # d = 0
        (40, 59, off, None, rsc.RSC_ERR_UNSUPPORTED),                               # d > 58
        (0, 50, off, None, rsc.RSC_ERR_INVALID_ARG),                                # no rows
        (40, 50, np.array([1, 10], np.int64), None, rsc.RSC_ERR_INVALID_ARG),       # offsets[0] != 0
        (40, 50, np.array([0, 10, 5], np.int64), None, rsc.RSC_ERR_INVALID_ARG),    # decreasing
        (40, 50, np.array([0, 0], np.int64), None, rsc.RSC_ERR_INVALID_ARG),        # no cells
        (40, 50, off, np.array([[1, 0]], np.int32), rsc.RSC_ERR_INVALID_ARG),       # a > b
        (40, 50, off, np.array([[0, 3]], np.int32), rsc.RSC_ERR_INVALID_ARG),       # b >= G
    ]
    for n, d, o, p, code in bad:
        with pytest.raises(rsc.RscError) as e:
            rsc.rsc_edistance_workspace_size(n, d, o, p)
        assert e.value.status == code, (n, d, o, p)


def test_knn_descent_argument_errors(L):
    size = rsc.rsc_knn_descent_workspace_size(1000, 50, 15)
    # lists, masks, 2 n R + n C slots (R = 32, C = 64), counters
    assert size >= 1000 * (15 * 8 + 16 + (2 * 32 + 64) * 8)
    assert rsc.rsc_knn_descent_workspace_size(2000, 50, 15) > size
    bad = [((1, 5, 2), {}), ((100, 0, 15), {}), ((100, 5, 1), {}), ((10, 5, 11), {}), ((100, 5, 65), {}),
           ((100, 5, 8), {"sample": 9}), ((100, 5, 8), {"rev_slots": 48}), ((100, 5, 8), {"cand_slots": 128}),
           ((100, 5, 8), {"max_iters": 65}), ((100, 5, 8), {"delta": -0.5}), ((100, 5, 8), {"delta": float("nan")})]
    for args, kw in bad:
        with pytest.raises(rsc.RscError) as e:
            rsc.rsc_knn_descent_workspace_size(*args, rsc.nnd_opts(**kw))
        assert e.value.status == rsc.RSC_ERR_INVALID_ARG, (args, kw)
    # the join's staged rows must fit in shared memory
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_knn_descent_workspace_size(1000, 4096, 64, rsc.nnd_opts(rev_slots=64))
    assert e.value.status == rsc.RSC_ERR_UNSUPPORTED
    # no workspace: refused on the host, before any launch
    st = L.rsc_knn_descent(ctypes.c_void_p(16), 100, 5, 8, None, ctypes.c_void_p(16), ctypes.c_void_p(16), None,
                           ctypes.byref(rsc.nnd_opts()), None, 0)
    assert st == rsc.RSC_ERR_WORKSPACE


def test_leiden_argument_errors(L):
    a = rsc.rsc_leiden_workspace_size(1000, 20000)
    assert a > 20000 * (4 + 8) * 3 and rsc.rsc_leiden_workspace_size(2000, 40000) > a
    for args in ((0, 10), (-1, 10), (10, -1)):
        with pytest.raises(rsc.RscError) as e:
            rsc.rsc_leiden_workspace_size(*args)
        assert e.value.status == rsc.RSC_ERR_INVALID_ARG
    o = rsc.leiden_opts()
    vp = ctypes.c_void_p(256)
    K, q = ctypes.c_int64(0), ctypes.c_double(0)
    # refused on the host before any launch: no workspace, bad options, NULL pointers
    assert L.rsc_leiden(vp, vp, vp, 10, 20, None, vp, ctypes.byref(K), ctypes.byref(q), ctypes.byref(o),
                        None, 0) == rsc.RSC_ERR_WORKSPACE
    for bad in (rsc.leiden_opts(resolution=-1.0), rsc.leiden_opts(n_iterations=-2), rsc.leiden_opts(max_rounds=-1)):
        assert L.rsc_leiden(vp, vp, vp, 10, 20, None, vp, None, None, ctypes.byref(bad), vp, 1 << 30) == \
            rsc.RSC_ERR_INVALID_ARG
    assert L.rsc_leiden(None, vp, vp, 10, 20, None, vp, None, None, ctypes.byref(o), vp, 1 << 30) == \
        rsc.RSC_ERR_INVALID_ARG
