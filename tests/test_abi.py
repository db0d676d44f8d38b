"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/lrq.h declares, and rejects invalid arguments on the host
before launching anything."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_20376_gb300 import build, lrq
    build.build()
    return lrq.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "lrq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lrq_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("lrq_sample_score", "lrq_rescore", "lrq_sample_directions", "lrq_cut_count"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2602_20376_gb300 import lrq
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in lrq.exported_symbols()


def test_status_strings(lib):
    from paper_2602_20376_gb300 import lrq
    assert lrq.lrq_abi_version() == 1
    for s in range(7):
        assert lrq.lrq_status_string(s).startswith("LRQ_")
    assert "UNKNOWN" in lrq.lrq_status_string(99)


def _call_score(lib, **kw):
    P = ctypes.c_void_p
    a = dict(V=P(256), n=1000, r=4, K=3, C=P(512), gen=0, seed=0, S=100, mode=1, top_m=10,
             scores=None, idx=P(1024), f=P(2048), ws=P(4096), ws_bytes=1 << 30, status=P(8192), stream=None)
    a.update(kw)
    return lib.lrq_sample_score(a["V"], a["n"], a["r"], a["K"], a["C"], a["gen"], a["seed"], a["S"], a["mode"],
                                a["top_m"], a["scores"], a["idx"], a["f"], a["ws"], a["ws_bytes"], a["status"],
                                a["stream"])


@pytest.mark.parametrize("kw,code", [
    (dict(n=0), 1), (dict(r=0), 1), (dict(r=9), 1), (dict(K=1), 1), (dict(K=65), 1),
    (dict(S=0), 1), (dict(top_m=0), 1), (dict(top_m=101), 1), (dict(top_m=513, S=1000), 1),
    (dict(mode=7), 1), (dict(K=9), 2), (dict(V=None), 1), (dict(status=None), 1),
    (dict(ws=None), 6), (dict(ws_bytes=10), 6), (dict(ws=ctypes.c_void_p(4096 + 16)), 6),
])
def test_sample_score_rejects_bad_arguments_on_host(lib, kw, code):
    # invalid arguments return before any launch (no GPU is touched)
    assert _call_score(lib, **kw) == code
    assert len(lib.lrq_last_error()) > 0


def test_rescore_and_cut_reject_bad_arguments(lib):
    P = ctypes.c_void_p
    args = [P(256), 100, 4, 3, P(512), 10, P(1024), 4, P(2048), None, P(4096), P(4100), P(8192), 1 << 20, P(9000),
            None]
    bad_m = list(args)
    bad_m[7] = 0
    assert lib.lrq_rescore(*bad_m) == 1
    bad_k = list(args)
    bad_k[3] = 1
    assert lib.lrq_rescore(*bad_k) == 1
    bad_ws = list(args)
    bad_ws[13] = 1
    assert lib.lrq_rescore(*bad_ws) == 6
    assert lib.lrq_cut_count(None, None, 10, None, P(256), None) == 1
    assert lib.lrq_sample_directions(0, -1, 4, P(256), None) == 1
    assert lib.lrq_sample_directions(0, 10, 0, P(256), None) == 1
    assert lib.lrq_set_timing_events(P(256), None) == 1


def test_workspace_queries(lib):
    from paper_2602_20376_gb300 import lrq
    a = lrq.lrq_sample_score_workspace_size(1 << 20, 4, 3, 1 << 16, lrq.LRQ_MODE_TC, 64)
    b = lrq.lrq_sample_score_workspace_size(1 << 20, 4, 3, 1 << 16, lrq.LRQ_MODE_FP32, 64)
    assert a > b > 0
    assert lrq.lrq_rescore_workspace_size(1 << 20, 4, 64) > 0
    with pytest.raises(lrq.LrqError):
        lrq.lrq_sample_score_workspace_size(1 << 20, 4, 9, 1 << 16, lrq.LRQ_MODE_TC, 64)


def test_mlp_batch_limit(lib):
    # the MLP's GEMMs put the batch rows on the grid's y axis, 32 per block
    P = ctypes.c_void_p
    dummy = P(256)
    args = (dummy, 24, 65535 * 32 + 1, dummy, dummy, dummy, dummy, 0, None)
    assert lib.lrq_mlp_forward(*args) == 2  # LRQ_EUNSUPPORTED
    assert lib.lrq_mlp_backward(dummy, 24, 65535 * 32 + 1, dummy, dummy, dummy, dummy, dummy, dummy, 0, None) == 2


def test_rescore_scratch_sizes(lib):
    # the re-scoring scratch is m x chunks x 16 doubles with at most 65536
    # coordinates per chunk: m = 64 fits the no-alloc entry point's fixed
    # 4 MiB up to n = 2^25, m = 4096 at n = 2^20 does not
    from paper_2602_20376_gb300 import lrq
    assert lrq.lrq_rescore_workspace_size(1 << 25, 4, 64) <= 4 * 1024 * 1024
    assert lrq.lrq_rescore_workspace_size((1 << 25) + 65536, 4, 64) > 4 * 1024 * 1024
    assert lrq.lrq_rescore_workspace_size(1 << 20, 4, 4096) > 4 * 1024 * 1024
    # independent of the rank: the partials are sized for the largest rank
    assert lrq.lrq_rescore_workspace_size(1 << 20, 1, 64) == lrq.lrq_rescore_workspace_size(1 << 20, 8, 64)


@pytest.mark.parametrize("n,r,K,budget,code", [
    (0, 2, 3, 0.0, 1), (12, 0, 3, 0.0, 1), (12, 2, 1, 0.0, 1),   # invalid
    (513, 1, 3, 0.0, 2), (6, 5, 3, 0.0, 2), (12, 2, 9, 0.0, 2),  # beyond the enumerator's limits
    (12, 2, 3, 1e5, 2),                                           # 2 * 12^5 = 497664 > budget
    (200, 3, 3, 0.0, 2),                                          # r n^(2r+1) > the default 1e12
])
def test_enumerate_rejects_bad_arguments_on_host(lib, n, r, K, budget, code):
    P = ctypes.c_void_p
    assert lib.lrq_enumerate(P(256), n, r, K, budget, P(512), P(1024), None, P(4096), 1 << 30, P(8192), None) == code
    assert len(lib.lrq_last_error()) > 0


def test_enumerate_workspace_and_null_checks(lib):
    from paper_2602_20376_gb300 import lrq
    assert lrq.lrq_enumerate_workspace_size(12, 2, 3) > 0
    P = ctypes.c_void_p
    assert lib.lrq_enumerate(P(256), 12, 2, 3, 0.0, None, P(1024), None, P(4096), 1 << 30, P(8192), None) == 1
    assert lib.lrq_enumerate(P(256), 12, 2, 3, 0.0, P(512), P(1024), None, P(4096), 16, P(8192), None) == 6


def test_truncate_rejects_bad_arguments_on_host(lib):
    from paper_2602_20376_gb300 import lrq
    P = ctypes.c_void_p
    dense = lrq.LrqMatrix(lrq.LRQ_MATRIX_DENSE_C128, 100, 256, 100, None, None, None, 0)
    csr = lrq.LrqMatrix(lrq.LRQ_MATRIX_CSR_LAPLACIAN, 100, None, 0, 256, 512, None, 600)
    assert lrq.lrq_truncate_workspace_size(dense, 4) > 100 * 4 * 16
    assert lrq.lrq_truncate_workspace_size(csr, 3, 50) > 100 * 50 * 8
    it = ctypes.c_int64(0)

    def call(Q, r=4, tol=0.0, max_iter=0, lam=P(1024), ws_bytes=1 << 30, status=P(8192)):
        return lib.lrq_truncate(ctypes.byref(Q), r, tol, max_iter, 1, None, None, lam, ctypes.byref(it), P(4096),
                                ws_bytes, status, None)
    assert call(dense, r=0) == 1
    assert call(dense, r=9) == 1
    assert call(dense, max_iter=5000) == 1
    assert call(dense, tol=2.0) == 1
    assert call(dense, lam=None) == 1
    assert call(dense, status=None) == 1
    assert call(dense, ws_bytes=64) == 6
    bad_ld = lrq.LrqMatrix(lrq.LRQ_MATRIX_DENSE_C128, 100, 256, 50, None, None, None, 0)
    assert call(bad_ld) == 1
    bad_kind = lrq.LrqMatrix(7, 100, 256, 100, None, None, None, 0)
    assert call(bad_kind) == 1
    small = lrq.LrqMatrix(lrq.LRQ_MATRIX_CSR_LAPLACIAN, 3, None, 0, 256, 512, None, 4)
    assert call(small, r=4) == 1  # r > n
    assert lib.lrq_truncate(None, 4, 0.0, 0, 1, None, None, P(1024), None, P(4096), 1 << 30, P(8192), None) == 1


def test_batched_plan_rejects_bad_problems_on_host(lib):
    from paper_2602_20376_gb300 import lrq
    P = ctypes.c_void_p

    def create(probs, top_m=1):
        arr = (lrq.LrqProblem * len(probs))(*probs)
        h = ctypes.c_void_p()
        return lib.lrq_batched_plan_create(arr, len(probs), top_m, ctypes.byref(h))
    ok = lrq.LrqProblem(256, 100, 4, 3, None, 1000, 1)
    for bad in (lrq.LrqProblem(None, 100, 4, 3, None, 1000, 1), lrq.LrqProblem(256, 0, 4, 3, None, 1000, 1),
                lrq.LrqProblem(256, 100, 9, 3, None, 1000, 1), lrq.LrqProblem(256, 100, 4, 1, None, 1000, 1),
                lrq.LrqProblem(256, 100, 4, 3, None, 8193, 1), lrq.LrqProblem(256, 40, 2, 3, 512, 0, 1)):
        assert create([ok, bad]) == 1
    # S = 0 asks for the exact solver: outside its limits the plan is refused
    for bad in (lrq.LrqProblem(256, 100, 4, 3, None, 0, 1), lrq.LrqProblem(256, 40, 2, 12, None, 0, 1),
                lrq.LrqProblem(256, 600, 1, 3, None, 0, 1), lrq.LrqProblem(256, 90, 2, 3, None, 0, 1)):
        assert create([ok, bad]) == 2
    assert create([ok], top_m=17) == 1
    assert create([ok], top_m=0) == 1
    assert lib.lrq_batched_plan_create(None, 1, 1, ctypes.byref(ctypes.c_void_p())) == 1
    assert lib.lrq_graph_launch(None, None) == 1
    assert lib.lrq_sample_score_batched(None, P(256), 1, P(512), P(1024), P(2048), None) == 1


def test_rank1_rejects_bad_arguments_on_host(lib):
    P = ctypes.c_void_p
    args = dict(q=P(256), n=100, K=3, z=P(512), f=P(1024), rp=None, ci=None, nnz=0, cut=None, zc=None, ws=P(4096),
                wsb=1 << 30, st=P(8192))

    def call(**kw):
        a = dict(args)
        a.update(kw)
        return lib.lrq_rank1_sweep(a["q"], a["n"], a["K"], a["z"], a["f"], a["rp"], a["ci"], a["nnz"], a["cut"],
                                   a["zc"], a["ws"], a["wsb"], a["st"], None)
    assert call(n=0) == 1
    assert call(K=1) == 1
    assert call(K=65) == 1
    assert call(q=None) == 1
    assert call(rp=P(300)) == 1          # graph without colidx / outputs
    assert call(wsb=8) == 6


def test_greedy_rejects_bad_arguments_on_host(lib):
    P = ctypes.c_void_p
    args = dict(rp=P(256), ci=P(512), n=100, nnz=400, K=3, z=P(1024), mr=10, cut=None, ws=P(4096), wsb=1 << 30,
                st=P(8192))

    def call(**kw):
        a = dict(args)
        a.update(kw)
        return lib.lrq_greedy_cut(a["rp"], a["ci"], a["n"], a["nnz"], a["K"], a["z"], a["mr"], a["cut"], None,
                                  None, None, a["ws"], a["wsb"], a["st"], None)
    assert call(n=0) == 1
    assert call(K=1) == 1
    assert call(K=9) == 1
    assert call(nnz=-1) == 1
    assert call(mr=-1) == 1
    assert call(z=None) == 1
    assert call(ci=None) == 1
    assert call(wsb=8) == 6
    need = ctypes.c_size_t(0)
    assert lib.lrq_greedy_workspace_size(100, ctypes.byref(need)) == 0 and need.value >= 500
    assert lib.lrq_greedy_workspace_size(0, ctypes.byref(need)) == 1


def test_spectral_energy_rejects_bad_arguments_on_host(lib):
    from paper_2602_20376_gb300 import lrq as L
    P = ctypes.c_void_p
    Q = L.LrqMatrix(L.LRQ_MATRIX_CSR_LAPLACIAN, 100, None, 0, 256, 512, None, 400)
    assert lib.lrq_spectral_energy(None, P(256), 2, P(512), P(1024), P(2048), None) == 1
    assert lib.lrq_spectral_energy(ctypes.byref(Q), P(256), -1, P(512), P(1024), P(2048), None) == 1
    assert lib.lrq_spectral_energy(ctypes.byref(Q), None, 2, P(512), P(1024), P(2048), None) == 1
    assert lib.lrq_spectral_energy(ctypes.byref(Q), P(256), 2, None, P(1024), P(2048), None) == 1
    bad = L.LrqMatrix(7, 100, None, 0, 256, 512, None, 400)
    assert lib.lrq_spectral_energy(ctypes.byref(bad), P(256), 2, P(512), P(1024), P(2048), None) == 1
    dense = L.LrqMatrix(L.LRQ_MATRIX_DENSE_C128, 100, 4096, 50, None, None, None, 0)
    assert lib.lrq_spectral_energy(ctypes.byref(dense), P(256), 2, P(512), P(1024), P(2048), None) == 1


@pytest.mark.parametrize("n,r,K,mode,code", [(0, 4, 8, 1, 1), (64, 9, 8, 1, 1), (64, 4, 1, 1, 1),
                                             (64, 4, 8, 7, 1), (64, 4, 9, 1, 2)])
def test_prepared_create_rejects_bad_arguments_on_host(lib, n, r, K, mode, code):
    h = ctypes.c_void_p()
    assert lib.lrq_prepared_create(n, r, K, mode, ctypes.byref(h)) == code
    assert not h.value


def test_prepared_sizes_and_unprepared_call(lib):
    from paper_2602_20376_gb300 import lrq
    sizes = {}
    for mode in (lrq.LRQ_MODE_FP32, lrq.LRQ_MODE_TC):
        h = ctypes.c_void_p()
        assert lib.lrq_prepared_create(100000, 4, 8, mode, ctypes.byref(h)) == 0
        nb = ctypes.c_size_t(0)
        assert lib.lrq_prepared_size(h, ctypes.byref(nb)) == 0
        sizes[mode] = nb.value
        # scoring before lrq_prepare is refused on the host
        st = lib.lrq_sample_score_prepared(h, ctypes.c_void_p(256), 1, 0, 1024, 4, None, ctypes.c_void_p(256),
                                           ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 30,
                                           ctypes.c_void_p(256), None)
        assert st == lrq.LRQ_EINVAL and "prepare" in lrq.lrq_last_error()
        # a buffer below the size is refused before any launch
        if nb.value:
            st = lib.lrq_prepare(h, ctypes.c_void_p(256), ctypes.c_void_p(256), nb.value - 1, ctypes.c_void_p(256),
                                 None)
            assert st == lrq.LRQ_EWORKSPACE
        lib.lrq_prepared_destroy(h)
    assert sizes[lrq.LRQ_MODE_FP32] == 0
    # the packed coordinate tiles dominate: at least 8 bytes per coordinate
    assert sizes[lrq.LRQ_MODE_TC] >= 8 * 100000
