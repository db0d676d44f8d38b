"""lrq_rescore_no_alloc: the re-scoring entry point for callers that cannot
allocate device memory (it uses the library's own fixed 4 MiB scratch array
instead of a caller workspace).

Checked through the C ABI against lrq_rescore on the same inputs, on two
calls in a row with different inputs (the shared scratch keeps the previous
call's contents, which must not leak into the next result), with the
re-scoring tolerance of the other tests: f within 1e-9 relative, identical
codes and winner.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2602_20376_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lrq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20376_gb300 import lrq as L
    L.load()
    return L


def _run_both(lrq, V, K, C, idx):
    Vd = torch.from_numpy(V).to(DEV)
    Cd = torch.from_numpy(C).to(DEV)
    idxd = torch.from_numpy(idx).to(DEV)
    m, n = idx.size, V.shape[0]
    ref = lrq.rescore(Vd, K, Cd, idxd, want_z=True)
    f = torch.empty(m, dtype=torch.float64, device=DEV)
    z = torch.empty((m, n), dtype=torch.uint8, device=DEV)
    best = torch.empty(1, dtype=torch.int64, device=DEV)
    best_f = torch.empty(1, dtype=torch.float64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    lrq.lrq_rescore_no_alloc(Vd, K, Cd, idxd, f, z, best, best_f, status)
    torch.cuda.synchronize()
    lrq.check_status(ref["dev_status"], "lrq_rescore")
    lrq.check_status(status, "lrq_rescore_no_alloc")
    return ref, dict(f=f, z=z, best=best, best_f=best_f)


def test_no_alloc_rescore_matches_workspace_rescore_twice(lrq):
    cases = [(300000, 4, 3, 64, 11), (5000, 3, 8, 17, 12)]
    for n, r, K, m, seed in cases:  # two calls in a row, different inputs
        V = I.factor(n, r, seed=seed, scales=np.linspace(2.0, 0.5, r), dtype=np.complex64)
        C = I.directions(1000, r, seed=seed + 1)
        idx = I.rng(seed).choice(1000, m, replace=False).astype(np.int64)
        ref, got = _run_both(lrq, V, K, C, idx)
        f_ref = ref["f"].cpu().numpy()
        f = got["f"].cpu().numpy()
        assert np.all(np.abs(f - f_ref) <= 1e-9 * f_ref)
        assert torch.equal(got["z"], ref["z"])
        assert int(got["best"].item()) == int(ref["best"].item())
        assert abs(float(got["best_f"].item()) - float(ref["best_f"].item())) <= 1e-9 * float(ref["best_f"].item())


def test_no_alloc_rescore_rejects_sizes_beyond_its_scratch(lrq):
    # m = 4096 at n = 2^20 needs more than the fixed 4 MiB: refused on the host
    n, r, m = 1 << 20, 4, 4096
    assert lrq.lrq_rescore_workspace_size(n, r, m) > 4 * 1024 * 1024
    V = torch.zeros((n, r), dtype=torch.complex64, device=DEV)
    C = torch.zeros((m, r), dtype=torch.complex64, device=DEV)
    idx = torch.arange(m, dtype=torch.int64, device=DEV)
    f = torch.empty(m, dtype=torch.float64, device=DEV)
    best = torch.empty(1, dtype=torch.int64, device=DEV)
    best_f = torch.empty(1, dtype=torch.float64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    with pytest.raises(lrq.LrqError) as ei:
        lrq.lrq_rescore_no_alloc(V, 3, C, idx, f, None, best, best_f, status)
    assert ei.value.status == lrq.LRQ_EUNSUPPORTED
    assert "4 MiB" in str(ei.value)


_SECOND_CONTEXT = r'''
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2602_20376_gb300 import inputs as I, lrq
L = lrq.load()
n, r, K, m = 20000, 4, 3, 16
V = I.factor(n, r, seed=21, scales=(2.0, 1.5, 1.0, 0.5), dtype=np.complex64)
C = I.directions(500, r, seed=22)
idx = I.rng(23).choice(500, m, replace=False).astype(np.int64)
dev = "cuda:0"
Vd, Cd, idxd = torch.from_numpy(V).to(dev), torch.from_numpy(C).to(dev), torch.from_numpy(idx).to(dev)
ref = lrq.rescore(Vd, K, Cd, idxd, want_z=True)
torch.cuda.synchronize()
lrq.check_status(ref["dev_status"], "lrq_rescore")
f_ref, z_ref, best_ref = ref["f"].cpu().numpy(), ref["z"].cpu().numpy(), int(ref["best"].item())


def primary_call():
    f = torch.empty(m, dtype=torch.float64, device=dev)
    z = torch.empty((m, n), dtype=torch.uint8, device=dev)
    b = torch.empty(1, dtype=torch.int64, device=dev)
    bf = torch.empty(1, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    lrq.lrq_rescore_no_alloc(Vd, K, Cd, idxd, f, z, b, bf, st)
    torch.cuda.synchronize()
    lrq.check_status(st, "lrq_rescore_no_alloc")
    return f.cpu().numpy(), z.cpu().numpy(), int(b.item())


def check(f, z, b):
    assert np.all(np.abs(f - f_ref) <= 1e-9 * f_ref), np.abs(f - f_ref).max()
    assert np.array_equal(z, z_ref) and b == best_ref


check(*primary_call())  # the primary context's scratch address is cached
# a second context of the same device, created and made current through the
# driver API, with its own buffers: the library must use this context's
# address of its scratch array, not the one cached for the primary context
cu = ctypes.CDLL("libcuda.so.1")
U64 = ctypes.c_uint64
assert cu.cuInit(0) == 0
devh = ctypes.c_int()
assert cu.cuDeviceGet(ctypes.byref(devh), 0) == 0
ctx = ctypes.c_void_p()
assert cu.cuCtxCreate_v2(ctypes.byref(ctx), 0, devh) == 0
bufs = []


def alloc(nbytes):
    p = U64()
    assert cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nbytes)) == 0
    bufs.append(p)
    return p.value


def upload(arr):
    arr = np.ascontiguousarray(arr)
    p = alloc(arr.nbytes)
    assert cu.cuMemcpyHtoD_v2(U64(p), arr.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(arr.nbytes)) == 0
    return p


def download(p, shape, dtype):
    out = np.empty(shape, dtype=dtype)
    assert cu.cuMemcpyDtoH_v2(out.ctypes.data_as(ctypes.c_void_p), U64(p), ctypes.c_size_t(out.nbytes)) == 0
    return out


pV, pC, pI = upload(V), upload(C), upload(idx)
pf, pz, pb, pbf = alloc(8 * m), alloc(m * n), alloc(8), alloc(8)
pst = upload(np.zeros(1, dtype=np.int32))
rc = L.lrq_rescore_no_alloc(pV, n, r, K, pC, C.shape[0], pI, m, pf, pz, pb, pbf, pst, None)
assert rc == 0, (rc, L.lrq_last_error())
assert cu.cuCtxSynchronize() == 0
assert int(download(pst, 1, np.int32)[0]) == 0
check(download(pf, m, np.float64), download(pz, (m, n), np.uint8), int(download(pb, 1, np.int64)[0]))
for p in bufs:
    assert cu.cuMemFree_v2(p) == 0
assert cu.cuCtxDestroy_v2(ctx) == 0  # the primary context is current again
check(*primary_call())
print("second context ok")
'''


def test_no_alloc_rescore_in_a_second_context(lrq):
    # the scratch array's device address belongs to a context: a caller in its
    # own driver-API context gets that context's address (checked in a fresh
    # process, so that this process's contexts are not disturbed)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _SECOND_CONTEXT, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "second context ok" in r.stdout
