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
