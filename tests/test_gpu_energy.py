"""lrq_spectral_energy (rho_r, Sec. 5 "When does low-rank work?") on the GPU
against the oracle's full-spectrum definition.

For a PSD Q the trace equals the sum of all eigenvalues, so the GPU value
(top r eigenvalues from lrq_truncate over an FP64 trace) and the oracle's
(LAPACK's whole spectrum) differ by rounding only: 1e-9 absolute on rho (the
truncation's eigenvalues are within 1e-9 ||Q|| and the trace is at least
||Q||).  The trace of a unit-weight Laplacian is an integer and exact."""
import numpy as np
import pytest

import oracle
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


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


def _rho(lrq, Qm, r):
    tr = lrq.truncate(Qm, r, want_c64=False)
    out = lrq.spectral_energy(Qm, tr["lam"])
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    return float(out["rho"].item()), float(out["trace"].item())


def test_dense_psd_matches_oracle(lrq):
    n = 500
    V = I.factor(n, 3, seed=70, scales=(4.0, 2.0, 1.0))
    G = I.complex_gaussian((n, n), seed=71)
    Q = V @ V.conj().T + 0.02 * (G @ G.conj().T) / n
    Qd = _dev(Q, np.complex128)
    for r in (1, 3, 6):
        rho, tr = _rho(lrq, lrq.dense_matrix(Qd), r)
        assert abs(tr - np.trace(Q).real) <= 1e-12 * abs(np.trace(Q).real)
        assert abs(rho - oracle.spectral_energy(Q, r)) <= 1e-9


@pytest.mark.parametrize("weighted", [False, True])
def test_laplacian_matches_oracle(lrq, weighted):
    rowptr, colidx, _ = I.sbm_graph(1500, 4.0, 8.0, seed=72)
    w = None
    if weighted:
        rows = np.repeat(np.arange(1500), np.diff(rowptr))
        lo, hi = np.minimum(rows, colidx), np.maximum(rows, colidx)
        w = I.rng(73).uniform(0.5, 2.0, 4096)[(lo * 7919 + hi * 104729) % 4096]
    keep = (_dev(rowptr, np.int32), _dev(colidx, np.int32), None if w is None else _dev(w, np.float64))
    Qm = lrq.laplacian_matrix(*keep)  # the struct holds raw device pointers: keep the tensors alive
    rho, tr = _rho(lrq, Qm, 2)
    L = oracle.laplacian_dense(rowptr, colidx, w)
    if not weighted:
        assert tr == float(np.count_nonzero(np.repeat(np.arange(1500), np.diff(rowptr)) != colidx))
    assert abs(tr - np.trace(L).real) <= 1e-12 * np.trace(L).real
    assert abs(rho - oracle.spectral_energy(L, 2)) <= 1e-9
    assert rho > 0.98


def test_torus_closed_form(lrq):
    k1, k2 = 16, 18
    rowptr, colidx = I.torus_graph(k1, k2)
    keep = (_dev(rowptr, np.int32), _dev(colidx, np.int32))
    Qm = lrq.laplacian_matrix(*keep)
    a = np.arange(k1)[:, None]
    b = np.arange(k2)[None, :]
    ev = np.sort((4 - 2 * np.cos(2 * np.pi * a / k1) - 2 * np.cos(2 * np.pi * b / k2)).ravel())[::-1]
    for r in (1, 2, 5):
        rho, tr = _rho(lrq, Qm, r)
        assert tr == 4 * k1 * k2
        assert abs(rho - (1 - ev[:r].sum() / (4 * k1 * k2))) <= 1e-10


def test_edgeless_graph_and_errors(lrq):
    rowptr = np.zeros(11, np.int32)
    colidx = np.zeros(0, np.int32)
    lam = _dev(np.zeros(2), np.float64)
    keep = (_dev(rowptr, np.int32), _dev(colidx, np.int32))
    out = lrq.spectral_energy(lrq.laplacian_matrix(*keep), lam)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    assert float(out["trace"].item()) == 0.0 and float(out["rho"].item()) == 0.0
    # a malformed graph
    rp, ci = I.torus_graph(4, 5)
    bad = np.array(ci)
    bad[3] = 99
    keep = (_dev(rp, np.int32), _dev(bad, np.int32))
    out = lrq.spectral_energy(lrq.laplacian_matrix(*keep), lam)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == lrq.LRQ_EINVAL
    # a negative trace (not PSD)
    Qd = _dev(-np.eye(6), np.complex128)
    out = lrq.spectral_energy(lrq.dense_matrix(Qd), lam)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == lrq.LRQ_EINVAL
