"""lrq_rank1_sweep (Sec. 2.5, Algorithm 1) on the GPU against the oracle.

The rank-1 optimum |q^H z|^2 is unique and compared within 1e-9 relative
(FP64 prefix sums vs the oracle's full re-evaluation of every state); the
codes must score that value.  The sweep scored on a graph's cut is integer
work: the best cut must equal the oracle's exactly, and the returned codes
must have that cut."""
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


def _run(lrq, q, K, rowptr=None, colidx=None):
    qd = torch.from_numpy(np.ascontiguousarray(q, dtype=np.complex128)).to(DEV)
    rp = None if rowptr is None else torch.from_numpy(np.asarray(rowptr, dtype=np.int32)).to(DEV)
    ci = None if colidx is None else torch.from_numpy(np.asarray(colidx, dtype=np.int32)).to(DEV)
    out = lrq.rank1_sweep(qd, K, rp, ci)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    return out


@pytest.mark.parametrize("n,K,seed", [(1, 3, 1), (7, 2, 2), (3000, 3, 3), (2048, 5, 4), (4097, 8, 5),
                                      (5000, 64, 6), (2049, 2, 7)])
def test_rank1_optimum_matches_oracle(lrq, n, K, seed):
    q = I.complex_gaussian((n,), seed=seed)
    out = _run(lrq, q, K)
    f_ref, _ = oracle.rank1_sweep(q, K)
    f = float(out["f"].item())
    z = out["z"].cpu().numpy()
    assert abs(f - f_ref) <= 1e-9 * f_ref
    assert abs(oracle.objective(q[:, None], K, z) - f) <= 1e-9 * f
    if K ** n <= 200000:
        f_bf, _ = oracle.bruteforce(q[:, None], K)
        assert abs(f_bf - f) <= 1e-9 * f_bf


def test_repeated_entries_and_zeros(lrq):
    # many equal entries (ties broken by index on both sides) and zero rows
    g = I.rng(8)
    q = np.repeat(I.complex_gaussian((40,), seed=9), 50)
    q[g.choice(q.size, 100, replace=False)] = 0
    out = _run(lrq, q, 3)
    f_ref, _ = oracle.rank1_sweep(q, 3)
    assert abs(float(out["f"].item()) - f_ref) <= 1e-9 * f_ref


@pytest.mark.parametrize("K", [2, 3, 4])
def test_sweep_cut_matches_oracle(lrq, K):
    rowptr, colidx, _ = I.sbm_graph(1500, 4.0, 8.0, seed=10 + K)
    q = I.complex_gaussian((1500,), seed=20 + K)
    out = _run(lrq, q, K, rowptr, colidx)
    best, _, cuts = oracle.rank1_sweep_cut(q, K, rowptr, colidx)
    assert int(out["cut"].item()) == best
    assert oracle.cut_count(rowptr, colidx, out["zcut"].cpu().numpy()) == best


def test_sweep_cut_bipartite_torus(lrq):
    k1, k2 = 30, 40
    rowptr, colidx = I.torus_graph(k1, k2)
    a = np.arange(k1)[:, None]
    b = np.arange(k2)[None, :]
    q = ((a + b) % 2 * 2 - 1).ravel().astype(np.complex128)
    out = _run(lrq, q, 2, rowptr, colidx)
    assert int(out["cut"].item()) == len(colidx) // 2


def test_non_finite_input_is_reported(lrq):
    q = I.complex_gaussian((100,), seed=30)
    q[5] = np.nan
    qd = torch.from_numpy(q).to(DEV)
    out = lrq.rank1_sweep(qd, 3)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == lrq.LRQ_EINVAL


@pytest.mark.slow
def test_sbm_million_rank1_path(lrq):
    # rank-1 truncation of the 10^6-vertex SBM Laplacian, the exact rank-1
    # optimum and the best cut along its sweep
    n = 1_000_000
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=1)
    rp = torch.from_numpy(rowptr).to(DEV)
    ci = torch.from_numpy(colidx).to(DEV)
    tr = lrq.truncate(lrq.laplacian_matrix(rp, ci), 1, max_iter=1000, want_c64=False)
    q = tr["V"][:, 0].contiguous()
    out = lrq.rank1_sweep(q, 3, rp, ci)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    zc = out["zcut"].cpu().numpy()
    assert oracle.cut_count(rowptr, colidx, zc) == int(out["cut"].item())
    z = out["z"].cpu().numpy()
    assert int(out["cut"].item()) >= oracle.cut_count(rowptr, colidx, z)
    qh = q.cpu().numpy()
    assert abs(oracle.objective(qh[:, None], 3, z) - float(out["f"].item())) <= 1e-9 * float(out["f"].item())


def test_two_eigvec_q_matches_oracle(lrq):
    # q = u_1 + i u_2 from the GPU truncation's V and lambda, against the
    # oracle's formula on the same inputs (one FP64 division per entry)
    n = 5001
    V = I.complex_gaussian((n, 3), seed=40)
    for lam in ([4.0, 2.5, 1.0], [3.0, -1.0, 0.5], [7.0, 0.0, 0.0]):
        Vd = torch.from_numpy(V).to(DEV)
        ld = torch.tensor(lam, dtype=torch.float64, device=DEV)
        q = lrq.two_eigvec_q(Vd, ld).cpu().numpy()
        q_ref = oracle.two_eigvec_q(V, np.array(lam))
        assert np.abs(q - q_ref).max() <= 1e-15 * np.abs(q_ref).max()


def test_two_eigvec_sweep_on_gpu_truncation(lrq):
    # the whole rank-1 path for K = 3 on a graph: GPU rank-2 truncation, q,
    # sweep with every state's cut; against the oracle's sweep on the same q
    rowptr, colidx, _ = I.sbm_graph(20000, 4.0, 8.0, seed=41)
    rp = torch.from_numpy(np.asarray(rowptr, np.int32)).to(DEV)
    ci = torch.from_numpy(np.asarray(colidx, np.int32)).to(DEV)
    tr = lrq.truncate(lrq.laplacian_matrix(rp, ci), 2, want_c64=False)
    q = lrq.two_eigvec_q(tr["V"], tr["lam"])
    out = lrq.rank1_sweep(q, 3, rp, ci)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    qh = q.cpu().numpy()
    f_ref, _ = oracle.rank1_sweep(qh, 3)
    assert abs(float(out["f"].item()) - f_ref) <= 1e-9 * f_ref
    assert set(np.unique(out["zcut"].cpu().numpy())) == {0, 1, 2}
    assert int(out["cut"].item()) == oracle.cut_count(rowptr, colidx, out["zcut"].cpu().numpy())
