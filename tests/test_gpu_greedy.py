"""lrq_greedy_cut (greedy Max-K-Cut local search, the refinement step of the
hybrid solver) on the GPU against the oracle.

The search is deterministic integer work: labels, rounds, moves and the
final cut must equal the oracle's exactly."""
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


def _run(lrq, rowptr, colidx, K, z0, max_rounds=1 << 20):
    out = lrq.greedy_cut(_dev(rowptr, np.int32), _dev(colidx, np.int32), K, _dev(z0, np.uint8), max_rounds)
    torch.cuda.synchronize()
    assert int(out["dev_status"].item()) == 0
    return out


def _check(lrq, rowptr, colidx, K, z0, max_rounds=None):
    out = _run(lrq, rowptr, colidx, K, z0, 1 << 20 if max_rounds is None else max_rounds)
    z_ref, rounds, moves, conv = oracle.greedy_cut(rowptr, colidx, K, z0, max_rounds)
    assert np.array_equal(out["z"].cpu().numpy(), z_ref)
    assert (out["rounds"], out["moves"], out["converged"]) == (rounds, moves, conv)
    assert int(out["cut"].item()) == oracle.cut_count(rowptr, colidx, z_ref)
    return out


@pytest.mark.parametrize("n,K,seed", [(2000, 2, 1), (2000, 3, 2), (3001, 4, 3), (1500, 8, 4), (1, 3, 5),
                                      (517, 5, 6)])
def test_greedy_matches_oracle_from_random_start(lrq, n, K, seed):
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=seed) if n > 1 else (np.array([0, 0]), np.array([], int), None)
    z0 = I.rng(100 + seed).integers(0, K, n).astype(np.uint8)
    _check(lrq, rowptr, colidx, K, z0)


def test_greedy_long_chain_of_rounds(lrq):
    # all-zero start on a torus: 26 rounds, across several batches of 8
    rowptr, colidx = I.torus_graph(24, 30)
    out = _check(lrq, rowptr, colidx, 3, np.zeros(24 * 30, np.uint8))
    assert out["rounds"] > 16 and out["converged"]


def test_greedy_round_limit(lrq):
    rowptr, colidx, _ = I.sbm_graph(3000, 4.0, 8.0, seed=7)
    z0 = np.zeros(3000, np.uint8)
    for mr in (0, 1, 7, 8, 9):
        out = _check(lrq, rowptr, colidx, 3, z0, max_rounds=mr)
        assert out["rounds"] == mr and not out["converged"]


def test_greedy_from_rank1_sweep(lrq):
    # the hybrid solver: rank-1 sweep's best-cut state, then greedy
    n = 20000
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=8)
    V, lam = oracle.truncate_laplacian(rowptr, colidx, 2)
    q = oracle.two_eigvec_q(V, lam)
    rp, ci = _dev(rowptr, np.int32), _dev(colidx, np.int32)
    sw = lrq.rank1_sweep(_dev(q, np.complex128), 3, rp, ci)
    torch.cuda.synchronize()
    z0 = sw["zcut"].cpu().numpy()
    out = _check(lrq, rowptr, colidx, 3, z0)
    assert int(out["cut"].item()) > int(sw["cut"].item())


def test_greedy_self_loops_parallel_edges_and_isolated_vertices(lrq):
    rowptr = np.array([0, 3, 5, 5, 6], np.int32)
    colidx = np.array([0, 1, 1, 0, 0, 3], np.int32)
    _check(lrq, rowptr, colidx, 2, np.zeros(4, np.uint8))


def test_greedy_invalid_labels_and_graph_are_reported(lrq):
    rowptr, colidx = I.torus_graph(6, 7)
    z0 = np.zeros(42, np.uint8)
    z0[5] = 3
    rp, ci = _dev(rowptr, np.int32), _dev(colidx, np.int32)
    for mr in (0, 5):
        with pytest.raises(lrq.LrqError) as ei:
            lrq.greedy_cut(rp, ci, 3, _dev(z0, np.uint8), mr)
        assert ei.value.status == lrq.LRQ_EINVAL
    bad = np.array(colidx)
    bad[11] = 42
    with pytest.raises(lrq.LrqError) as ei:
        lrq.greedy_cut(rp, _dev(bad, np.int32), 3, _dev(np.zeros(42), np.uint8), 5)
    assert ei.value.status == lrq.LRQ_EINVAL


@pytest.mark.slow
def test_greedy_one_million_vertices(lrq):
    # the Max-3-Cut workload size: n = 10^6 planted SBM, random start
    n = 1_000_000
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=1)
    z0 = I.rng(9).integers(0, 3, n).astype(np.uint8)
    _check(lrq, rowptr, colidx, 3, z0)


@pytest.mark.slow
def test_hybrid_greedy_readings_at_one_million_vertices(lrq, capsys):
    # the hybrid solver's workload (SBM n = 10^6, K = 3): from the rank-1
    # sweep's best-cut state the GPU's parallel rounds and the oracle's
    # sequential steepest ascent (the other reading of "steepest ascent")
    # both end in single-move local optima; the cuts are recorded and must
    # agree within 1%
    n = 1_000_000
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=1)
    rp, ci = _dev(rowptr, np.int32), _dev(colidx, np.int32)
    tr = lrq.truncate(lrq.laplacian_matrix(rp, ci), 2, max_iter=1000, seed=0, want_c64=False)
    q = lrq.two_eigvec_q(tr["V"], tr["lam"])
    sw = lrq.rank1_sweep(q, 3, rp, ci)
    torch.cuda.synchronize()
    z0 = sw["zcut"].cpu().numpy()
    par = _run(lrq, rowptr, colidx, 3, z0)
    cut_par = int(par["cut"].item())
    zs, moves = oracle.greedy_sequential(rowptr, colidx, 3, z0)
    cut_seq = oracle.cut_count(rowptr, colidx, zs)
    with capsys.disabled():
        print("\nhybrid greedy at n = 10^6: start cut %d; parallel rounds %d (%d rounds, %d moves); "
              "sequential steepest ascent %d (%d moves)" % (int(sw["cut"].item()), cut_par, par["rounds"],
                                                            par["moves"], cut_seq, moves))
    assert cut_par > int(sw["cut"].item()) and cut_seq > int(sw["cut"].item())
    assert abs(cut_par - cut_seq) <= 0.01 * cut_seq
