"""lrq_truncate (Sec. 4.1, Algorithm 3) on the GPU against the oracle.

Eigenvalues are unique and compared directly: within 1e-9 ||Q|| of the
oracle's FP64 eigendecomposition (LAPACK for dense Q, ARPACK for the graph
Laplacian) or of a closed form.  Eigenvectors are unique up to a phase only
for simple eigenvalues, and for repeated ones only the eigenspace is: the
tests therefore check residuals ||Q u - lambda u|| and orthonormality, and
compare the truncated operator V V^H with the oracle's where the r-th and
(r+1)-th eigenvalues are separated.
"""
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


def _dense(lrq, Q, r, **kw):
    Qd = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.complex128)).to(DEV)
    out = lrq.truncate(lrq.dense_matrix(Qd), r, **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def _laplacian(lrq, rowptr, colidx, r, weights=None, **kw):
    rp = torch.from_numpy(np.asarray(rowptr, dtype=np.int32)).to(DEV)
    ci = torch.from_numpy(np.asarray(colidx, dtype=np.int32)).to(DEV)
    w = None if weights is None else torch.from_numpy(np.asarray(weights, dtype=np.float64)).to(DEV)
    out = lrq.truncate(lrq.laplacian_matrix(rp, ci, w), r, **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def _eigvecs(V, lam):
    keep = lam > 0
    U = np.zeros_like(V)
    U[:, keep] = V[:, keep] / np.sqrt(lam[keep])[None, :]
    return U, keep


def _check_pairs(apply, V, lam, scale, res_tol=1e-8):
    U, keep = _eigvecs(V, lam)
    if not keep.any():
        return
    Uk = U[:, keep]
    G = Uk.conj().T @ Uk
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-9
    R = apply(Uk) - Uk * lam[keep][None, :]
    assert np.linalg.norm(R, axis=0).max() <= res_tol * scale


def test_dense_low_rank_plus_noise(lrq):
    # Q = V V^H + sigma H, sigma = 0.05 ||V V^H||_2 (approximately low rank)
    n, r = 600, 4
    V0 = I.factor(n, r, seed=31, scales=(4.0, 3.0, 2.0, 1.0))
    Q0 = V0 @ V0.conj().T
    H = I.hermitian_gaussian(n, seed=32)
    Q = Q0 + 0.05 * np.linalg.norm(Q0, 2) * H / np.linalg.norm(H, 2)
    out = _dense(lrq, Q, r)
    Vo, lam_o = oracle.truncate_dense(Q, r)
    scale = np.abs(lam_o).max()
    assert np.all(np.diff(out["lam"]) <= 0)
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * scale
    P = out["V"] @ out["V"].conj().T
    Po = Vo @ Vo.conj().T
    assert np.abs(P - Po).max() <= 1e-7 * scale
    _check_pairs(lambda U: Q @ U, out["V"], out["lam"], scale)
    assert np.array_equal(out["V32"], out["V"].astype(np.complex64))


def test_dense_exact_rank_below_r(lrq):
    # rank 2 with r = 4: two zero eigenvalues, whose columns carry nothing
    n = 200
    V0 = I.factor(n, 2, seed=33)
    Q = V0 @ V0.conj().T
    out = _dense(lrq, Q, 4)
    _, lam_o = oracle.truncate_dense(Q, 4)
    scale = lam_o.max()
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * scale
    P = out["V"] @ out["V"].conj().T
    assert np.abs(P - Q).max() <= 1e-9 * scale


def test_dense_negative_eigenvalues_dropped(lrq):
    # a diagonal Q with negative entries among the r largest
    d = np.array([3.0, -5.0, 1.0, -0.5, -2.0, -7.0])
    out = _dense(lrq, np.diag(d).astype(np.complex128), 4)
    assert np.allclose(out["lam"], [3.0, 1.0, -0.5, -2.0], atol=1e-12)
    assert np.allclose(out["V"][:, 2:], 0)
    assert np.allclose(np.abs(out["V"][:, 0]) ** 2, [3, 0, 0, 0, 0, 0], atol=1e-12)


@pytest.mark.parametrize("n,r", [(1, 1), (3, 3), (8, 8), (33, 5)])
def test_dense_tiny_sizes(lrq, n, r):
    Q = I.hermitian_gaussian(n, seed=40 + n) + 3.0 * np.eye(n)
    out = _dense(lrq, Q, r)
    _, lam_o = oracle.truncate_dense(Q, r)
    scale = max(np.abs(np.linalg.eigvalsh(Q)).max(), 1e-300)
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * scale
    _check_pairs(lambda U: Q @ U, out["V"], out["lam"], scale)


def test_torus_closed_form_with_repeated_eigenvalues(lrq):
    # 12 x 12 torus: 8 (checkerboard, simple), then 6 + sqrt(3) four times
    k1 = k2 = 12
    rowptr, colidx = I.torus_graph(k1, k2)
    out = _laplacian(lrq, rowptr, colidx, 5)
    a = np.arange(k1)[:, None]
    b = np.arange(k2)[None, :]
    ev = np.sort((4 - 2 * np.cos(2 * np.pi * a / k1) - 2 * np.cos(2 * np.pi * b / k2)).ravel())[::-1]
    assert np.abs(out["lam"] - ev[:5]).max() <= 1e-9 * 8
    assert np.isclose(ev[1], 6 + np.sqrt(3)) and np.isclose(ev[4], 6 + np.sqrt(3))
    L = oracle.laplacian_dense(rowptr, colidx)
    _check_pairs(lambda U: L @ U, out["V"], out["lam"], 8.0)
    checker = ((a + b) % 2 * 2 - 1).ravel() / np.sqrt(k1 * k2)
    u1 = out["V"][:, 0] / np.sqrt(out["lam"][0])
    assert abs(abs(np.vdot(checker, u1)) - 1.0) < 1e-9


def test_sbm_laplacian_matches_arpack(lrq):
    rowptr, colidx, _ = I.sbm_graph(20000, 4.0, 8.0, seed=34)
    out = _laplacian(lrq, rowptr, colidx, 3)
    Vo, lam_o = oracle.truncate_laplacian(rowptr, colidx, 3)
    scale = lam_o[0]
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * scale
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(len(colidx)), colidx, rowptr), shape=(20000, 20000))
    L = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    _check_pairs(lambda U: L @ U, out["V"], out["lam"], scale)
    Uo, _ = _eigvecs(Vo, lam_o)
    U, _ = _eigvecs(out["V"], out["lam"])
    gaps = np.abs(np.diff(np.concatenate([lam_o, [oracle.truncate_laplacian(rowptr, colidx, 4)[1][3]]])))
    for j in range(3):
        if min(gaps[max(j - 1, 0)], gaps[j]) > 1e-3 * scale:
            assert abs(abs(np.vdot(Uo[:, j], U[:, j])) - 1) < 1e-8


def test_weighted_laplacian_matches_oracle(lrq):
    rowptr, colidx, _ = I.sbm_graph(3000, 4.0, 8.0, seed=35)
    g = I.rng(36)
    # symmetric weights: w_ij = w_ji from an edge hash
    rows = np.repeat(np.arange(3000), np.diff(rowptr))
    lo, hi = np.minimum(rows, colidx), np.maximum(rows, colidx)
    table = g.uniform(0.5, 2.0, 4096)
    w = table[(lo * 7919 + hi * 104729) % 4096]
    out = _laplacian(lrq, rowptr, colidx, 4, weights=w)
    _, lam_o = oracle.truncate_laplacian(rowptr, colidx, 4, weights=w)
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * lam_o[0]
    L = oracle.laplacian_dense(rowptr, colidx, w)
    _check_pairs(lambda U: L @ U, out["V"], out["lam"], lam_o[0])


def test_invalid_inputs_are_reported(lrq):
    rowptr, colidx = I.torus_graph(4, 5)
    bad = np.array(colidx)
    bad[7] = 1000
    with pytest.raises(lrq.LrqError) as ei:
        _laplacian(lrq, rowptr, bad, 2)
    assert ei.value.status == lrq.LRQ_EINVAL
    bad_rp = np.array(rowptr)
    bad_rp[3], bad_rp[4] = bad_rp[4], bad_rp[3]
    with pytest.raises(lrq.LrqError) as ei:
        _laplacian(lrq, bad_rp, colidx, 2)
    assert ei.value.status == lrq.LRQ_EINVAL
    Q = I.hermitian_gaussian(10, seed=37)
    Q[2, 3] = np.inf
    with pytest.raises(lrq.LrqError) as ei:
        _dense(lrq, Q, 2)
    assert ei.value.status == lrq.LRQ_EINVAL


def test_max_iter_too_small_is_reported(lrq):
    Q = I.hermitian_gaussian(300, seed=38)
    with pytest.raises(lrq.LrqError) as ei:
        _dense(lrq, Q, 4, max_iter=3)
    assert ei.value.status == lrq.LRQ_ENOCONV


def test_deterministic(lrq):
    Q = I.hermitian_gaussian(150, seed=39)
    a = _dense(lrq, Q, 3, seed=5)
    b = _dense(lrq, Q, 3, seed=5)
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["lam"], b["lam"])


@pytest.mark.slow
def test_sbm_one_million_vertices(lrq):
    # the Max-3-Cut workload: planted 3-partition SBM, n = 10^6, p_in n = 4,
    # p_out n = 8; rank-3 truncation of the Laplacian
    n = 1_000_000
    rowptr, colidx, _ = I.sbm_graph(n, 4.0, 8.0, seed=1)
    out = _laplacian(lrq, rowptr, colidx, 3, max_iter=1000)
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(len(colidx)), colidx, rowptr), shape=(n, n))
    L = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    scale = out["lam"][0]
    _check_pairs(lambda U: L @ U, out["V"], out["lam"], scale)
    _, lam_o = oracle.truncate_laplacian(rowptr, colidx, 3)
    assert np.abs(out["lam"] - lam_o).max() <= 1e-9 * scale
