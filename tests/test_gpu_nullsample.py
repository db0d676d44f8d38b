"""lrq_sample_null_directions (the null-vector sampler of Sec. 5, the
randomised Algorithm 2) on the GPU against the oracle.

Both sides draw the same rows from the stated Philox convention and take
the rank decision by the same elimination rule in FP64, so the draw counts
must be identical; the directions agree to complex64 rounding (the oracle's
null vector comes from an SVD, the kernel's from back-substitution: 1e-6
absolute on unit-norm rows)."""
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


def _sample(lrq, V, K, S, seed):
    out = lrq.sample_null_directions(torch.from_numpy(np.ascontiguousarray(V, np.complex64)).to(DEV), K, S, seed)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,r,K,S,seed", [(1000, 2, 3, 3000, 1), (700, 4, 8, 1000, 2), (500, 1, 2, 2000, 3),
                                          (300, 8, 5, 300, 4), (5, 3, 3, 500, 5), (2, 2, 3, 2000, 6)])
def test_null_directions_match_oracle(lrq, n, r, K, S, seed):
    V = I.factor(n, r, seed=40 + seed, scales=np.linspace(2.0, 0.5, r), dtype=np.complex64)
    out = _sample(lrq, V, K, S, seed)
    assert int(out["dev_status"].item()) == 0
    C_ref, draws = oracle.null_directions(V.astype(np.complex128), K, seed, S)
    assert int(out["draws"].item()) == int(draws.sum())
    C = out["C"].cpu().numpy()
    assert np.abs(C - C_ref).max() <= 1e-6


def test_zero_rows_and_real_factors(lrq):
    # real V (the Laplacian case) with zero rows: zero rows of the augmented
    # matrix make many draws dependent; both sides must reject the same ones
    g = I.rng(50)
    V = g.standard_normal((400, 2)).astype(np.complex64)
    V[g.choice(400, 150, replace=False)] = 0
    out = _sample(lrq, V, 3, 2000, 7)
    assert int(out["dev_status"].item()) == 0
    C_ref, draws = oracle.null_directions(V.astype(np.complex128), 3, 7, 2000)
    assert int(out["draws"].item()) == int(draws.sum()) > 2000
    assert np.abs(out["C"].cpu().numpy() - C_ref).max() <= 1e-6


def test_rank_deficient_factor_is_reported(lrq):
    V = I.factor(50, 3, seed=51, dtype=np.complex64)
    V[:, 2] = 0
    out = _sample(lrq, V, 4, 64, 8)
    assert int(out["dev_status"].item()) == lrq.LRQ_EUNSUPPORTED
    assert int(out["draws"].item()) == 64 * 64
    assert not out["C"].abs().any()


def test_null_directions_scored_by_the_scoring_path(lrq):
    # the sampler's output is an ordinary direction set for lrq_sample_score.
    # A null vector puts 2r - 1 coordinates exactly on a boundary, where either
    # neighbouring code is a correct rounding (Eq. 9 ties): each such
    # coordinate may move V^H z by |omega^a - omega^b| ||V_i|| = 2 sin(pi/K) ||V_i||
    n, r, K, S = 4000, 3, 3, 4096
    V = I.factor(n, r, seed=52, scales=(3.0, 2.0, 1.0), dtype=np.complex64)
    Vd = torch.from_numpy(V).to(DEV)
    out = _sample(lrq, V, K, S, 9)
    sc = lrq.sample_score(Vd, K, C=out["C"], mode=lrq.LRQ_MODE_FP32, top_m=8, want_scores=True)
    torch.cuda.synchronize()
    f = sc["scores"].cpu().numpy().astype(np.float64)
    f_ref = oracle.score(V.astype(np.complex128), K, out["C"].cpu().numpy().astype(np.complex128))
    tie = (2 * r - 1) * 2 * np.sin(np.pi / K) * np.linalg.norm(V.astype(np.complex128), axis=1).max()
    assert np.all(np.abs(np.sqrt(f) - np.sqrt(f_ref)) <= tie + 1e-5 * np.sqrt(f_ref))
