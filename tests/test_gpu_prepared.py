"""GPU: a prepared instance (lrq_prepare + lrq_sample_score_prepared) gives
the same top-m, scores and drawn directions as lrq_sample_score on the same
V, C, K, mode and top_m -- both run the same kernels on the same operands,
so the comparison is bit for bit -- and keeps giving them after many calls
with other directions.  The one-shot path is itself checked against the
oracle in test_gpu_parity.py; one case here also checks the prepared path
against the oracle directly."""
import numpy as np
import pytest

import oracle as O
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,r,K,S", [(1, 1, 2, 5), (3001, 4, 3, 700), (5000, 2, 8, 4100), (2049, 6, 7, 513)])
def test_prepared_equals_one_shot(lrq, mode, n, r, K, S):
    V = _dev(I.factor(n, r, seed=n + r + K, scales=np.linspace(2.0, 0.5, r), dtype=np.complex64))
    top_m = min(16, S)
    pi = lrq.PreparedInstance(n, r, K, mode=mode).prepare(V)
    for rep in range(3):
        C = _dev(I.directions(S, r, seed=100 * rep + S))
        one = lrq.sample_score(V, K, C=C.clone(), mode=mode, top_m=top_m, want_scores=True)
        pre = pi.sample_score(C=C.clone(), top_m=top_m, want_scores=True)
        torch.cuda.synchronize()
        lrq.check_status(one["dev_status"])
        lrq.check_status(pre["dev_status"])
        lrq.check_status(pi.dev_status)
        assert torch.equal(one["scores"], pre["scores"])
        assert torch.equal(one["top_idx"], pre["top_idx"])
        assert torch.equal(one["top_f"], pre["top_f"])
    # drawn directions: the same seed gives the same stream and the same result
    one = lrq.sample_score(V, K, S=S, seed=77, mode=mode, top_m=top_m)
    pre = pi.sample_score(S=S, seed=77, top_m=top_m)
    torch.cuda.synchronize()
    assert torch.equal(one["C"], pre["C"])
    assert torch.equal(one["top_idx"], pre["top_idx"])
    assert torch.equal(one["top_f"], pre["top_f"])
    pi.close()


def test_prepared_matches_oracle_fp32(lrq):
    n, r, K, S = 4097, 3, 5, 600
    V = I.factor(n, r, seed=5, dtype=np.complex64)
    C = I.directions(S, r, seed=6)
    pi = lrq.PreparedInstance(n, r, K, mode=0).prepare(_dev(V))
    out = pi.sample_score(C=_dev(C), top_m=8, want_scores=True)
    torch.cuda.synchronize()
    lrq.check_status(out["dev_status"])
    ref = O.score(V.astype(np.complex128), K, C.astype(np.complex128))
    got = out["scores"].double().cpu().numpy()
    assert np.max(np.abs(got - ref) / np.maximum(ref, 1e-30)) < 1e-5


def test_reprepare_follows_new_instance(lrq):
    n, r, K, S = 3000, 4, 8, 1024
    V1 = _dev(I.factor(n, r, seed=1, dtype=np.complex64))
    V2 = _dev(I.factor(n, r, seed=2, dtype=np.complex64))
    C = _dev(I.directions(S, r, seed=3))
    pi = lrq.PreparedInstance(n, r, K, mode=1)
    pi.prepare(V1)
    a = pi.sample_score(C=C, top_m=4, want_scores=True)["scores"].clone()
    pi.prepare(V2)
    b = pi.sample_score(C=C, top_m=4, want_scores=True)["scores"].clone()
    ref2 = lrq.sample_score(V2, K, C=C, mode=1, top_m=4, want_scores=True)["scores"]
    torch.cuda.synchronize()
    assert not torch.equal(a, b)
    assert torch.equal(b, ref2)


@pytest.mark.parametrize("mode", [0, 1])
def test_prepare_flags_non_finite_instance(lrq, mode):
    V = I.factor(500, 2, seed=4, dtype=np.complex64)
    V[17, 1] = np.nan
    pi = lrq.PreparedInstance(500, 2, 4, mode=mode).prepare(_dev(V))
    torch.cuda.synchronize()
    assert int(pi.dev_status.item()) == lrq.LRQ_EINVAL
