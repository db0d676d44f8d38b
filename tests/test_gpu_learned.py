"""Learned-proposal kernels on the GPU against the FP64 oracle
(oracle/learned.py): features and gauge, MLP forward and backward (FP32
operands: 1e-5 relative; BF16 operands: within a first-order rounding bound
derived from |X| |W|), vMF loss and gradient (FP64 inside: 1e-9 on the loss,
float rounding on dO), the sampler's law, and Adam."""
import math

import numpy as np
import pytest

from oracle import learned as OL
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


def _t(x, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV) if dtype is None else \
        torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def test_features_and_gauge_match_oracle(lrq):
    B, n, r = 3, 700, 4
    V = np.stack([I.factor(n, r, seed=50 + b, scales=(3.0, 1.5, 1.0, 0.5), dtype=np.complex64) for b in range(B)])
    lam = np.array([[9.0, 2.25, 1.0, 0.25], [5.0, 4.0, 3.0, 1.0], [1.0, 1.0, 0.5, 0.1]])
    Vg = torch.empty((B, n, r), dtype=torch.complex64, device=DEV)
    feat = torch.empty((B, 24), dtype=torch.float32, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    lrq.lrq_proposal_features(_t(V), _t(lam), Vg, feat, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    for b in range(B):
        f_ref = OL.features(V[b].astype(np.complex128), lam[b])
        f = feat[b].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(f - f_ref) <= 1e-6 * np.maximum(1.0, np.abs(f_ref))), (b, f, f_ref)
        G = OL.gauge_fix(V[b].astype(np.complex128))
        assert np.abs(Vg[b].cpu().numpy() - G).max() <= 2e-6 * np.abs(G).max()


def _mlp_case(F=24, B=96, seed=60):
    g = I.rng(seed)
    params = (g.standard_normal(OL.n_params(F)) * 0.08).astype(np.float32)
    X = g.standard_normal((B, F)).astype(np.float32)
    return params, X


def _run_fwd(lrq, params, X, bf16):
    B = X.shape[0]
    H1 = torch.empty((B, 256), device=DEV)
    H2 = torch.empty((B, 256), device=DEV)
    O = torch.empty((B, 160), device=DEV)
    lrq.lrq_mlp_forward(_t(params), _t(X), H1, H2, O, bf16)
    torch.cuda.synchronize()
    return O.cpu().numpy().astype(np.float64), H1, H2


def test_mlp_forward_fp32_matches_oracle(lrq):
    params, X = _mlp_case()
    O, _, _ = _run_fwd(lrq, params, X, False)
    O_ref, _ = OL.mlp_forward(params.astype(np.float64), X.astype(np.float64))
    assert np.abs(O - O_ref).max() <= 1e-5 * np.abs(O_ref).max()


def test_mlp_forward_bf16_within_rounding_bound(lrq):
    params, X = _mlp_case(seed=61)
    O, _, _ = _run_fwd(lrq, params, X, True)
    p = params.astype(np.float64)
    W1, b1, W2, b2, W3, b3 = OL.unpack(p, X.shape[1])
    O_ref, (X64, H1, H2) = OL.mlp_forward(p, X.astype(np.float64))
    # first-order bound: each GEMM operand is rounded to bfloat16 (relative
    # error 2^-8 each, 2^-7 per product) and the layers are 1-Lipschitz in
    # their input through ReLU
    u = 2.0 ** -7
    e1 = u * np.abs(X64) @ np.abs(W1)
    e2 = e1 @ np.abs(W2) + u * (np.abs(H1) + e1) @ np.abs(W2)
    e3 = e2 @ np.abs(W3) + u * (np.abs(H2) + e2) @ np.abs(W3)
    assert np.all(np.abs(O - O_ref) <= 1.05 * e3 + 1e-6)


def _bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("bf16", [False, True])
def test_mlp_backward_matches_oracle(lrq, bf16):
    params, X = _mlp_case(seed=62)
    B = X.shape[0]
    O, H1, H2 = _run_fwd(lrq, params, X, bf16)
    dO = I.rng(63).standard_normal((B, 160)).astype(np.float32)
    grads = torch.empty(OL.n_params(24), device=DEV)
    scratch = torch.empty((2, B, 256), device=DEV)
    lrq.lrq_mlp_backward(_t(params), _t(X), H1, H2, _t(dO), grads, scratch, bf16)
    torch.cuda.synchronize()
    g = grads.cpu().numpy().astype(np.float64)
    if not bf16:
        _, cache = OL.mlp_forward(params.astype(np.float64), X.astype(np.float64))
        g_ref = OL.mlp_backward(params.astype(np.float64), cache, dO.astype(np.float64))
        assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
        return
    # BF16 operands: the oracle's backward on the operands the kernels see
    # (weights, inputs, the kernels' own activations and dO rounded to
    # bfloat16); what is left is the rounding of the two inner gradients
    # dH2, dH1 (2^-8 relative) that the oracle keeps exact
    cache = (_bf16(X), _bf16(H1.cpu().numpy()), _bf16(H2.cpu().numpy()))
    g_ref = OL.mlp_backward(_bf16(params), cache, _bf16(dO))
    assert np.linalg.norm(g - g_ref) <= 1e-2 * np.linalg.norm(g_ref)
    # and against exact FP64 arithmetic throughout: a few percent
    _, c64 = OL.mlp_forward(params.astype(np.float64), X.astype(np.float64))
    g64 = OL.mlp_backward(params.astype(np.float64), c64, dO.astype(np.float64))
    assert np.linalg.norm(g - g64) <= 0.1 * np.linalg.norm(g64)


def _head_case(B, seed):
    g = I.rng(seed)
    O = g.standard_normal((B, 16, 10))
    O[:, :, 8] = g.uniform(-3.0, 60.0, (B, 16))  # kappa from ~0.05 (series) to 60 (expansion)
    return O.reshape(B, 160).astype(np.float32)


def test_vmf_nll_and_gradient_match_oracle(lrq):
    B, T = 5, 37
    O = _head_case(B, 64)
    x = I.rng(65).standard_normal((B, T, 8))
    x = (x / np.linalg.norm(x, axis=2, keepdims=True)).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    dO = torch.empty((B, 160), device=DEV)
    lrq.lrq_vmf_nll(_t(O), _t(x), loss, dO)
    torch.cuda.synchronize()
    l_ref = OL.nll(O.astype(np.float64), x.astype(np.float64))
    g_ref = OL.nll_grad(O.astype(np.float64), x.astype(np.float64))
    assert abs(float(loss.item()) - l_ref) <= 1e-9 * abs(l_ref)
    g = dO.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(g - g_ref) <= 1e-6 * np.abs(g_ref) + 1e-9 * np.abs(g_ref).max())


def test_vmf_sampler_law(lrq):
    # one dominant component: mean resultant length A_8(kappa), unit norm,
    # the part orthogonal to mu without a preferred direction
    g = I.rng(66)
    mu = g.standard_normal(8)
    mu /= np.linalg.norm(mu)
    S = 1 << 16
    for kappa in [0.7, 8.0, 120.0]:
        O = np.zeros((1, 16, 10), dtype=np.float64)
        O[0, :, :8] = mu
        O[0, :, 8] = kappa + math.log(-math.expm1(-kappa))  # softplus^{-1}(kappa)
        O[0, 1:, 9] = -60.0
        C = torch.empty((1, S, 4), dtype=torch.complex64, device=DEV)
        st = torch.zeros(1, dtype=torch.int32, device=DEV)
        lrq.lrq_vmf_sample(_t(O.reshape(1, 160).astype(np.float32)), S, 1, 123, C, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        Xs = torch.view_as_real(C[0]).reshape(S, 8).cpu().numpy().astype(np.float64)
        assert np.abs(np.linalg.norm(Xs, axis=1) - 1).max() < 1e-6
        t = Xs @ mu
        se = t.std() / math.sqrt(S)
        assert abs(t.mean() - OL.a8(kappa)) < 5 * se + 1e-6, kappa
        perp = Xs - t[:, None] * mu[None, :]
        assert np.abs(perp.mean(axis=0)).max() < 5 * perp.std() / math.sqrt(S) + 1e-7


def test_vmf_sampler_mixture_weights_and_rotation(lrq):
    # four components with weights 0.4, 0.3, 0.2, 0.1 and means on the real
    # axes of c_1 .. c_4; K = 8 rotations spread each phase over 8 classes
    S = 1 << 16
    O = np.zeros((1, 16, 10))
    eye = np.eye(8)
    w = np.array([0.4, 0.3, 0.2, 0.1])
    for m in range(16):
        O[0, m, :8] = eye[2 * m] if m < 4 else eye[0]
        O[0, m, 8] = 400.0
        O[0, m, 9] = math.log(w[m]) if m < 4 else -80.0
    C = torch.empty((1, S, 4), dtype=torch.complex64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    lrq.lrq_vmf_sample(_t(O.reshape(1, 160).astype(np.float32)), S, 8, 321, C, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Cn = C[0].cpu().numpy().astype(np.complex128)
    comp = np.argmax(np.abs(Cn), axis=1)  # the rotation does not change the moduli
    from scipy import stats
    assert stats.chisquare(np.bincount(comp, minlength=4)[:4], w * S).pvalue > 1e-4
    # rotation class of each sample: the phase of its dominant coordinate
    ph = np.angle(Cn[np.arange(S), comp])
    k = np.mod(np.round(ph * 8 / (2 * np.pi)), 8).astype(int)
    assert stats.chisquare(np.bincount(k, minlength=8)).pvalue > 1e-4
    # in the canonical window the component-0 samples sit next to their mean
    canon = OL.to_real8(OL.canonicalize(Cn[comp == 0], 8))
    assert np.all(canon[:, 0] > 0.8)


def test_adam_step_matches_oracle(lrq):
    g = I.rng(67)
    n = 5000
    p = g.standard_normal(n).astype(np.float32)
    gr = g.standard_normal(n).astype(np.float32)
    m = (0.1 * g.standard_normal(n)).astype(np.float32)
    v = (0.1 * g.random(n)).astype(np.float32)
    P, G, M, Vv = _t(p), _t(gr), _t(m), _t(v)
    lrq.lrq_adam_step(P, G, M, Vv, 7, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    torch.cuda.synchronize()
    p_ref, m_ref, v_ref = OL.adam_step(p.astype(np.float64), gr.astype(np.float64), m.astype(np.float64),
                                       v.astype(np.float64), 7, lr=3e-3)
    assert np.abs(P.cpu().numpy() - p_ref).max() <= 1e-6
    assert np.abs(M.cpu().numpy() - m_ref).max() <= 1e-6
    assert np.abs(Vv.cpu().numpy() - v_ref).max() <= 1e-6


def test_vmf_modes_match_oracle(lrq):
    # random heads, plus one instance with tied logits and a zero u
    g = I.rng(69)
    O = g.standard_normal((5, OL.N_OUT)).astype(np.float32)
    Oh = O.reshape(5, OL.N_COMP, OL.HEAD)
    Oh[4, :, 9] = np.float32(0.25) * (np.arange(OL.N_COMP) % 3)
    Oh[4, 6, :8] = 0.0
    C = torch.empty((5, 16, 4), dtype=torch.complex64, device=DEV)
    lrq.lrq_vmf_modes(_t(O), C)
    torch.cuda.synchronize()
    ref = OL.vmf_modes(O.astype(np.float64))
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-6


@pytest.mark.parametrize("K,r", [(8, 4), (3, 2), (5, 7)])
def test_proposal_targets_match_oracle(lrq, K, r):
    # gathered directions in the canonical window (Sec. 2.3), against the
    # oracle's canonicalize of the same rows; an index outside [0, S) is
    # reported and yields zeros
    S, m = 3000, 257
    C = I.directions(S, r, seed=70 + K)
    idx = I.rng(71).choice(S, m, replace=False).astype(np.int64)
    out = torch.empty((m, 2 * r), dtype=torch.float32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    lrq.lrq_proposal_targets(_t(C), K, _t(idx), out, status)
    torch.cuda.synchronize()
    lrq.check_status(status, "lrq_proposal_targets")
    ref = OL.to_real8(OL.canonicalize(C[idx].astype(np.complex128), K))
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6
    bad = idx.copy()
    bad[5] = S
    lrq.lrq_proposal_targets(_t(C), K, _t(bad), out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == lrq.LRQ_EINVAL
    assert np.all(out.cpu().numpy()[5] == 0)


@pytest.mark.parametrize("B", [1, 2, 97])
def test_standardize_matches_oracle(lrq, B):
    g = I.rng(72 + B)
    feat = (g.standard_normal((B, 24)) * np.linspace(0.1, 30.0, 24) + 7.0).astype(np.float32)
    feat[:, 3] = 1.5  # constant feature: its standard deviation is clamped
    F = _t(feat)
    mean = torch.empty(24, device=DEV)
    std = torch.empty(24, device=DEV)
    X = torch.empty_like(F)
    lrq.lrq_standardize_fit(F, mean, std)
    lrq.lrq_standardize(F, mean, std, X)
    torch.cuda.synchronize()
    m_ref, s_ref = OL.standardize_fit(feat.astype(np.float64))
    assert np.allclose(mean.cpu().numpy(), m_ref, rtol=1e-6, atol=1e-6)
    assert np.allclose(std.cpu().numpy(), s_ref, rtol=1e-6, atol=1e-9)
    ref = OL.standardize(feat.astype(np.float64), mean.cpu().numpy().astype(np.float64),
                         std.cpu().numpy().astype(np.float64))
    assert np.abs(X.cpu().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


@pytest.mark.slow
@pytest.mark.parametrize("hard", [False, True])
def test_trained_proposal_beats_uniform_and_fixed_direction(lrq, hard):
    # angular synchronisation at n = 1024 (K = 8, rank-4 truncation), at the
    # workload's sigma and in the high-noise regime (sigma sqrt(n) ~ n / 4):
    # train on the top 1% of 2^14 uniform directions of 256 instances, then
    # on 64 held-out instances count the draws each stream needs to reach
    # 0.999 of the best of 2^16 uniform draws.  The learned stream (16
    # mixture modes, then vMF draws) must need 4x fewer draws than uniform
    # sampling at the median, and within 16 draws reach the level on more
    # instances than the fixed direction e_1 followed by uniform draws (on
    # as many when e_1 already reaches it everywhere)
    from paper_2602_20376_gb300 import proposal as P
    n, ntrain, neval = 1024, 256, 64
    sig = P.sigma_hard(n) if hard else P.SIGMA_EASY
    V, lam = P.truncate_instances(n, range(10 ** 6, 10 ** 6 + ntrain + neval), sigma_range=sig)
    Vg, feat = P.features(V, lam)
    targets = P.training_targets(Vg[:ntrain], 8, 1 << 14, 555)
    model = P.Proposal(feat.shape[1], seed=0)
    model.fit_standardizer(feat[:ntrain])
    losses = P.train(model, feat[:ntrain], targets, 600, 64, 1e-3)
    assert float(losses[-10:].mean()) < float(losses[:10].mean()) - 1.0
    rows = P.evaluate(model, Vg[ntrain:], feat[ntrain:], 8, 1 << 16, 777)
    assert P.median_gain(rows) >= 4.0
    learned16, e1_16 = P.reached_within(rows, 2, 16), P.reached_within(rows, 3, 16)
    if e1_16 == neval:
        assert learned16 == neval
    else:
        assert learned16 > e1_16
