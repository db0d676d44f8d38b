"""Pins for the learned-proposal oracle against independent facts: library
Bessel functions, limits of the vMF normaliser, central finite differences of
every gradient, the vMF mean resultant length of Wood's sampler, invariances
of the features and the one-step closed form of Adam."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import learned as L
from paper_2602_20376_gb300 import inputs as I


@pytest.mark.parametrize("nu", [3, 4])
def test_log_bessel_matches_scipy(nu):
    for k in [1e-3, 0.1, 1.0, 5.0, 17.0, 29.9, 30.1, 45.0, 200.0, 3000.0]:
        ref = math.log(special.ive(nu, k)) + k
        assert abs(L.log_bessel_i(nu, k) - ref) <= 1e-11 * max(1.0, abs(ref)), (nu, k)


def test_vmf_normaliser_limits():
    # kappa -> 0: the uniform density on S^7, whose area is 2 pi^4 / 3! = pi^4 / 3
    assert abs(L.log_c8(1e-7) + math.log(math.pi ** 4 / 3)) < 1e-10
    # A_8(kappa) ~ kappa / 8 for small kappa, 1 - 7 / (2 kappa) for large kappa
    assert abs(L.a8(1e-4) - 1e-4 / 8) < 1e-10
    k = 1e4
    assert abs(L.a8(k) - (1 - 7 / (2 * k))) < 1e-6


def test_dlogc8_is_minus_a8():
    for k in [0.3, 2.0, 12.0, 29.0, 31.0, 150.0]:
        h = 1e-5 * max(1.0, k)
        fd = (L.log_c8(k + h) - L.log_c8(k - h)) / (2 * h)
        assert abs(fd + L.a8(k)) < 1e-7, k


def test_single_flat_component_gives_uniform_nll():
    # one component with kappa -> 0 and the rest with -inf logits: density 3 / pi^4
    O = np.zeros((1, L.N_OUT))
    O = O.reshape(1, L.N_COMP, L.HEAD)
    O[0, :, :8] = 1.0
    O[0, :, 8] = -40.0            # softplus ~ 4e-18
    O[0, 1:, 9] = -1e3
    x = I.rng(1).standard_normal((1, 5, 8))
    x /= np.linalg.norm(x, axis=2, keepdims=True)
    assert abs(L.nll(O.reshape(1, -1), x) - math.log(math.pi ** 4 / 3)) < 1e-9


def _random_head(B, seed):
    g = I.rng(seed)
    O = g.standard_normal((B, L.N_OUT))
    O = O.reshape(B, L.N_COMP, L.HEAD)
    O[:, :, 8] = g.uniform(-1, 4, (B, L.N_COMP))
    return O.reshape(B, L.N_OUT)


def test_nll_gradient_matches_finite_differences():
    B, T = 2, 7
    O = _random_head(B, 2)
    x = I.rng(3).standard_normal((B, T, 8))
    x /= np.linalg.norm(x, axis=2, keepdims=True)
    G = L.nll_grad(O, x)
    idx = I.rng(4).choice(O.size, 60, replace=False)
    for flat in idx:
        b, j = divmod(int(flat), L.N_OUT)
        h = 1e-6
        Op, Om = O.copy(), O.copy()
        Op[b, j] += h
        Om[b, j] -= h
        fd = (L.nll(Op, x) - L.nll(Om, x)) / (2 * h)
        assert abs(fd - G[b, j]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (b, j, fd, G[b, j])


def test_mlp_backward_matches_finite_differences():
    F, B = 24, 3
    g = I.rng(5)
    params = g.standard_normal(L.n_params(F)) * 0.1
    X = g.standard_normal((B, F))
    R = g.standard_normal((B, L.N_OUT))  # loss = sum(O * R)
    O, cache = L.mlp_forward(params, X)
    grad = L.mlp_backward(params, cache, R)
    for k in g.choice(params.size, 80, replace=False):
        h = 1e-6
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        fd = ((L.mlp_forward(p1, X)[0] - L.mlp_forward(p2, X)[0]) * R).sum() / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_wood_sampler_mean_resultant_length():
    rng = np.random.default_rng(6)
    mu = rng.standard_normal(8)
    mu /= np.linalg.norm(mu)
    for kappa in [0.5, 5.0, 60.0]:
        X = L.wood_sample(mu, kappa, 20000, rng)
        assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-12)
        t = X @ mu
        se = t.std() / math.sqrt(len(t))
        assert abs(t.mean() - L.a8(kappa)) < 5 * se, kappa
        # the part orthogonal to mu has no preferred direction
        perp = X - t[:, None] * mu[None, :]
        assert np.abs(perp.mean(axis=0)).max() < 5 * perp.std() / math.sqrt(len(t))


def test_features_invariances():
    V = I.factor(300, 4, seed=7, scales=(3.0, 2.0, 1.0, 0.5))
    lam = np.array([9.0, 4.0, 1.0, 0.25])
    f = L.features(V, lam)
    assert f.size == 24
    # moduli only: any column phase leaves them unchanged, and the gauge
    # fixes the phases to the same V
    ph = np.exp(1j * I.rng(8).uniform(0, 2 * np.pi, 4))
    assert np.allclose(L.features(V * ph[None, :], lam), f, atol=1e-12)
    assert np.allclose(L.gauge_fix(V * ph[None, :]), L.gauge_fix(V), atol=1e-12)
    G = L.gauge_fix(V)
    i = np.argmax(np.abs(G), axis=0)
    assert np.all(np.abs(G[i, np.arange(4)].imag) < 1e-15) and np.all(G[i, np.arange(4)].real > 0)
    # scaling V and lambda together changes no feature; the normalised means are 1
    assert np.allclose(L.features(2.0 * V, 4.0 * lam), f, atol=1e-12)
    assert np.allclose(f[4], (np.abs(V) ** 2).sum() * 300 / lam.sum() / 300)


def test_canonical_window_and_equivalence():
    K = 8
    C = I.directions(500, 4, seed=9, dtype=np.complex128)
    Cc = L.canonicalize(C, K)
    a = np.angle(Cc[:, 0])
    assert np.all(a > -np.pi / K - 1e-12) and np.all(a <= np.pi / K + 1e-12)
    # each row differs from the original by a K-th root of unity
    ratio = Cc[:, 0] / C[:, 0]
    k = np.round(np.angle(ratio) * K / (2 * np.pi))
    assert np.allclose(ratio, np.exp(2j * np.pi * k / K))


def test_adam_first_step_closed_form():
    g = I.rng(10)
    p = g.standard_normal(50)
    gr = g.standard_normal(50)
    out, m, v = L.adam_step(p, gr, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    assert np.allclose(out, p - 0.01 * np.sign(gr), atol=1e-15)


def test_features_moments_of_complex_gaussian_factor():
    # For i.i.d. CN(0, 1) entries, |V_ij|^2 ~ Exp(1): with lambda_j the column
    # sums of |V_ij|^2, b_ij = n |V_ij|^2 / lambda_j has mean exactly 1 and,
    # as n grows, the Exp(1) variance, skewness and excess kurtosis 1, 2, 6;
    # a_i = n ||V_i||^2 / sum(lambda) is Gamma(r, 1) / r: 1, 1/r, 2/sqrt(r),
    # 6/r.  A dropped "- 3", a wrong power or a missing normalisation moves a
    # value far outside the sampling tolerance (5 standard errors of the
    # estimators at n = 2^20: about 0.014, 0.08 and 0.6 for Exp(1)).
    n, r = 1 << 20, 4
    g = I.rng(31)
    V = (g.standard_normal((n, r)) + 1j * g.standard_normal((n, r))) / math.sqrt(2.0)
    lam = (np.abs(V) ** 2).sum(axis=0)
    f = L.features(V, lam)
    assert np.allclose(f[:r], lam / lam.sum(), atol=1e-15)
    assert np.allclose(f[:r], 1.0 / r, atol=5e-3)
    row = f[r:r + 4]
    assert abs(row[0] - 1.0) < 1e-12
    assert abs(row[1] - 1.0 / r) < 0.01
    assert abs(row[2] - 2.0 / math.sqrt(r)) < 0.04
    assert abs(row[3] - 6.0 / r) < 0.3
    for j in range(r):
        col = f[r + 4 + 4 * j:r + 8 + 4 * j]
        assert abs(col[0] - 1.0) < 1e-12
        assert abs(col[1] - 1.0) < 0.014
        assert abs(col[2] - 2.0) < 0.08
        assert abs(col[3] - 6.0) < 0.6


def test_features_population_moments_by_hand():
    # one column with |V_i1|^2 = (0, 0, 0, 4) and lambda = 1: b = (0, 0, 0, 16)
    # has mean 4, population variance 48, third central moment 384 (skewness
    # 384 / 48^1.5 = 2 / sqrt(3)), fourth (3 * 256 + 20736) / 4 = 5376 (excess
    # kurtosis 5376 / 48^2 - 3 = -2/3); the row quantity is the same vector
    V = np.array([[0.0], [0.0], [0.0], [2.0]], dtype=np.complex128)
    f = L.features(V, np.array([1.0]))
    k = 5376.0 / 48.0 ** 2 - 3.0
    assert np.allclose(f, [1.0, 4.0, 48.0, 2.0 / math.sqrt(3.0), k, 4.0, 48.0, 2.0 / math.sqrt(3.0), k], atol=1e-12)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2,
    # so the bias-corrected step is lr g / (|g| + eps) at every t: after t
    # steps the parameters have moved by t lr g / (|g| + eps)
    g = I.rng(11)
    p0 = g.standard_normal(40)
    gr = g.standard_normal(40)
    lr, b1, b2, eps = 0.003, 0.9, 0.999, 1e-3
    p, m, v = p0.copy(), np.zeros(40), np.zeros(40)
    for t in range(1, 26):
        p, m, v = L.adam_step(p, gr, m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        assert np.allclose(m, (1 - b1 ** t) * gr, rtol=1e-12, atol=1e-15)
        assert np.allclose(v, (1 - b2 ** t) * gr * gr, rtol=1e-12, atol=1e-15)
        assert np.allclose(p, p0 - t * lr * gr / (np.abs(gr) + eps), rtol=1e-12, atol=1e-14)


def test_standardize_invariants():
    g = I.rng(12)
    feat = g.standard_normal((50, 6)) * np.array([1.0, 10.0, 0.1, 3.0, 1.0, 1.0]) + 5.0
    feat[:, 4] = 2.5  # a constant feature
    mean, std = L.standardize_fit(feat)
    X = L.standardize(feat, mean, std)
    keep = [0, 1, 2, 3, 5]
    assert np.allclose(X[:, keep].mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(X[:, keep].std(axis=0, ddof=1), 1.0, atol=1e-12)
    assert std[4] == 1e-6 and np.all(X[:, 4] == 0.0)
    # a single row: centred to zero, unscaled
    m1, s1 = L.standardize_fit(feat[:1])
    assert np.all(s1 == 1.0) and np.all(L.standardize(feat[:1], m1, s1) == 0.0)


def test_vmf_modes_by_hand():
    # component m: u = (m + 1) e_(m mod 8), so mu_m = e_(m mod 8); logits
    # -(m mod 5): ranks go 0, 5, 10, 15 (logit 0), then 1, 6, 11, ...
    O = np.zeros((1, L.N_COMP, L.HEAD))
    for m in range(L.N_COMP):
        O[0, m, m % 8] = m + 1.0
        O[0, m, 8] = 0.3
        O[0, m, 9] = -(m % 5)
    O[0, 7, :8] = 0.0  # a zero u: the mode is e_1 by convention
    got = L.vmf_modes(O.reshape(1, -1))[0]
    order = [0, 5, 10, 15, 1, 6, 11, 2, 7, 12, 3, 8, 13, 4, 9, 14]
    for rank, m in enumerate(order):
        want = np.zeros(8)
        want[0 if m == 7 else m % 8] = 1.0
        assert np.array_equal(got[rank], want[0::2] + 1j * want[1::2]), (rank, m)
    # the order is the mixture weights' order (softmax is monotone)
    _, _, logpi = L.head(O.reshape(1, -1))
    assert np.all(np.diff(logpi[0][order]) <= 0)


def test_vmf_modes_unit_norm_and_direction():
    rng = np.random.default_rng(5)
    O = rng.standard_normal((3, L.N_OUT))
    modes = L.vmf_modes(O)
    Oh = O.reshape(3, L.N_COMP, L.HEAD)
    for b in range(3):
        ranks = np.argsort(-Oh[b, :, 9], kind="stable")
        for rank, m in enumerate(ranks):
            c = modes[b, rank]
            assert abs(np.linalg.norm(c) - 1.0) < 1e-12
            u = Oh[b, m, :8]
            # mu is the positive multiple of u
            x = L.to_real8(c[None])[0]
            assert np.dot(x, u) > 0 and np.allclose(x * np.linalg.norm(u), u, atol=1e-12)
