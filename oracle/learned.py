"""FP64 CPU oracle of the learned proposal (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU legs may import it.

The learned proposal maps spectral features of a rank-4 factor V to a
mixture of von Mises-Fisher (vMF) densities on the unit sphere S^7 of
C^4 = R^8, from which candidate directions are drawn instead of uniformly.
The paper's own facts it uses: directions c and omega^k c give the same
assignment up to a global phase and the same objective (the K-fold
equivalence of the rounding, Sec. 2.3), and one coordinate of c can be put
in a canonical angular window of width 2 pi / K (Sec. 2.1).

Definitions implemented here, in plain FP64 numpy:

* gauge: rotate each column of V so that its entry of largest modulus
  (lowest row index on ties) is real and positive (eigenvector phases are
  arbitrary; this fixes them).
* features (F = 4 r + r + 4 = 24 for r = 4): lambda_j / sum(lambda); for
  a_i = ||V_i||^2 n / sum(lambda) and for b_ij = |V_ij|^2 n / lambda_j per
  column j: mean, variance, skewness, excess kurtosis.
* MLP: F -> 256 -> 256 -> 160, ReLU after the two hidden layers,
  y = x W + b with W stored (in x out) row-major.
* head: 16 components, each 10 outputs: u (8, mu = u / ||u||), kappa =
  softplus(o_8), mixture logit o_9 (weights = softmax over components).
* vMF on S^{p-1}, p = 8: density C_p(kappa) exp(kappa mu . x) with
  C_p(kappa) = kappa^{p/2-1} / ((2 pi)^{p/2} I_{p/2-1}(kappa)); here
  C_8 = kappa^3 / ((2 pi)^4 I_3(kappa)) and d log C_8 / d kappa =
  -I_4(kappa) / I_3(kappa) (from I_nu' = I_{nu+1} + nu I_nu / kappa).
* I_nu: power series sum_k (kappa/2)^{2k+nu} / (k! (k+nu)!) for kappa <= 30,
  the large-argument expansion e^kappa / sqrt(2 pi kappa) * sum_j (-1)^j
  prod_{i<=j} (4 nu^2 - (2i-1)^2) / (j! (8 kappa)^j) above.
* loss: mean over targets x of -log sum_m pi_m C_8(kappa_m) exp(kappa_m
  mu_m . x), and its gradient with respect to the network outputs.
* modes: the component means ordered by mixture weight (largest logit
  first, lower index on ties), the proposal's most probable directions.
* Wood's rejection sampler for vMF (A. T. A. Wood, Simulation of the von
  Mises Fisher distribution, 1994), used here only to check the sampler's
  law statistically.
* canonical window: multiply c by omega^{-k} so that arg c_1 lies in
  (-pi/K, pi/K].
* feature standardisation: centre each feature on its mean over the
  training rows, divide by the sample standard deviation (ddof 1, at least
  1e-6; 1 for a single row).
* Adam (Kingma and Ba, 2015) with bias correction.

Parity pins live in tests/test_oracle_learned.py.  Parity unpinned: the
gain of the learned proposal over uniform sampling (an empirical claim).
"""
from __future__ import annotations

import math

import numpy as np

P_DIM = 8          # S^7 in R^8 = C^4
N_COMP = 16
HEAD = 10          # per component: 8 (mu) + kappa + logit
WIDTH = 256
N_OUT = N_COMP * HEAD
SERIES_MAX_KAPPA = 30.0


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------
def gauge_fix(V):
    V = np.asarray(V, dtype=np.complex128)
    out = V.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))  # first maximum on ties
        a = V[i, j]
        if abs(a) > 0:
            out[:, j] = V[:, j] * (abs(a) / a)
    return out


def _moments(a):
    m = a.mean()
    d = a - m
    var = (d ** 2).mean()
    if var <= 0:
        return [m, 0.0, 0.0, 0.0]
    sd = math.sqrt(var)
    return [m, var, (d ** 3).mean() / sd ** 3, (d ** 4).mean() / var ** 2 - 3.0]


def features(V, lam):
    V = np.asarray(V, dtype=np.complex128)
    lam = np.asarray(lam, dtype=np.float64)
    n, r = V.shape
    total = lam.sum()
    f = list(lam / total)
    a = (np.abs(V) ** 2).sum(axis=1) * n / total
    f += _moments(a)
    for j in range(r):
        f += _moments(np.abs(V[:, j]) ** 2 * n / lam[j])
    return np.array(f)


# --------------------------------------------------------------------------
# Bessel functions and the vMF normaliser
# --------------------------------------------------------------------------
def log_bessel_i(nu: int, kappa: float) -> float:
    kappa = float(kappa)
    if kappa <= SERIES_MAX_KAPPA:
        half = 0.5 * kappa
        t = half ** nu / math.factorial(nu)
        s = t
        k = 0
        while True:
            t *= half * half / ((k + 1) * (k + 1 + nu))
            s += t
            k += 1
            if t < 1e-18 * s or k > 500:
                break
        return math.log(s)
    mu = 4.0 * nu * nu
    s, t = 1.0, 1.0
    for j in range(1, 12):
        t *= -(mu - (2 * j - 1) ** 2) / (j * 8.0 * kappa)
        s += t
    return kappa - 0.5 * math.log(2 * math.pi * kappa) + math.log(s)


def log_c8(kappa: float) -> float:
    return 3.0 * math.log(kappa) - 4.0 * math.log(2 * math.pi) - log_bessel_i(3, kappa)


def a8(kappa: float) -> float:
    """I_4 / I_3, the mean resultant length of vMF on S^7 (and -d log C_8/d kappa)."""
    return math.exp(log_bessel_i(4, kappa) - log_bessel_i(3, kappa))


# --------------------------------------------------------------------------
# MLP
# --------------------------------------------------------------------------
def param_shapes(F: int):
    return [(F, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, N_OUT), (N_OUT,)]


def unpack(params, F: int):
    out, o = [], 0
    for shp in param_shapes(F):
        k = int(np.prod(shp))
        out.append(np.asarray(params[o:o + k], dtype=np.float64).reshape(shp))
        o += k
    return out


def n_params(F: int) -> int:
    return sum(int(np.prod(s)) for s in param_shapes(F))


def mlp_forward(params, X):
    W1, b1, W2, b2, W3, b3 = unpack(params, X.shape[1])
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    O = H2 @ W3 + b3
    return O, (X, H1, H2)


def mlp_backward(params, cache, dO):
    X, H1, H2 = cache
    W1, b1, W2, b2, W3, b3 = unpack(params, X.shape[1])
    dW3 = H2.T @ dO
    db3 = dO.sum(axis=0)
    dH2 = (dO @ W3.T) * (H2 > 0)
    dW2 = H1.T @ dH2
    db2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0)
    dW1 = X.T @ dH1
    db1 = dH1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (dW1, db1, dW2, db2, dW3, db3)])


# --------------------------------------------------------------------------
# mixture head, loss and gradient
# --------------------------------------------------------------------------
def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def head(O):
    O = np.asarray(O, dtype=np.float64).reshape(-1, N_COMP, HEAD)
    u = O[:, :, :P_DIM]
    mu = u / np.linalg.norm(u, axis=2, keepdims=True)
    kappa = softplus(O[:, :, P_DIM])
    logit = O[:, :, P_DIM + 1]
    logpi = logit - np.log(np.exp(logit - logit.max(axis=1, keepdims=True)).sum(axis=1, keepdims=True)) \
        - logit.max(axis=1, keepdims=True)
    return mu, kappa, logpi


def nll(O, targets):
    """Mean over all (instance, target) pairs of -log p(x); targets B x T x 8."""
    mu, kappa, logpi = head(O)
    B, T, _ = targets.shape
    lc = np.vectorize(log_c8)(kappa)
    total = 0.0
    for b in range(B):
        ell = logpi[b][None, :] + lc[b][None, :] + kappa[b][None, :] * (targets[b] @ mu[b].T)  # T x M
        mx = ell.max(axis=1, keepdims=True)
        total += -(mx[:, 0] + np.log(np.exp(ell - mx).sum(axis=1))).sum()
    return total / (B * T)


def nll_grad(O, targets):
    """d nll / d O (B x 160), by the chain rule through the head."""
    O = np.asarray(O, dtype=np.float64).reshape(-1, N_COMP, HEAD)
    mu, kappa, logpi = head(O)
    B, T, _ = targets.shape
    u = O[:, :, :P_DIM]
    un = np.linalg.norm(u, axis=2)
    lc = np.vectorize(log_c8)(kappa)
    A = np.vectorize(a8)(kappa)
    sig = 1.0 / (1.0 + np.exp(-O[:, :, P_DIM]))
    pi = np.exp(logpi)
    G = np.zeros_like(O)
    for b in range(B):
        dots = targets[b] @ mu[b].T  # T x M
        ell = logpi[b][None, :] + lc[b][None, :] + kappa[b][None, :] * dots
        g = np.exp(ell - ell.max(axis=1, keepdims=True))
        g /= g.sum(axis=1, keepdims=True)  # responsibilities, T x M
        # logits: d(-log p)/d logit_k = pi_k - gamma_k
        G[b, :, P_DIM + 1] = (pi[b][None, :] - g).sum(axis=0)
        # kappa: -gamma (mu.x - A(kappa)), times softplus' = sigmoid
        G[b, :, P_DIM] = (-(g * (dots - A[b][None, :]))).sum(axis=0) * sig[b]
        # mu = u / ||u||: -gamma kappa (x - (mu.x) mu) / ||u||
        for m in range(N_COMP):
            proj = targets[b] - dots[:, m:m + 1] * mu[b, m][None, :]
            G[b, m, :P_DIM] = -(g[:, m:m + 1] * kappa[b, m] * proj).sum(axis=0) / un[b, m]
    return G.reshape(B, N_OUT) / (B * T)


# --------------------------------------------------------------------------
# sampling and the canonical window
# --------------------------------------------------------------------------
def wood_sample(mu, kappa, N, rng):
    """N draws from vMF(mu, kappa) on S^{p-1} by Wood's rejection method."""
    mu = np.asarray(mu, dtype=np.float64)
    p = mu.size
    b = (-2.0 * kappa + math.sqrt(4.0 * kappa * kappa + (p - 1) ** 2)) / (p - 1)
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + (p - 1) * math.log(1.0 - x0 * x0)
    out = np.empty((N, p))
    for s in range(N):
        while True:
            z = rng.beta((p - 1) / 2.0, (p - 1) / 2.0)
            w = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
            if kappa * w + (p - 1) * math.log(1.0 - x0 * w) - c >= math.log(rng.random()):
                break
        v = rng.standard_normal(p)
        v -= (v @ mu) * mu
        v /= np.linalg.norm(v)
        out[s] = w * mu + math.sqrt(max(0.0, 1.0 - w * w)) * v
    return out


def vmf_modes(O):
    """Per instance the component means mu_m = u_m / ||u_m|| (e_1 when u_m = 0)
    as complex 4-vectors (c_j = mu[2j] + i mu[2j+1]), ordered by mixture
    weight: largest logit first, lower component index on ties.  B x 16 x 4."""
    O = np.asarray(O, dtype=np.float64).reshape(-1, N_COMP, HEAD)
    B = O.shape[0]
    out = np.empty((B, N_COMP, P_DIM // 2), dtype=np.complex128)
    for b in range(B):
        order = sorted(range(N_COMP), key=lambda m: (-O[b, m, P_DIM + 1], m))
        for rank, m in enumerate(order):
            u = O[b, m, :P_DIM]
            nrm = math.sqrt(float(np.dot(u, u)))
            mu = u / nrm if nrm > 0 else np.eye(P_DIM)[0]
            out[b, rank] = mu[0::2] + 1j * mu[1::2]
    return out


def canonicalize(C, K: int):
    """Rows c of C times omega^{-k} so that arg c_1 lies in (-pi/K, pi/K]."""
    C = np.asarray(C, dtype=np.complex128)
    ang = np.angle(C[:, 0])
    k = np.ceil(ang * K / (2 * np.pi) - 0.5)  # arg - 2 pi k / K in (-pi/K, pi/K]
    return C * np.exp(-2j * np.pi * k / K)[:, None]


def to_real8(C):
    C = np.asarray(C, dtype=np.complex128)
    out = np.empty((C.shape[0], 2 * C.shape[1]))
    out[:, 0::2] = C.real
    out[:, 1::2] = C.imag
    return out


# --------------------------------------------------------------------------
# feature standardisation
# --------------------------------------------------------------------------
def standardize_fit(feat):
    """Per feature: mean over the rows and sample standard deviation (ddof 1,
    at least 1e-6; 1 for a single row)."""
    feat = np.asarray(feat, dtype=np.float64)
    mean = feat.mean(axis=0)
    if feat.shape[0] < 2:
        return mean, np.ones(feat.shape[1])
    return mean, np.maximum(feat.std(axis=0, ddof=1), 1e-6)


def standardize(feat, mean, std):
    return (np.asarray(feat, dtype=np.float64) - mean) / std


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------
def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
