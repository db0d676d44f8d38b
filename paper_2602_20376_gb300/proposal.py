"""Learned proposal: training and evaluation driver over the C ABI.

Every numerical step of the method runs in liblrq's kernels (truncation,
features, feature standardisation, MLP forward/backward, vMF loss, vMF
sampling, Adam, scoring with its top-m selection, the canonical window of
the targets); this module only orders the calls and keeps tensors.  PyTorch
provides device memory, the synthetic instance generator (seeded torch
generators on the device) and the evaluation's bookkeeping (prefix maxima of
the score streams).

Instances (angular synchronisation): Q = x x^H + sigma W with x_i uniform on
A_8, sigma ~ U[0.5, 2], W Hermitian with CN(0, 1) entries above the diagonal
and N(0, 1) on it; V = the rank-4 truncation of Q (lrq_truncate).
Targets: the top 1% of S_train uniform directions by score, expressed in the
gauge of lrq_proposal_features and moved to the canonical window
arg c_1 in (-pi/K, pi/K] (Sec. 2.3: c and omega^k c score the same).
Metric: for a held-out instance, U* = the best score of S_max uniform
directions; S_u (S_l) = the shortest prefix of the uniform (learned) stream
whose best reaches 0.999 U*; reported as the median of S_u / S_l.  The
learned stream is the mixture's 16 component means by weight
(lrq_vmf_modes), then vMF draws.  The fixed-direction baseline stream is e_1
(the leading eigenvector's direction in the gauge), then the uniform stream.
"""
from __future__ import annotations

import math

import torch

from . import lrq

R = 4
K_ANGSYNC = 8
WIDTH = 256
N_OUT = 160


SIGMA_EASY = (0.5, 2.0)     # the angular-synchronisation workload: ||sigma W|| ~ 2 sigma sqrt(n) << n


def sigma_hard(n: int):
    """The high-noise regime: sigma sqrt(n) in [3n/16, 5n/16], so that
    ||sigma W|| ~ 2 sigma sqrt(n) ~ n / 2 is comparable to lambda_1 = n
    (sigma in [12, 20] at n = 4096)."""
    return (0.1875 * math.sqrt(n), 0.3125 * math.sqrt(n))


def make_instance(n: int, seed: int, device="cuda", sigma_range=SIGMA_EASY):
    """Q (n x n complex128 on the device), the planted x and sigma."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    k = torch.randint(0, K_ANGSYNC, (n,), generator=g, device=device)
    x = torch.polar(torch.ones(n, dtype=torch.float64, device=device), 2 * math.pi * k.double() / K_ANGSYNC)
    lo, hi = sigma_range
    sigma = lo + (hi - lo) * torch.rand((), generator=g, device=device, dtype=torch.float64).item()
    G = torch.randn((n, n), generator=g, device=device, dtype=torch.complex128)  # CN(0, 1)
    W = torch.triu(G, 1)
    W = W + W.conj().T
    W.diagonal().copy_(torch.randn(n, generator=g, device=device, dtype=torch.float64).to(torch.complex128))
    Q = torch.outer(x, x.conj()) + sigma * W
    return Q, k, sigma


def truncate_instances(n: int, seeds, device="cuda", sigma_range=SIGMA_EASY):
    """V (B x n x 4 complex64) and lambda (B x 4 float64) for each seed."""
    Vs, lams = [], []
    for s in seeds:
        Q, _, _ = make_instance(n, s, device, sigma_range)
        out = lrq.truncate(lrq.dense_matrix(Q), R, tol=1e-8, seed=int(s), want_c128=False, want_c64=True,
                           device=device)
        Vs.append(out["V32"])
        lams.append(out["lam"])
        del Q
    return torch.stack(Vs), torch.stack(lams)


def features(V, lam):
    B, n, r = V.shape
    F = lrq.lrq_proposal_num_features(r)
    Vg = torch.empty_like(V)
    feat = torch.empty((B, F), dtype=torch.float32, device=V.device)
    status = torch.zeros(1, dtype=torch.int32, device=V.device)
    lrq.lrq_proposal_features(V, lam, Vg, feat, status)
    lrq.check_status(status, "lrq_proposal_features")
    return Vg, feat


def uniform_scores(Vg, K: int, S: int, seed: int, want_C=False):
    """FP32 scores of S uniform directions (drawn on the device from seed)."""
    out = lrq.sample_score(Vg, K, C=None, S=S, seed=seed, mode=lrq.LRQ_MODE_FP32, top_m=1, want_scores=True)
    lrq.check_status(out["dev_status"], "uniform scoring")
    return (out["scores"], out["C"]) if want_C else out["scores"]


def scores_of(Vg, K: int, C):
    out = lrq.sample_score(Vg, K, C=C, mode=lrq.LRQ_MODE_FP32, top_m=1, want_scores=True)
    lrq.check_status(out["dev_status"], "proposal scoring")
    return out["scores"]


def training_targets(Vg, K: int, S_train: int, seed: int, frac=0.01):
    """Per instance the top frac of S_train uniform directions (the scoring's
    top-m selection), in the canonical window (lrq_proposal_targets)."""
    T = max(1, int(round(frac * S_train)))
    dev = Vg.device
    out = torch.empty((Vg.shape[0], T, 2 * R), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    for b in range(Vg.shape[0]):
        sc = lrq.sample_score(Vg[b], K, C=None, S=S_train, seed=seed + b, mode=lrq.LRQ_MODE_FP32, top_m=T)
        lrq.check_status(sc["dev_status"], "target scoring")
        lrq.lrq_proposal_targets(sc["C"], K, sc["top_idx"], out[b], status)
    lrq.check_status(status, "lrq_proposal_targets")
    return out  # B x T x 8


class Proposal:
    """Parameters, Adam state and feature standardisation of the network."""

    def __init__(self, F: int, seed: int = 0, device="cuda", bf16=True):
        self.F = F
        self.bf16 = bf16
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        shapes = [(F, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, N_OUT), (N_OUT,)]
        parts = []
        for shp in shapes:
            if len(shp) == 2:
                parts.append(torch.randn(shp, generator=g, device=device) * math.sqrt(2.0 / shp[0]))
            else:
                parts.append(torch.zeros(shp, device=device))
        p = torch.cat([t.reshape(-1) for t in parts])
        assert p.numel() == lrq.lrq_proposal_num_params(F)
        self.params = p.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.mean = torch.zeros(F, device=device)
        self.std = torch.ones(F, device=device)

    def standardize(self, feat):
        X = torch.empty_like(feat)
        lrq.lrq_standardize(feat.contiguous(), self.mean, self.std, X)
        return X

    def fit_standardizer(self, feat):
        lrq.lrq_standardize_fit(feat.contiguous(), self.mean, self.std)

    def forward(self, X):
        B = X.shape[0]
        H1 = torch.empty((B, WIDTH), device=X.device)
        H2 = torch.empty((B, WIDTH), device=X.device)
        O = torch.empty((B, N_OUT), device=X.device)
        lrq.lrq_mlp_forward(self.params, X, H1, H2, O, self.bf16)
        return O, (H1, H2)

    def train_step(self, X, targets, lr):
        B = X.shape[0]
        O, (H1, H2) = self.forward(X)
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
        dO = torch.empty_like(O)
        lrq.lrq_vmf_nll(O, targets, loss, dO)
        grads = torch.empty_like(self.params)
        scratch = torch.empty((2, B, WIDTH), device=X.device)
        lrq.lrq_mlp_backward(self.params, X, H1, H2, dO, grads, scratch, self.bf16)
        self.t += 1
        lrq.lrq_adam_step(self.params, grads, self.m, self.v, self.t, lr=lr)
        return loss

    def modes(self, X):
        O, _ = self.forward(X)
        C = torch.empty((X.shape[0], 16, R), dtype=torch.complex64, device=X.device)
        lrq.lrq_vmf_modes(O, C)
        return C

    def sample(self, X, S: int, K: int, seed: int):
        O, _ = self.forward(X)
        C = torch.empty((X.shape[0], S, R), dtype=torch.complex64, device=X.device)
        status = torch.zeros(1, dtype=torch.int32, device=X.device)
        lrq.lrq_vmf_sample(O, S, K, seed, C, status)
        lrq.check_status(status, "lrq_vmf_sample")
        return C


def train(model: Proposal, feat, targets, steps: int, batch: int, lr: float, seed: int = 0):
    B = feat.shape[0]
    X = model.standardize(feat)
    g = torch.Generator(device=feat.device)
    g.manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, B, (min(batch, B),), generator=g, device=feat.device)
        losses.append(model.train_step(X[idx].contiguous(), targets[idx].contiguous(), lr))
    return torch.cat(losses).cpu()


def prefix_to_reach(scores, target):
    """1-based length of the shortest prefix whose best reaches target (inf if none)."""
    hit = torch.nonzero(torch.cummax(scores, dim=0).values >= target)
    return float(hit[0, 0].item() + 1) if hit.numel() else math.inf


def evaluate(model: Proposal, Vg, feat, K: int, S_max: int, seed: int, level=0.999):
    """Per instance (U*, S_u, S_l, S_e1u, S_draws), each S the 1-based length of
    the shortest prefix of its stream reaching level U* (inf if none):
    S_u uniform directions; S_l the learned stream (16 modes, then
    S_max - 16 vMF draws); S_e1u the fixed direction e_1 followed by the
    uniform stream; S_draws the vMF draws alone."""
    X = model.standardize(feat)
    M = model.modes(X)
    C = model.sample(X, S_max - M.shape[1], K, seed)
    e1 = torch.zeros((1, R), dtype=torch.complex64, device=Vg.device)
    e1[0, 0] = 1.0
    rows = []
    for b in range(Vg.shape[0]):
        fu = uniform_scores(Vg[b], K, S_max, seed + 7919 * (b + 1))
        ustar = float(fu.max().item())
        lev = level * ustar
        fm = scores_of(Vg[b], K, M[b].contiguous())
        fd = scores_of(Vg[b], K, C[b].contiguous())
        fe = float(scores_of(Vg[b], K, e1).max().item())
        su = prefix_to_reach(fu, lev)
        rows.append((ustar, su, prefix_to_reach(torch.cat([fm, fd]), lev), 1.0 if fe >= lev else 1.0 + su,
                     prefix_to_reach(fd, lev)))
    return rows


def median_gain(rows, baseline=1):
    """Median of S_baseline / S_l (baseline 1: uniform sampling; 3: e_1, then
    uniform)."""
    ratios = sorted(r[baseline] / r[2] for r in rows)
    return ratios[len(ratios) // 2]


def reached_within(rows, col: int, budget: int) -> int:
    """Instances whose stream in column col reaches the level within budget draws."""
    return sum(1 for r in rows if r[col] <= budget)
