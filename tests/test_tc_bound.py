"""The error bound the GPU parity tests allow the tensor-core scoring mode
(test_gpu_parity._tc_bound), checked against a numpy emulation of that
mode's arithmetic (tests/tc_emulator.py: F16 projections with F16
accumulation, sign decisions, hi + lo E4M3 class sums in FP32): the
emulated scores stay inside the bound, including on rows spread over many
orders of magnitude, and the bound is not vacuous."""
import numpy as np
import pytest

import oracle as O
import tc_emulator as E
from paper_2602_20376_gb300 import inputs as I
from test_gpu_parity import _tc_bound


def test_e4m3_rounding():
    # exact values stay, halfway cases go to the even significand, the
    # subnormal step is 2^-9, the largest finite value is 448
    assert E.e4m3(1.0) == 1.0 and E.e4m3(-1.0) == -1.0
    assert E.e4m3(1.0625) == 1.0 and E.e4m3(1.1875) == 1.25
    assert E.e4m3(2.0 ** -9) == 2.0 ** -9 and E.e4m3(2.0 ** -11) == 0.0
    assert E.e4m3(448.0) == 448.0 and E.e4m3(1000.0) == 448.0
    x = np.linspace(-300, 300, 20001)
    err = np.abs(E.e4m3(x) - x)
    assert np.all(err <= np.maximum(np.abs(x) * 2.0 ** -4, 2.0 ** -10) + 1e-12)


@pytest.mark.parametrize("n,r,K,S,seed", [(96, 4, 3, 48, 1), (80, 4, 4, 40, 2), (64, 2, 2, 32, 3),
                                           (70, 3, 5, 30, 4), (64, 4, 8, 24, 5)])
def test_emulated_scores_within_the_bound(n, r, K, S, seed):
    V = I.factor(n, r, seed=seed, scales=np.linspace(2.0, 0.5, r), dtype=np.complex64)
    C = I.directions(S, r, seed=seed + 100)
    f = E.score(V, K, C)
    ref = O.score(V, K, C)
    bound = _tc_bound(V, K, C) + 1e-5 * np.sqrt(ref)
    dev = np.abs(np.sqrt(f) - np.sqrt(ref))
    assert np.all(dev <= bound), (np.max(dev / bound), np.argmax(dev / bound))
    assert np.max(dev / bound) > 1e-4  # the bound is not vacuous


@pytest.mark.parametrize("K", [3, 4])
def test_emulated_heavy_tailed_rows_within_the_bound(K):
    # rows over ten orders of magnitude: the per-coordinate scales of GEMM2
    rng = np.random.default_rng(9)
    V = I.factor(64, 4, seed=9, dtype=np.complex64)
    V = (V * (10.0 ** rng.uniform(-10, 0, size=64))[:, None]).astype(np.complex64)
    C = I.directions(32, 4, seed=10)
    f = E.score(V, K, C)
    ref = O.score(V, K, C)
    bound = _tc_bound(V, K, C) + 1e-5 * np.sqrt(ref)
    assert np.all(np.abs(np.sqrt(f) - np.sqrt(ref)) <= bound)


def test_k3_middle_line_needs_one_scale_per_coordinate():
    # p_1 = -(p_0 + p_2) is read from an F16 sum of two projections: with a
    # power-of-two scale per line instead of per coordinate the sum mixes
    # scales, and the heavy-tailed case leaves the bound
    rng = np.random.default_rng(9)
    V = I.factor(64, 4, seed=9, dtype=np.complex64)
    V = (V * (10.0 ** rng.uniform(-10, 0, size=64))[:, None]).astype(np.complex64)
    C = I.directions(32, 4, seed=10)
    ref = O.score(V, 3, C)
    bound = _tc_bound(V, 3, C) + 1e-5 * np.sqrt(ref)
    f = E.score(V, 3, C, per_line_scale=True)
    assert np.any(np.abs(np.sqrt(f) - np.sqrt(ref)) > bound)
