"""Pins for the FP64 reference MLP: finite differences of the plain FP64
network, and the BF16-rounding emulation against numpy's own casts."""

import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_rounding_matches_round_to_nearest_even():
    # values with known bfloat16 images (8 significant bits)
    v = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, 3.140625, -2.5, 65504.0, 1e-30], dtype=np.float64)
    r = M.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway 1 + 2^-8 -> ties to even (1.0)
    assert r[2] == 1.0078125  # above halfway -> up
    assert r[3] == 1.0078125
    assert r[4] == 3.140625 and r[5] == -2.5
    # every result has at most 8 significant bits
    m, e = np.frexp(r[r != 0])
    assert np.all((m * 256) == np.round(m * 256))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    din, h, dout, B = 5, 7, 6, 4
    n = din * h + h + h * h + h + h * dout + dout
    p = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((B, din))
    T = rng.standard_normal((B, dout)) * 2 + 1
    mu, sd = M.standardise(T)
    loss, g = M.loss_and_grads(p, X, T, mu, sd, din, h, dout, bf16_rounding=False)
    eps = 1e-6
    for i in rng.choice(n, 40, replace=False):
        d = np.zeros(n)
        d[i] = eps
        lp, _ = M.loss_and_grads(p + d, X, T, mu, sd, din, h, dout, bf16_rounding=False)
        lm, _ = M.loss_and_grads(p - d, X, T, mu, sd, din, h, dout, bf16_rounding=False)
        assert g[i] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-9)


def test_standardised_targets_have_zero_loss_at_exact_fit():
    # a network whose output layer reproduces the standardised targets exactly
    din, h, dout, B = 3, 4, 2, 5
    rng = np.random.default_rng(1)
    T = rng.standard_normal((B, dout))
    mu, sd = M.standardise(T)
    p = np.zeros(din * h + h + h * h + h + h * dout + dout)
    # zero weights: output = b3; loss = mean(((T - mu)/sd - b3)^2) = 1 for b3 = 0
    loss, _ = M.loss_and_grads(p, rng.standard_normal((B, din)), T, mu, sd, din, h, dout, bf16_rounding=False)
    assert loss == pytest.approx(1.0, rel=1e-12)
