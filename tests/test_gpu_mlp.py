"""The warm-start MLP's kernels against the FP64 reference network.

Gradients, loss and predictions of the CUDA path (BF16 GEMM operands, FP32
accumulation) are compared with oracle/mlp.py, which rounds to BF16 at the
same points and otherwise computes in FP64; the first Adam step is checked
against its closed form; training is checked to lower the loss and to be
deterministic."""

import numpy as np
import pytest

from oracle import mlp as M
from paper_2311_12180_gb300 import pdlp as P
from paper_2311_12180_gb300.warmstart import init_params

pytestmark = pytest.mark.gpu


def _blocks(din, h, dout):
    sizes = [din * h, h, h * h, h, h * dout, dout]
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    o = np.cumsum([0] + sizes)
    return [(names[i], slice(o[i], o[i + 1])) for i in range(6)]


def _problem(din, h, dout, samples, seed):
    rng = np.random.default_rng(seed)
    p = init_params(din, h, dout, seed).astype(np.float64)
    # non-zero biases so that every bias path is exercised
    for name, sl in _blocks(din, h, dout):
        if name.startswith("b"):
            p[sl] = rng.uniform(-0.2, 0.2, sl.stop - sl.start)
    p = p.astype(np.float32)
    X = rng.standard_normal((samples, din)).astype(np.float32)
    A = rng.standard_normal((din, dout))
    T = (np.tanh(X @ A / 3) * 4 + rng.uniform(-1, 1, dout) * 10).astype(np.float32)
    return p, X, T


@pytest.mark.parametrize("din,h,dout,batch", [(16, 64, 300, 32), (13, 72, 1100, 48), (16, 256, 2600, 40)])
def test_loss_and_gradients_match_oracle(din, h, dout, batch):
    p, X, T = _problem(din, h, dout, 100, din * 7 + dout)
    idx = np.random.default_rng(1).choice(100, batch, replace=False).astype(np.int32)
    with P.Mlp(din, h, dout, max_batch=64) as net:
        net.set_params(p)
        net.set_data(X, T)
        loss, g = net.gradients(idx)
        mu_d, sd_d = net.stats()
    mu, sd = M.standardise(T.astype(np.float64))
    assert np.allclose(mu_d, mu, rtol=1e-6, atol=1e-6) and np.allclose(sd_d, sd, rtol=1e-6)
    loss_o, g_o = M.loss_and_grads(p, X[idx], T[idx], mu, sd, din, h, dout, bf16_rounding=True)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    for name, sl in _blocks(din, h, dout):
        a, b = g[sl].astype(np.float64), g_o[sl]
        scale = np.abs(b).max()
        assert scale > 0, name
        # rounding the same FP32 value to BF16 on both sides differs only where
        # FP32 accumulation order moves a value across a rounding boundary
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b), name
        assert np.abs(a - b).max() <= 1e-2 * scale, name


def test_gradients_match_plain_fp64_network_loosely():
    # against the un-rounded FP64 network: BF16 operand rounding is the only
    # difference, about 2^-8 relative per operand
    din, h, dout, batch = 16, 64, 300, 32
    p, X, T = _problem(din, h, dout, 64, 5)
    idx = np.arange(batch, dtype=np.int32)
    with P.Mlp(din, h, dout, max_batch=batch) as net:
        net.set_params(p)
        net.set_data(X, T)
        loss, g = net.gradients(idx)
    mu, sd = M.standardise(T.astype(np.float64))
    loss_o, g_o = M.loss_and_grads(p, X[idx], T[idx], mu, sd, din, h, dout, bf16_rounding=False)
    assert loss == pytest.approx(loss_o, rel=3e-2)
    for name, sl in _blocks(din, h, dout):
        assert np.linalg.norm(g[sl] - g_o[sl]) <= 5e-2 * np.linalg.norm(g_o[sl]), name


@pytest.mark.parametrize("count", [1, 37, 300])
def test_predict_matches_oracle_forward(count):
    din, h, dout = 16, 96, 700
    p, X, T = _problem(din, h, dout, max(count, 50), 11)
    with P.Mlp(din, h, dout, max_batch=64) as net:  # predict runs in chunks of 64
        net.set_params(p)
        net.set_data(X, T)
        Y = net.predict(X[:count])
    mu, sd = M.standardise(T.astype(np.float64))
    Yo = M.forward(p, X[:count], M.f32(mu), M.f32(sd), din, h, dout, bf16_rounding=True)
    assert Y.shape == (count, dout)
    err = np.abs(Y - Yo) / sd
    assert err.max() <= 1e-2 and np.sqrt((err ** 2).mean()) <= 1e-3


def test_first_adam_step_closed_form():
    # Adam's first step moves every parameter by lr * g / (|g| + eps) against
    # the gradient (bias-corrected moments equal g and g^2)
    din, h, dout, batch = 16, 64, 300, 32
    p, X, T = _problem(din, h, dout, 64, 3)
    idx = np.arange(batch, dtype=np.int32)
    lr, eps = 1e-3, 1e-8
    with P.Mlp(din, h, dout, max_batch=batch) as net:
        net.set_params(p)
        net.set_data(X, T)
        _, g = net.gradients(idx)
        net.train(idx[None, :], lr=lr, eps=eps)
        p1 = net.get_params()
    g64 = g.astype(np.float64)
    expect = p.astype(np.float64) - lr * g64 / (np.abs(g64) + eps)
    assert np.abs(p1 - expect).max() <= 1e-6 + 1e-6 * np.abs(expect).max()


def test_training_lowers_loss_and_is_deterministic():
    din, h, dout = 16, 128, 400
    p, X, T = _problem(din, h, dout, 1024, 21)
    rng = np.random.default_rng(4)
    idx = np.stack([rng.choice(1024, 64, replace=False) for _ in range(400)]).astype(np.int32)
    runs = []
    for _ in range(2):
        with P.Mlp(din, h, dout, max_batch=64) as net:
            net.set_params(p)
            net.set_data(X, T)
            losses = net.train(idx, lr=2e-3)
            runs.append((losses, net.get_params()))
    losses = runs[0][0]
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_invalid_arguments_rejected():
    with P.Mlp(4, 8, 5, max_batch=8) as net:
        X = np.zeros((10, 4), np.float32)
        T = np.zeros((10, 5), np.float32)
        with pytest.raises(P.PdlpError):  # no data yet
            net.gradients(np.zeros(4, np.int32))
        net.set_data(X, T)
        with pytest.raises(P.PdlpError):  # batch above max_batch
            net.gradients(np.zeros(9, np.int32))
        with pytest.raises(P.PdlpError):  # index out of range
            net.train(np.full((2, 4), 10, np.int32))


def test_gemm_wait_timeout_is_reported_and_context_survives(monkeypatch):
    # one CTA of the first GEMM never receives its first operand stage: its
    # bounded mbarrier wait runs out (2 s), the call reports the error, and
    # the next call computes the same gradients as before
    din, h, dout, batch = 16, 64, 300, 32
    p, X, T = _problem(din, h, dout, 64, 8)
    idx = np.arange(batch, dtype=np.int32)
    with P.Mlp(din, h, dout, max_batch=batch) as net:
        net.set_params(p)
        net.set_data(X, T)
        loss0, g0 = net.gradients(idx)
        monkeypatch.setenv("PDLP_TEST_GEMM_STALL", "1")
        with pytest.raises(P.PdlpError) as e:
            net.gradients(idx)
        assert "timed out" in str(e.value)
        monkeypatch.delenv("PDLP_TEST_GEMM_STALL")
        loss1, g1 = net.gradients(idx)
    assert loss1 == loss0 and np.array_equal(g1, g0)
