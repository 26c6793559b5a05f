"""FP64 reference of the warm-start MLP (test infrastructure only).

in -> hidden -> ReLU -> hidden -> ReLU -> out, loss = mean squared error on
per-output standardised targets.  With bf16=True every quantity the CUDA
path rounds to BF16 (inputs, weights as GEMM operands, hidden activations,
the output gradient and the hidden-layer gradients as GEMM operands) is
rounded here at the same point, all arithmetic otherwise FP64, so the two
sides differ only by FP32 accumulation order.  With bf16=False it is the
plain FP64 network, pinned by finite differences in the tests.

Parameter layout (flat): W1 (in x hidden), b1, W2 (hidden x hidden), b2,
W3 (hidden x out), b3; W row-major [in][out].
"""

from __future__ import annotations

import numpy as np


def bf16(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def unpack(p, din, h, dout):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((din, h), (h,), (h, h), (h,), (h, dout), (dout,)):
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape))
        o += k
    assert o == p.size
    return out


def standardise(T):
    """Per-output mean and (population) standard deviation, floored at 1e-6."""
    T = np.asarray(T, dtype=np.float64)
    mu = T.mean(axis=0)
    sd = np.sqrt(((T - mu) ** 2).mean(axis=0))
    return mu, np.maximum(sd, 1e-6)


def loss_and_grads(p, X, T, mu, sd, din, h, dout, bf16_rounding=True):
    """Loss and flat gradient for inputs X (B x in) and raw targets T (B x out)."""
    r = bf16 if bf16_rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p, din, h, dout)
    if bf16_rounding:
        b1, b2, b3, mu, sd = f32(b1), f32(b2), f32(b3), f32(mu), f32(sd)
    X = r(X)
    W1r, W2r, W3r = r(W1), r(W2), r(W3)
    H1 = r(np.maximum(X @ W1r + b1, 0.0))
    H2 = r(np.maximum(H1 @ W2r + b2, 0.0))
    Y = H2 @ W3r + b3
    Tt = (np.asarray(T, dtype=np.float64) - mu) / sd
    D = Y - Tt
    B, O = D.shape
    loss = float((D * D).mean())
    dY = 2.0 * D / (B * O)
    dYr = r(dY)
    gW3 = H2.T @ dYr
    gb3 = dY.sum(axis=0)
    dZ2 = (dYr @ W3r.T) * (H2 > 0)
    dZ2r = r(dZ2)
    gW2 = H1.T @ dZ2r
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2r @ W2r.T) * (H1 > 0)
    dZ1r = r(dZ1)
    gW1 = X.T @ dZ1r
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def forward(p, X, mu, sd, din, h, dout, bf16_rounding=True):
    """Prediction in target units."""
    r = bf16 if bf16_rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p, din, h, dout)
    H1 = r(np.maximum(r(X) @ r(W1) + b1, 0.0))
    H2 = r(np.maximum(H1 @ r(W2) + b2, 0.0))
    return (H2 @ r(W3) + b3) * sd + mu
