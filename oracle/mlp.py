"""FP64 reference of the learned scheduler's network (test infrastructure only).

The network: x (16) -> z1 = W1 x + b1 -> h1 = GELU(z1) (64) -> z2 = W2 h1 + b2 ->
h2 = GELU(z2) (64) -> o = W3 h2 + b3 (17); GELU(z) = z * Phi(z) (exact, erf form).
Loss per sample: cross-entropy of softmax(o[0:16]) against class k-1, plus
(o[16] - priority)^2; the batch loss is the mean.  Parameters are one flat
vector in the order W1, b1, W2, b2, W3, b3 (row-major, output-major).

bf16_round() rounds FP32 values to bfloat16 (round to nearest, ties to even),
so that the reference can run with the same weights as the BF16 forward pass.
Pinned by finite differences and a zero-weight closed form in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, HID, OUT = 16, 64, 17
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(params[off:off + size], dtype=np.float64).reshape(shape)
        off += size
    return out


def pack(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SHAPES])


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, x):
    p = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (x, z1, h1, z2, h2)


def loss(params, x, k, prio):
    o, _ = forward(params, x)
    logits = o[:, :16]
    m = logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(logits - m).sum(axis=1)) + m[:, 0]
    kk = np.clip(np.asarray(k), 1, 16) - 1
    ce = lse - logits[np.arange(len(kk)), kk]
    return float(np.mean(ce + (o[:, 16] - np.asarray(prio, np.float64)) ** 2))


def loss_grad(params, x, k, prio):
    """Mean loss and its gradient with respect to the flat parameter vector."""
    p = unpack(params)
    o, (x, z1, h1, z2, h2) = forward(params, x)
    B = x.shape[0]
    logits = o[:, :16]
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    sm = e / e.sum(axis=1, keepdims=True)
    kk = np.clip(np.asarray(k), 1, 16) - 1
    diff = o[:, 16] - np.asarray(prio, np.float64)
    L = float(np.mean(np.log(e.sum(axis=1)) + m[:, 0] - logits[np.arange(B), kk] + diff ** 2))
    do = np.zeros_like(o)
    do[:, :16] = sm
    do[np.arange(B), kk] -= 1.0
    do[:, 16] = 2.0 * diff
    do /= B
    g = {"W3": do.T @ h2, "b3": do.sum(axis=0)}
    dz2 = (do @ p["W3"]) * gelu_grad(z2)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"], g["b1"] = dz1.T @ x, dz1.sum(axis=0)
    return L, pack(g)


def predict(params, x):
    o, _ = forward(params, x)
    return np.argmax(o[:, :16], axis=1).astype(np.int32) + 1, o[:, 16]
