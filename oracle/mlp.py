"""Float64 reference of the active-block predictor (TEST INFRASTRUCTURE ONLY).

Only tests/ and the benchmark may import this; it shares no code with the
CUDA library.  The predictor is a plain multilayer perceptron

    x~ = r(x),  h1 = r(relu(W1 x~ + b1)),  h2 = relu(W2 h1 + b2),
    z  = w3 . h2 + b3,

with 8 inputs, two hidden layers of 64 and one logit out, where r is the
rounding of a float32 value to bfloat16 (round to nearest, ties to even) when
`bf16` is set and the identity otherwise.  Its loss on a sample (x, y) is the
weighted binary cross entropy of the logit,

    l = w(y) * (softplus(z) - y z),   w(1) = pos_weight, w(0) = 1,

averaged over the samples; the gradient treats r as the identity
(straight-through).  Parameters are one flat vector in the order W1[64][8],
b1[64], W2[64][64], b2[64], w3[64], b3.

Pinned (tests/test_oracle_mlp.py) by finite differences of the loss, by
closed forms of hand-set weights, and by bfloat16 values fixed by the format.
"""
import numpy as np

N_IN, N_HID = 8, 64
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_HID + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    assert p.shape[0] == N_PARAMS
    o = 0
    W1 = p[o:o + N_HID * N_IN].reshape(N_HID, N_IN); o += N_HID * N_IN
    b1 = p[o:o + N_HID]; o += N_HID
    W2 = p[o:o + N_HID * N_HID].reshape(N_HID, N_HID); o += N_HID * N_HID
    b2 = p[o:o + N_HID]; o += N_HID
    w3 = p[o:o + N_HID]; o += N_HID
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16_round(x):
    """Round to bfloat16 (8-bit significand) after rounding to float32, ties
    to even; returned as float64.  (NaN and infinities are not used here.)"""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lower = u & 0xFFFF
    upper = u >> 16
    round_up = (lower > 0x8000) | ((lower == 0x8000) & ((upper & 1) == 1))
    upper = upper + round_up.astype(np.uint64)
    out = (upper << 16).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def forward(params, X, bf16=True):
    """Logits of the rows of X (N x 8).  Returns (z, cache)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_IN)
    r = bf16_round if bf16 else (lambda v: v)
    xr = r(X)
    a1 = xr @ W1.T + b1
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    return z, (xr, a1, h1, a2, h2)


def loss_and_grad(params, X, Y, pos_weight=1.0, bf16=True):
    """Mean weighted BCE over the samples and its gradient (flat vector)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    Y = np.asarray(Y, dtype=np.float64).reshape(-1)
    z, (xr, a1, h1, a2, h2) = forward(params, X, bf16)
    n = Y.shape[0]
    w = np.where(Y > 0.5, float(pos_weight), 1.0)
    softplus = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    loss = float(np.sum(w * (softplus - Y * z)) / n)
    p = 1.0 / (1.0 + np.exp(-z))
    dz = w * (p - Y) / n                       # dL/dz
    gw3 = h2.T @ dz
    gb3 = np.sum(dz)
    d2 = np.outer(dz, w3) * (a2 > 0)           # dL/da2
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)                  # dL/da1 (rounding passed through)
    gW1 = d1.T @ xr
    gb1 = d1.sum(0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)
