"""FP64 reference of the learned stand-in's network (test infrastructure only).

A plain numpy statement of what the engine's quantile network computes: an MLP
32-256-256-256-256-16 with ReLU on the hidden layers, the pinball loss
sum_j mask_j rho_tau_j(y_j - yhat_j) averaged over rows, with
rho_tau(u) = u (tau - 1[u < 0]), and its gradient by backpropagation.
Parameters are one flat vector: for each layer W [out x in] row-major, then b.
Optionally the weights and layer inputs are rounded to bfloat16 first, as the
tensor-core path does.  The paper has no counterpart of this network.
"""
from __future__ import annotations

import numpy as np

DIMS = [32, 256, 256, 256, 256, 16]
N_PARAMS = sum(DIMS[i] * DIMS[i + 1] + DIMS[i + 1] for i in range(len(DIMS) - 1))


def bf16(a):
    """Round to bfloat16 (round to nearest even) and return as float64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for i in range(len(DIMS) - 1):
        n_in, n_out = DIMS[i], DIMS[i + 1]
        W = p[o:o + n_in * n_out].reshape(n_out, n_in)
        o += n_in * n_out
        b = p[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


def forward(p, x, round_bf16=False):
    """Returns the list of layer inputs and the output."""
    layers = unpack(p)
    h = np.asarray(x, dtype=np.float64)
    inputs = []
    for i, (W, b) in enumerate(layers):
        hin = bf16(h) if round_bf16 else h
        Wr = bf16(W) if round_bf16 else W
        inputs.append(h)
        z = hin @ Wr.T + b
        h = np.maximum(z, 0.0) if i < len(layers) - 1 else z
    return inputs, h


def pinball(yhat, y, tau, mask):
    u = y - yhat
    return float(np.sum(mask * u * (tau - (u < 0))) / yhat.shape[0])


def grad(p, x, y, tau, mask, round_bf16=False):
    """Mean pinball loss and its gradient with respect to the flat parameters."""
    layers = unpack(p)
    inputs, yhat = forward(p, x, round_bf16)
    rows = yhat.shape[0]
    u = y - yhat
    G = -mask * (tau - (u < 0)) / rows                 # d loss / d yhat
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        hin = bf16(inputs[i]) if round_bf16 else inputs[i]
        Wr = bf16(W) if round_bf16 else W
        grads.append((G.T @ hin, G.sum(0)))
        if i > 0:
            Gin = bf16(G) @ Wr if round_bf16 else G @ Wr
            G = Gin * (inputs[i] > 0)                  # ReLU of the layer that produced inputs[i]
    flat = []
    for dW, db in reversed(grads):
        flat += [dW.ravel(), db]
    return pinball(yhat, y, tau, mask), np.concatenate(flat), yhat
