"""FP64 CPU reference of the warm-start network (test infrastructure only).

Only tests may use this module.  It is the plain definition the GPU
training kernels are checked against: a point-set encoder -- a shared
per-point MLP 3 -> 128 -> 128 -> 256 with ReLU, a max over the points, and a
two-layer head 256 -> 256 (ReLU) -> n_out -- its mean-squared-error loss
against a target vector, and the loss gradients by the chain rule.  Nothing
here is from the paper (the warm start is not part of fast CPD); the network
predicts a starting point for the paper's EM loop.

Parameter layout (the GPU side uses the same order and shapes): for each
layer l, W_l (fan_in x fan_out, row-major) then b_l (fan_out):
    l0: 3 x 128, l1: 128 x 128, l2: 128 x 256, l3: 256 x 256, l4: 256 x n_out.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(3, 128), (128, 128), (128, 256), (256, 256)]   # + (256, n_out)


def shapes(n_out: int):
    return LAYERS + [(256, n_out)]


def unpack(params: np.ndarray, n_out: int):
    """Flat parameter vector -> [(W, b)] in layer order."""
    out, o = [], 0
    for fi, fo in shapes(n_out):
        W = params[o:o + fi * fo].reshape(fi, fo)
        o += fi * fo
        b = params[o:o + fo]
        o += fo
        out.append((W, b))
    assert o == params.size
    return out


def forward(params, Y, n_out):
    """Y: (B, N, 3).  Returns the prediction (B, n_out) and the activations."""
    P = unpack(np.asarray(params, np.float64), n_out)
    Y = np.asarray(Y, np.float64)
    B, N, _ = Y.shape
    h = Y.reshape(B * N, 3)
    acts = [h]
    for l in range(3):                                   # shared per-point MLP, ReLU
        W, b = P[l]
        h = np.maximum(h @ W + b, 0.0)
        acts.append(h)
    h3 = h.reshape(B, N, 256)
    g = h3.max(axis=1)                                   # max over the points
    arg = h3.argmax(axis=1)                              # first maximum (ties: lowest index)
    W, b = P[3]
    z = np.maximum(g @ W + b, 0.0)
    W, b = P[4]
    pred = z @ W + b
    return pred, dict(acts=acts, g=g, arg=arg, z=z)


def loss(pred, target):
    """Mean squared error over the batch and outputs."""
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    return float((d * d).mean())


def gradients(params, Y, target, n_out):
    """d loss / d params (flat, same layout) by the chain rule."""
    P = unpack(np.asarray(params, np.float64), n_out)
    Y = np.asarray(Y, np.float64)
    B, N, _ = Y.shape
    pred, a = forward(params, Y, n_out)
    dpred = 2.0 * (pred - np.asarray(target, np.float64)) / pred.size
    grads = [None] * 5
    # head
    W4, _ = P[4]
    grads[4] = (a["z"].T @ dpred, dpred.sum(0))
    dz = (dpred @ W4.T) * (a["z"] > 0)
    W3, _ = P[3]
    grads[3] = (a["g"].T @ dz, dz.sum(0))
    dg = dz @ W3.T                                       # (B, 256)
    # max-pool: the gradient goes to the arg-max point of each feature
    dh = np.zeros((B, N, 256))
    bi = np.arange(B)[:, None]
    fi = np.arange(256)[None, :]
    dh[bi, a["arg"], fi] = dg
    dh = dh.reshape(B * N, 256)
    for l in (2, 1, 0):
        W, _ = P[l]
        dpre = dh * (a["acts"][l + 1] > 0)
        grads[l] = (a["acts"][l].T @ dpre, dpre.sum(0))
        dh = dpre @ W.T
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def n_params(n_out: int) -> int:
    return sum(fi * fo + fo for fi, fo in shapes(n_out))
