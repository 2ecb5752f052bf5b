"""FP64 CPU reference of the warm-start network (test infrastructure only).

A multilayer perceptron y = W_L tanh(... tanh(W_1 x + b_1) ...) + b_L with
tanh on every hidden layer and a linear output, the mean-squared error
    loss = 1/(n m) sum_s sum_j (y_sj - t_sj)^2
over n samples and m outputs, its gradient by the chain rule written out by
hand, and one Adam update (Kingma & Ba, bias-corrected moments).  It shares
no code with the CUDA kernels it checks; its gradient is itself checked
against central finite differences by tests/test_oracle_pins.py.

Parameters are a list [(W_1, b_1), ..., (W_L, b_L)] with W_l of shape
(out_l, in_l), FP64.
"""
from __future__ import annotations

import numpy as np


def init_params(sizes, seed: int = 0):
    """Uniform +-sqrt(6 / (in + out)) weights (Glorot), zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        out.append((rng.uniform(-a, a, (fan_out, fan_in)), np.zeros(fan_out)))
    return out


def forward(params, x):
    """Returns the output and the list of layer outputs (input first)."""
    acts = [np.asarray(x, dtype=np.float64)]
    for l, (W, b) in enumerate(params):
        z = acts[-1] @ W.T + b
        acts.append(np.tanh(z) if l + 1 < len(params) else z)
    return acts[-1], acts


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def gradients(params, x, t):
    """d loss / d (W_l, b_l) for every layer, by back-propagation:
    dL/dy = 2 (y - t) / (n m); for a layer z = a W^T + b: dL/dW = dz^T a,
    dL/db = sum_s dz, dL/da = dz W; through tanh, dz = da (1 - tanh(z)^2)."""
    y, acts = forward(params, x)
    n, m = y.shape
    dz = 2.0 * (y - t) / (n * m)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        a = acts[l]
        grads[l] = (dz.T @ a, dz.sum(axis=0))
        if l > 0:
            da = dz @ W
            dz = da * (1.0 - a * a)          # a = tanh(z) of layer l - 1
    return grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; state = (step, [(mW, mb)], [(vW, vb)]) or None."""
    if state is None:
        state = (0, [(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                 [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    step, m, v = state
    step += 1
    new, m2, v2 = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        mW = beta1 * mW + (1 - beta1) * gW
        mb = beta1 * mb + (1 - beta1) * gb
        vW = beta2 * vW + (1 - beta2) * gW * gW
        vb = beta2 * vb + (1 - beta2) * gb * gb
        c1, c2 = 1 - beta1 ** step, 1 - beta2 ** step
        new.append((W - lr * (mW / c1) / (np.sqrt(vW / c2) + eps), b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)))
        m2.append((mW, mb))
        v2.append((vW, vb))
    return new, (step, m2, v2)


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, sizes):
    out, o = [], 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = vec[o:o + fan_in * fan_out].reshape(fan_out, fan_in)
        o += fan_in * fan_out
        b = vec[o:o + fan_out]
        o += fan_out
        out.append((W.copy(), b.copy()))
    return out
