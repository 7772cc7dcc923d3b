"""FP64 reference of the warm-start network (test infrastructure only).

A plain numpy multilayer perceptron with the architecture and conventions of
the library's FP32 training kernels, written out layer by layer:

    x_std = (x - x_mean) / x_std            input standardisation
    h_1 = tanh(W_1 x_std + b_1), ..., h_L = tanh(W_L h_{L-1} + b_L)
    y_std = W_out h_L + b_out               linear output
    loss = mean over samples and outputs of (y_std - (y - y_mean)/y_std)^2

Parameters are flattened layer by layer as [W (out x in, row-major), b] for
the hidden layers then the output layer -- the order the library uses.  The
gradients are checked against central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(sizes):
    return [(sizes[i + 1], sizes[i]) for i in range(len(sizes) - 1)]


def n_params(sizes):
    return sum(o * i + o for o, i in layer_shapes(sizes))


def unflatten(theta, sizes):
    out, p = [], 0
    for o, i in layer_shapes(sizes):
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


def forward(theta, sizes, X, x_mean, x_std):
    layers = unflatten(np.asarray(theta, dtype=np.float64), sizes)
    h = (np.asarray(X, dtype=np.float64) - x_mean) / x_std
    acts = [h]
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.tanh(z) if li < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(theta, sizes, X, Y, x_mean, x_std, y_mean, y_std):
    """MSE loss (mean over n * outputs) in standardised output units and its
    gradient with respect to the flattened parameters (backpropagation)."""
    layers = unflatten(np.asarray(theta, dtype=np.float64), sizes)
    out, acts = forward(theta, sizes, X, x_mean, x_std)
    T = (np.asarray(Y, dtype=np.float64) - y_mean) / y_std
    n, m = T.shape
    diff = out - T
    loss = np.mean(diff ** 2)
    delta = 2.0 * diff / (n * m)          # d loss / d output
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h_prev = acts[li]
        gW = delta.T @ h_prev
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            delta = (delta @ W) * (1.0 - acts[li] ** 2)   # through tanh of layer li-1's output
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
