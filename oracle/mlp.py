"""Latency model of the learned planner, CPU reference.  TEST INFRASTRUCTURE ONLY.

A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (FP64
here), trained on the mean squared error; gradients by the chain rule,
written out layer by layer; updates by Adam (Kingma and Ba, 2015) with
bias correction.  Parameters are packed as W1 [in][h], b1 [h], W2 [h][h],
b2 [h], W3 [h][1], b3 [1] (row-major, x as a row vector, h = x W + b), the
order the library uses too.  Initial weights are inputs on both sides.
"""
import numpy as np


def sizes(n_in, hidden):
    return [(n_in, hidden), (hidden,), (hidden, hidden), (hidden,), (hidden, 1), (1,)]


def unpack(flat, n_in, hidden):
    out, off = [], 0
    for shp in sizes(n_in, hidden):
        k = int(np.prod(shp))
        out.append(np.asarray(flat[off:off + k], dtype=np.float64).reshape(shp))
        off += k
    return out


def pack(params):
    return np.concatenate([p.ravel() for p in params])


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1 + b1
    a1 = np.maximum(z1, 0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0)
    return (a2 @ W3 + b3)[:, 0], (z1, a1, z2, a2)


def loss_and_grads(params, X, y):
    """Mean squared error (1/n) sum (f(x) - y)^2 and its gradient."""
    W1, b1, W2, b2, W3, b3 = params
    n = X.shape[0]
    f, (z1, a1, z2, a2) = forward(params, X)
    r = f - y
    loss = float(np.mean(r * r))
    d3 = (2.0 / n) * r[:, None]            # dL/d(output)
    gW3 = a2.T @ d3
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3.T) * (z2 > 0)
    gW2 = a1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (z1 > 0)
    gW1 = X.T @ d1
    gb1 = d1.sum(axis=0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam(params, X, y, steps, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam; returns the parameters and the loss before each step."""
    params = [p.copy() for p in params]
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    losses = []
    for t in range(1, steps + 1):
        loss, g = loss_and_grads(params, X, y)
        losses.append(loss)
        for i in range(len(params)):
            m[i] = beta1 * m[i] + (1 - beta1) * g[i]
            v[i] = beta2 * v[i] + (1 - beta2) * g[i] * g[i]
            mh = m[i] / (1 - beta1 ** t)
            vh = v[i] / (1 - beta2 ** t)
            params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params, losses
