"""Warm-start network of the learned local stage: plain FP64 reference.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module; the library never does.

The paper does not contain this part: it only suggests (Sec. 6) that local
spaces computed once could be reused for new inputs.  The build's warm start
maps a subdomain's ply-angle perturbation field to an initial block for the
local eigensolver.  What is computed here is the textbook definition of each
piece, written out without any blocking or fusion:

* a multilayer perceptron with tanh hidden layers and a linear output layer,
  y = W_L tanh(... tanh(W_1 x + b_1) ...) + b_L, weights stored [out][in];
* the mean-squared-error loss L = 1/(B d) sum (y - t)^2 over a batch of B
  rows with d outputs each, and its gradients by the chain rule;
* one Adam step (Kingma and Ba, "Adam: A Method for Stochastic
  Optimization", ICLR 2015, Algorithm 1) with bias-corrected moments;
* orthogonal Procrustes alignment of a basis to a reference basis
  (Schoenemann 1966: Q = U V^T from the SVD U S V^T of X^T X_ref);
* the largest principal angle between two subspaces (Bjorck and Golub 1973:
  arccos of the smallest singular value of Q_x^T Q_y).

Parameters travel as one flat vector in the order W_1, b_1, W_2, b_2, ...,
the layout the C ABI uses.
"""
import numpy as np


def param_count(sizes):
    """Number of parameters of an MLP with layer widths ``sizes``."""
    return sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))


def unpack(params, sizes):
    """Flat parameter vector -> list of (W [out][in], b [out]) views."""
    params = np.asarray(params)
    out, off = [], 0
    for i in range(len(sizes) - 1):
        n_in, n_out = sizes[i], sizes[i + 1]
        W = params[off:off + n_out * n_in].reshape(n_out, n_in)
        off += n_out * n_in
        b = params[off:off + n_out]
        off += n_out
        out.append((W, b))
    if off != params.size:
        raise ValueError("parameter vector does not match the layer sizes")
    return out


def forward(params, sizes, X):
    """Forward pass over a batch X [B][sizes[0]].

    Returns (Y, acts): Y [B][sizes[-1]] and the list of layer inputs
    (acts[0] = X, acts[l] = tanh output of hidden layer l) kept for backward.
    """
    layers = unpack(np.asarray(params, dtype=np.float64), sizes)
    h = np.asarray(X, dtype=np.float64)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if l + 1 < len(layers):
            h = np.tanh(z)
            acts.append(h)
        else:
            h = z
    return h, acts


def mse(Y, T):
    """Mean-squared error over all B x d entries."""
    D = np.asarray(Y, dtype=np.float64) - np.asarray(T, dtype=np.float64)
    return float(np.mean(D * D))


def backward(params, sizes, X, T):
    """Loss and gradient (flat, same layout as ``params``) of mse(forward(X), T)."""
    layers = unpack(np.asarray(params, dtype=np.float64), sizes)
    Y, acts = forward(params, sizes, X)
    T = np.asarray(T, dtype=np.float64)
    B, d = Y.shape
    loss = float(np.mean((Y - T) ** 2))
    g = 2.0 * (Y - T) / (B * d)          # dL/dY
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h_in = acts[l]
        gW = g.T @ h_in                   # [out][in]
        gb = g.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            g = (g @ W) * (1.0 - acts[l] ** 2)   # through tanh of the layer below
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1).  Returns (params, m, v), new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return params - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def procrustes(X, X_ref):
    """X Q with Q orthogonal minimising ||X Q - X_ref||_F (both [n][k])."""
    U, _, Vt = np.linalg.svd(np.asarray(X).T @ np.asarray(X_ref))
    return np.asarray(X) @ (U @ Vt)


def max_angle(X, Y):
    """Largest principal angle (radians) between span(X) and span(Y), Euclidean."""
    Qx, _ = np.linalg.qr(np.asarray(X, dtype=np.float64))
    Qy, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64))
    s = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))
