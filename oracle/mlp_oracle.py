"""Plain FP64 numpy reference of the guess network (test infrastructure only).

Architecture (the learned initial guess added beside the paper's method; the paper has
no counterpart): x_hat = (x - mu_x)/sd_x; a0 = tanh(W0 x_hat + b0); a1 = tanh(W1 a0 + b1);
a2 = tanh(W2 a1 + b2); y_hat = W3 a2 + b3; loss = mean over rows and outputs of
(y_hat - (y - mu_y)/sd_y)^2.  Gradients by the chain rule, written out layer by layer.
Pinned by central finite differences in tests/test_oracle_pins_mlp.py.  Parameters are
the flat array W0 [H][F], b0, W1 [H][H], b1, W2 [H][H], b2, W3 [O][H], b3.
"""
import numpy as np


def unpack(p, F, H, O):
    dims = [F, H, H, H, O]
    out, o = [], 0
    for l in range(4):
        W = p[o:o + dims[l + 1] * dims[l]].reshape(dims[l + 1], dims[l])
        o += dims[l + 1] * dims[l]
        b = p[o:o + dims[l + 1]]
        o += dims[l + 1]
        out.append((W, b))
    return out


def forward(p, norm, X, F, H, O):
    layers = unpack(np.asarray(p, dtype=np.float64), F, H, O)
    mu_x, sd_x = norm[:F], norm[F:2 * F]
    a = (X - mu_x) / sd_x
    acts = [a]
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.tanh(z) if l < 3 else z
        acts.append(a)
    return acts


def loss_grad(p, norm, X, Y, F, H, O):
    p = np.asarray(p, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    norm = np.asarray(norm, dtype=np.float64)
    layers = unpack(p, F, H, O)
    acts = forward(p, norm, X, F, H, O)
    mu_y, sd_y = norm[2 * F:2 * F + O], norm[2 * F + O:]
    t = (Y - mu_y) / sd_y
    e = acts[4] - t
    n = X.shape[0]
    loss = float((e ** 2).sum() / (n * O))
    d = 2.0 * e / (n * O)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, b = layers[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * (1.0 - acts[l] ** 2)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def predict(p, norm, X, F, H, O):
    norm = np.asarray(norm, dtype=np.float64)
    y = forward(p, norm, np.asarray(X, dtype=np.float64), F, H, O)[4]
    return y * norm[2 * F + O:] + norm[2 * F:2 * F + O]
