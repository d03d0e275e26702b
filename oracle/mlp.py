"""Learned tendency correction: FP64 CPU reference (oracle; test infrastructure).

The paper has no learned component; this is the reference for the small
per-node MLP of the learned coarse-grid correction.  Written from the
definitions, with backpropagation by hand:

  features  x_i = [(U_f(x_j) - U_f(x_i)) / s_in[f]  for f in 0..3, j in the
                   stencil of i after the centre]          (4 (n-1) values)
                  followed by the node's own values U_f(x_i) / s_own[f]   (4)
  network   f(x) = h2 W3 + b3, h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2)
            y = f(x) - f(0): a locally uniform state (all differences zero)
            gets no correction, as the fine and coarse steps agree there
  output    delta_f = y_f * s_out[f]   (a tendency, added as dt * delta)
  loss      L = mean over samples and outputs of (y - t / s_out)^2

Weights are used as given; a caller that runs the network in BF16 passes
BF16-rounded weights (``bf16_round``) so both sides take the same values.
"""
import numpy as np


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    a32 = np.asarray(a, np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, n_in, width, n_out=4):
    """Split a flat parameter vector [W1, b1, W2, b2, W3, b3] (row-major)."""
    p = np.asarray(params, np.float64)
    o = 0
    shapes = [(n_in, width), (width,), (width, width), (width,), (width, n_out), (n_out,)]
    out = []
    for shp in shapes:
        k = int(np.prod(shp))
        out.append(p[o:o + k].reshape(shp))
        o += k
    return out


def features(U, idx, nodes_i, s_in, s_own):
    """Scaled stencil differences and own values of nodes ``nodes_i`` of the
    state U [4, n_all] (ghosts filled) with stencils idx [N, n], centre first:
    [len(nodes_i), 4(n-1) + 4]."""
    U = np.asarray(U, np.float64)
    nb = idx[nodes_i, 1:]                                   # [B, n-1]
    diff = U[:, nb] - U[:, nodes_i][:, :, None]             # [4, B, n-1]
    diff = diff / np.asarray(s_in, np.float64)[:, None, None]
    own = (U[:, nodes_i] / np.asarray(s_own, np.float64)[:, None]).T
    return np.concatenate([diff.transpose(1, 0, 2).reshape(len(nodes_i), -1), own], axis=1)


def forward(X, params, n_in, width):
    """Hidden activations and y = f(X) - f(0)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, width)
    h1 = np.tanh(X @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    z1 = np.tanh(b1)
    z2 = np.tanh(z1 @ W2 + b2)
    return h1, h2, (h2 @ W3 + b3) - (z2 @ W3 + b3)


def loss_and_grad(X, T, params, n_in, width):
    """Loss and its gradient with respect to the flat parameters; T holds the
    scaled targets t / s_out [B, 4]."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, width)
    h1, h2, y = forward(X, params, n_in, width)
    B = X.shape[0]
    r = y - T
    L = np.mean(r * r)
    dy = 2.0 * r / (B * y.shape[1])
    # the x = 0 branch enters with the opposite sign and the summed dy
    z1 = np.tanh(b1)
    z2 = np.tanh(z1 @ W2 + b2)
    dz = -dy.sum(axis=0)
    dW3 = h2.T @ dy + np.outer(z2, dz)
    db3 = dy.sum(axis=0) + dz
    dh2 = (dy @ W3.T) * (1.0 - h2 * h2)
    dz2 = (W3 @ dz) * (1.0 - z2 * z2)
    dW2 = h1.T @ dh2 + np.outer(z1, dz2)
    db2 = dh2.sum(axis=0) + dz2
    dh1 = (dh2 @ W2.T) * (1.0 - h1 * h1)
    dz1 = (W2 @ dz2) * (1.0 - z1 * z1)
    dW1 = X.T @ dh1
    db1 = dh1.sum(axis=0) + dz1
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g


def n_params(n_in, width, n_out=4):
    return n_in * width + width + width * width + width + width * n_out + n_out
