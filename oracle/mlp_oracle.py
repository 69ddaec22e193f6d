"""CPU oracle of the autotuner's cost model (test infrastructure only).

Plain numpy float64 versions of the network, its mean-squared-error gradient
and one Adam step, following the same parameter layout as the library's
dkss_mlp_* kernels (include/dkss.h): W1[H][F], b1[H], W2[H][H], b2[H], w3[H],
b3.  Pins (tests/test_oracle_pins.py): the gradient against central finite
differences, the forward pass against a closed form, the first Adam step
against its closed form -lr * g / (|g| + eps).
"""
import numpy as np

F = 12
H = 32
NPARAM = H * F + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x):
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for each row of x."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(p, x, t):
    return float(np.mean((forward(p, x) - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, x, t):
    """Gradient of loss(p, x, t) by back-propagation."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    dy = 2.0 * (y - t) / B
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def adam_step(p, g, m1, m2, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015); returns (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
