"""Oracle: the small MLP of the learned smoother parameters (plain numpy, fp64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

North-star extension, not in the paper (the paper fixes omega = 1 and the
weight transition): a network 6 -> 64 tanh -> 64 tanh -> 2 maps level features
to two raw outputs.  Parameters packed as W1[6][64], b1[64], W2[64][64], b2[64],
W3[64][2], b3[2].  Loss: weighted mean squared error
(1/B) sum_b w_b sum_o (y_bo - t_bo)^2.  The gradient is the chain rule written
out; tests pin it against central finite differences.  Adam: Kingma & Ba (2015),
bias-corrected moments.
"""
import numpy as np

IN, HID, OUT = 6, 64, 2
SIZES = [("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("W3", (HID, OUT)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def init(seed=0):
    """Glorot-uniform weights, zero biases."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            p[name] = g.uniform(-lim, lim, size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def forward(theta, x):
    p = unpack(theta)
    h1 = np.tanh(x @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    y = h2 @ p["W3"] + p["b3"]
    return y, h1, h2


def loss(theta, x, t, w=None):
    y, _, _ = forward(theta, x)
    B = x.shape[0]
    w = np.ones(B) if w is None else np.asarray(w, dtype=np.float64)
    return float(np.sum(w[:, None] * (y - t) ** 2) / B)


def grad(theta, x, t, w=None):
    """Analytic gradient of loss() by the chain rule."""
    p = unpack(theta)
    y, h1, h2 = forward(theta, x)
    B = x.shape[0]
    w = np.ones(B) if w is None else np.asarray(w, dtype=np.float64)
    dy = 2.0 * w[:, None] * (y - t) / B            # d loss / d y
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"].T) * (1.0 - h2 ** 2)       # through tanh
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"].T) * (1.0 - h1 ** 2)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
