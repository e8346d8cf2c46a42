"""FP64 reference of the smooth-face gate MLP (24 -> 32 -> 32 -> 1, ReLU,
ReLU, sigmoid) and of its binary cross-entropy loss and gradient.

TEST INFRASTRUCTURE ONLY: the GPU training kernels' logits and gradients are
checked against these functions; the functions themselves are pinned by
central finite differences of the loss.  Parameter layout: W1[32][24], b1[32],
W2[32][32], b2[32], W3[32], b3 (1889 values).
"""
import numpy as np

NIN, NH = 24, 32
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init(seed=0):
    """He-style initialisation (used to start training)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / NIN), (NH, NIN)), "b1": np.zeros(NH),
         "W2": rng.normal(0, np.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": rng.normal(0, np.sqrt(1.0 / NH), NH), "b3": np.zeros(1)}
    return pack(d)


def forward(p, X):
    """Logits z and the hidden activations."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["W3"] + w["b3"][0]
    return z, (X, a1, h1, a2, h2)


def loss(p, X, y, pos_weight=1.0):
    """Mean weighted BCE: mean_i w_i (softplus(z_i) - y_i z_i), w_i = pos_weight if y_i else 1."""
    z, _ = forward(p, X)
    y = np.asarray(y, dtype=np.float64)
    wgt = np.where(y > 0, pos_weight, 1.0)
    sp = np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))
    return float(np.mean(wgt * (sp - y * z)))


def grad(p, X, y, pos_weight=1.0):
    """Analytic gradient of `loss` by back-propagation."""
    w = unpack(p)
    z, (X, a1, h1, a2, h2) = forward(p, X)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    wgt = np.where(y > 0, pos_weight, 1.0) / n
    dz = wgt * (1.0 / (1.0 + np.exp(-z)) - y)
    g = {"W3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, w["W3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return pack(g)
