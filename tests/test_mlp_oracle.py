"""Pins of the FP64 MLP reference (oracle/mlp_oracle.py): the analytic
gradient equals central finite differences of the loss; the loss has its
closed form at z = 0 (log 2 per sample)."""
import numpy as np

from oracle import mlp_oracle as mo


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mo.init(1)
    X = rng.normal(size=(40, mo.NIN))
    y = (rng.random(40) < 0.4).astype(np.float64)
    g = mo.grad(p, X, y, pos_weight=3.0)
    h = 1e-6
    idx = rng.choice(mo.NPARAM, size=60, replace=False)
    for i in idx:
        e = np.zeros(mo.NPARAM)
        e[i] = h
        fd = (mo.loss(p + e, X, y, 3.0) - mo.loss(p - e, X, y, 3.0)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_at_zero_logit_is_log2():
    p = np.zeros(mo.NPARAM)
    X = np.random.default_rng(2).normal(size=(10, mo.NIN))
    y = np.array([0, 1] * 5, dtype=np.float64)
    assert abs(mo.loss(p, X, y) - np.log(2.0)) < 1e-15
    assert mo.NPARAM == 1889
