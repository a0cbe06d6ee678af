"""Oracle of the learned pre-flagger: backward pass against central finite
differences, Adam's first step, features on fields with known gradients."""
import numpy as np

from oracle import mlp as M
from paper_2211_12867_gb300 import inputs as I


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = I.mlp_init(3)
    X = rng.uniform(0, 0.5, (16, 64))
    t = (rng.random(16) < 0.4).astype(float)
    g = M.grad(theta, X, t)
    idx = np.concatenate([rng.integers(0, M.N_PARAMS, 60), [M.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss(tp, X, t) - M.loss(tm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_is_a_signed_lr_step():
    theta = np.zeros(5)
    g = np.array([1.0, -2.0, 3e-3, 0.0, -1e-4])
    th, m, v = M.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, lr=1e-3)
    assert np.allclose(th[[0, 1, 2]], -1e-3 * np.sign(g[[0, 1, 2]]), rtol=1e-4)
    assert th[3] == 0.0


def test_features_of_an_index_linear_density():
    n = (12, 12, 12)
    P = np.zeros((8,) + tuple(s + 4 for s in n))
    j = np.arange(n[1] + 4)[None, :, None] - 2
    rho = 2.0 + 0.1 * j * np.ones(P.shape[1:])
    P[0] = rho
    P[1] = rho * 5.0           # v_r = 5 everywhere: no gradient
    P[4] = 1.0 / 0.5 + 0.5 * P[1] ** 2 / rho     # p = 1 with gamma = 1.5
    f = M.features_from_padded(P, 1.5)
    # per cell: |d rho| / rho / 3 with central differences of 0.1 per index
    jj = np.arange(12)
    cell = 0.1 / (2.0 + 0.1 * jj) / 3.0
    for b in range(4):
        expect = cell[3 * b:3 * b + 3].mean()
        assert np.allclose(f.reshape(4, 4, 4)[:, b, :], expect, rtol=1e-12)
    assert np.all(f > 0)
