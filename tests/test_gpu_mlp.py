"""Learned pre-flagger on the GPU against the NumPy oracle: features,
forward, gradients (FP32 kernels vs FP64 oracle, element by element), Adam,
training, and what the trained network gains over the plain estimator."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import make_pair, wind_setup
from oracle import mlp as M
from paper_2211_12867_gb300 import harness as H
from paper_2211_12867_gb300 import inputs as I

pytestmark = pytest.mark.gpu
STR = dict(x_min=(0.1, math.pi / 6, 0.0), x_max=(2.0, 5 * math.pi / 6, 2 * math.pi), stretch=True)


def _grad_magnitudes(theta, X, T):
    """Running-error magnitudes of the gradient: the same chain with every
    sum taken over absolute values (forward pre-activations, the output error
    y - t as |y| + |t| plus the sigmoid's sensitivity, backward products), so
    that |g_fp32 - g_exact| <= c eps_32 mag for a modest c."""
    W1, b1, W2, b2, w3, b3 = M.unpack(theta)
    y, (_, a1, h1, a2, h2, z) = M.forward(theta, X)
    B = X.shape[0]
    m1, m2 = a1 > 0, a2 > 0
    h1m = (np.abs(X) @ np.abs(W1).T + np.abs(b1)) * m1
    h2m = (h1m @ np.abs(W2).T + np.abs(b2)) * m2
    zm = h2m @ np.abs(w3) + abs(b3)
    dzm = (np.abs(y) + np.abs(T) + y * (1 - y) * zm) / B
    dh2m = np.outer(dzm, np.abs(w3)) * m2
    dh1m = (dh2m @ np.abs(W2)) * m1
    return np.concatenate([(dh1m.T @ np.abs(X)).ravel(), dh1m.sum(0), (dh2m.T @ h1m).ravel(), dh2m.sum(0),
                           h2m.T @ dzm, [dzm.sum()]])


def test_features_match_oracle():
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), **STR)
    wind_setup(g, o)
    g.step(20)
    o.set_state(g.get_state(0))
    o.t = g.step(0)[0]
    o.ghost_fill()
    F = g.mlp_features()
    for n in range(o.nleaves):
        ref = M.features_from_padded(o.get_padded(n, 0), 1.5)
        assert np.allclose(F[n], ref, rtol=2e-5, atol=1e-7), n


def test_features_are_deterministic():
    """The features of a leaf are the same bits on every call and for every
    ensemble member holding the same state (the sub-cube sums reduce in a
    fixed order)."""
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), n_members=2, **STR)
    wind_setup(g, o, member=0)
    wind_setup(g, o, member=1)
    g.step(10)
    F1, F2 = g.mlp_features(), g.mlp_features()
    assert np.array_equal(F1, F2)
    n0 = g.n_leaves(0)
    assert np.array_equal(F1[:n0], F1[n0:])
    o.set_state(g.get_state(0))
    o.ghost_fill()
    for n in range(o.nleaves):
        ref = M.features_from_padded(o.get_padded(n, 0), 1.5)
        assert np.allclose(F1[n], ref, rtol=2e-5, atol=1e-7), n


def test_forward_and_gradient_match_oracle():
    g, _ = make_pair(n=(24, 12, 12), nb=(12, 12, 12), **STR)
    rng = np.random.default_rng(0)
    theta = I.mlp_init(1).astype(np.float32)
    g.mlp_set_params(theta)
    X = rng.uniform(0, 0.3, (300, 64)).astype(np.float32)
    T = (rng.random(300) < 0.3).astype(np.float32)
    y = g.mlp_predict(X)
    yo, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y, yo, rtol=1e-5, atol=1e-6)
    gg, loss = g.mlp_grad(X, T)
    th, X64, T64 = theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    go = M.grad(th, X64, T64)
    # element by element: 1e-5 of the value, plus 1e-6 (about 16 FP32 ulps)
    # of the element's running-error magnitude, which covers the cancellation
    # FP32 cannot resolve (sums of mixed-sign terms in the forward
    # activations, in y - t and in the batch sums)
    mag = _grad_magnitudes(th, X64, T64)
    bound = 1e-5 * np.abs(go) + 1e-6 * mag
    bad = np.flatnonzero(np.abs(gg - go) > bound)
    assert bad.size == 0, (bad[:10], gg[bad[:10]], go[bad[:10]])
    assert abs(loss - M.loss(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))) < 1e-5


def test_adam_steps_match_oracle():
    g, _ = make_pair(n=(24, 12, 12), nb=(12, 12, 12), **STR)
    rng = np.random.default_rng(1)
    theta = I.mlp_init(2).astype(np.float32)
    g.mlp_set_params(theta)
    X = rng.uniform(0, 0.3, (64, 64)).astype(np.float32)
    T = (rng.random(64) < 0.5).astype(np.float32)
    g.mlp_dataset_clear()
    g.mlp_dataset_add(X, T)
    g.mlp_train(64, epochs=3, batch=64, lr=1e-3, seed=5)     # full batch: order does not matter
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for step in range(1, 4):
        th, m, v = M.adam_step(th, M.grad(th, X.astype(np.float64), T.astype(np.float64)), m, v, step)
    got = g.mlp_get_params()
    assert np.abs(got - th).max() < 1e-5


def test_training_separates_a_seeded_problem():
    g, _ = make_pair(n=(24, 12, 12), nb=(12, 12, 12), **STR)
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (4000, 64)).astype(np.float32)
    T = (X[:, :8].mean(1) > 0.5).astype(np.float32)
    g.mlp_set_params(I.mlp_init(3).astype(np.float32))
    g.mlp_dataset_clear()
    g.mlp_dataset_add(X, T)
    losses = g.mlp_train(3200, epochs=40, batch=256, lr=3e-3, seed=7)
    assert losses[-1] < 0.5 * losses[0]
    acc = ((g.mlp_predict(X[3200:]) > 0.5) == (T[3200:] > 0.5)).mean()
    assert acc > 0.9, acc


def test_learned_mode_flags_refinable_blocks_only():
    """flag_refine in the learned mode = the plain flags, set to +1 where the
    network's probability exceeds 1/2 on a block below its member's finest
    level (same kernels, so the decision is bit-exact)."""
    from paper_2211_12867_gb300.icarus import FLAG_LEARNED, FLAG_PLAIN
    g, o = make_pair(n=(48, 24, 48), nb=(12, 12, 12), max_level=3, max_blocks=4000, **STR)
    wind_setup(g, o)
    # records the background speed the criterion's gate needs; the CME itself
    # starts long after this test ends
    g.inject_cone_cme(0, t_start=100.0, **I.cme_config2(seed=0))
    g.step(10)
    crit = dict(e_refine=0.02, e_coarsen=0.005, eps=0.01, dv=-1e9)
    g.flag_refine(**crit, mode=FLAG_PLAIN)
    g.regrid()
    tree = g.tree(0)
    assert tree[:, 0].max() == 2, "the test wants refined leaves"
    # a network whose probabilities straddle 1/2 over these blocks
    th = I.mlp_init(4).astype(np.float32)
    g.mlp_set_params(th)
    p = g.mlp_predict_leaves()
    th[-1] -= np.float32(np.log(np.median(p) / (1 - np.median(p))))   # centre the output bias
    g.mlp_set_params(th)
    prob = g.mlp_predict_leaves()
    assert 0 < (prob > 0.5).sum() < len(prob)
    plain = g.flag_refine(**crit, mode=FLAG_PLAIN)
    for lmax in (3, 2):
        g.set_member_max_level(0, lmax)
        learned = g.flag_refine(**crit, mode=FLAG_LEARNED)
        want = np.where((prob > 0.5) & (tree[:, 0] < lmax), 1, plain)
        assert np.array_equal(learned, want), lmax
