"""NumPy FP64 oracle of the learned refinement pre-flagger.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; the predictor follows the workload's
recipe: per block, the index-space gradient magnitude of density, radial
speed and pressure, each divided by the cell's own magnitude, averaged over
the three variables and over 4 x 4 x 4 sub-cubes of the block -> 64 inputs;
an MLP 64 -> 128 (ReLU) -> 128 (ReLU) -> 1 (sigmoid); binary cross-entropy;
Adam.  Written plainly: full matrices, natural order, no fusion.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 64, 128


def features_from_padded(P, gamma):
    """P: padded conserved block [8][n0+4][n1+4][n2+4] (2 ghost layers).
    Returns the 64 features (sub-cube means, sub-cube index (a, b, c) in
    row-major order with a along r)."""
    rho = P[0]
    vr = P[1] / P[0]
    ke = 0.5 * (P[1] ** 2 + P[2] ** 2 + P[3] ** 2) / P[0]
    me = 0.5 * (P[5] ** 2 + P[6] ** 2 + P[7] ** 2)
    p = (gamma - 1.0) * (P[4] - ke - me)
    n = [s - 4 for s in P.shape[1:]]
    inner = (slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2]))
    g = np.zeros(n)
    for u in (rho, vr, p):
        gsq = np.zeros(n)
        for d in range(3):
            up = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
            um = list(up)
            up[d] = slice(3, 3 + n[d])
            um[d] = slice(1, 1 + n[d])
            c = 0.5 * (u[tuple(up)] - u[tuple(um)])
            gsq += c * c
        g += np.sqrt(gsq) / (np.abs(u[inner]) + 1e-30)
    g /= 3.0
    s = [k // 4 for k in n]
    out = np.zeros(64)
    for a in range(4):
        for b in range(4):
            for c in range(4):
                out[(a * 4 + b) * 4 + c] = g[a * s[0]:(a + 1) * s[0], b * s[1]:(b + 1) * s[1],
                                             c * s[2]:(c + 1) * s[2]].mean()
    return out


def unpack(theta):
    """flat parameter vector -> (W1[128,64], b1[128], W2[128,128], b2[128], w3[128], b3)"""
    o = 0
    W1 = theta[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = theta[o:o + N_H]; o += N_H
    W2 = theta[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = theta[o:o + N_H]; o += N_H
    w3 = theta[o:o + N_H]; o += N_H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1


def forward(theta, X):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    y = 1.0 / (1.0 + np.exp(-z))
    return y, (X, a1, h1, a2, h2, z)


def loss(theta, X, t):
    y, _ = forward(theta, X)
    y = np.clip(y, 1e-12, 1 - 1e-12)
    return float(np.mean(-(t * np.log(y) + (1 - t) * np.log(1 - y))))


def grad(theta, X, t):
    """gradient of the mean binary cross-entropy with respect to theta"""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    y, (X, a1, h1, a2, h2, z) = forward(theta, X)
    B = X.shape[0]
    dz = (y - t) / B
    gw3 = h2.T @ dz
    gb3 = dz.sum()
    dh2 = np.outer(dz, w3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def adam_step(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
