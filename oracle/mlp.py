"""FP64 oracle of the learned troubled-cell indicator (test infrastructure).

The paper frames troubled-cell detection as its own step, judged by
sensitivity and specificity (Sec. 4.2: detection, then limiting). This
indicator replaces the TVB detection with a small multilayer perceptron that
decides which cells the TVB procedure processes; the plain TVB trigger gives
the labels and is the reference it is scored against. Nothing here is printed
in the paper; the choices are:

* features of a cell (8 n(d) + 2D + 8D values): the Legendre coefficients of
  the 8 MHD conserved variables (for the LDF basis, B is first mapped exactly
  to per-component Legendre coefficients), each variable divided by
  s_v = |mean_v| + max over the 2D face neighbours |mean_nb,v - mean_v| + 1e-12,
  then the neighbour density ratios rho_nb/rho - 1 in the order
  -x, +x, -y, +y, -z, +z, then for each direction a and variable v the
  degree-1 coefficient along a divided by M~ dx (the TVB slope scale); on an
  octree the neighbour mean of a side is the average of the leaves across it
  and dx the leaf's own size;
* network: in -> 64 -> 64 -> 1, ReLU hidden layers, sigmoid output;
* loss: mean binary cross-entropy; optimiser: Adam.
Weights are one flat vector: W1[64][in], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
from __future__ import annotations

from fractions import Fraction
import numpy as np

from . import basis as B
from . import mhd

H = 64


def n_in(S):
    return 8 * S.n + 2 * S.D + 8 * S.D


def n_params(nin):
    return H * nin + H + H * H + H + H + 1


def unpack(theta, nin):
    i = 0
    W1 = theta[i:i + H * nin].reshape(H, nin); i += H * nin
    b1 = theta[i:i + H]; i += H
    W2 = theta[i:i + H * H].reshape(H, H); i += H * H
    b2 = theta[i:i + H]; i += H
    w3 = theta[i:i + H]; i += H
    b3 = theta[i]
    return W1, b1, W2, b2, w3, b3


def init_params(nin, seed=0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / nin), (H, nin))
    W2 = rng.normal(0, np.sqrt(2.0 / H), (H, H))
    w3 = rng.normal(0, np.sqrt(1.0 / H), H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])


def ldf_to_legendre(S):
    """T[j, c, l] = <phi_j,c, P_l> / <P_l, P_l>: exact componentwise Legendre
    coefficients of each LDF basis vector (degree <= d)."""
    T = np.zeros((len(S.ldf), S.D, S.n))
    for j, vec in enumerate(S.ldf):
        for c, comp in enumerate(vec):
            if not comp:
                continue
            for l, k in enumerate(S.modes):
                T[j, c, l] = float(B.pintegrate(B.pmul(comp, S.legendre[l])) / B.legendre_mass(k))
    return T


def coefficients(S, w):
    """a[cell, v, l]: Legendre coefficients of the 8 MHD variables."""
    a = np.zeros((S.C, 8, S.n))
    for r, (kind, v, i) in enumerate(S.rows):
        if kind == "L" and v < 8:
            a[:, v, i] = w[:, r]
    if S.divb == "powell":
        T = ldf_to_legendre(S)
        ldf0 = 5 * S.n
        wl = w[:, ldf0:ldf0 + len(S.ldf)]
        for c in range(S.D):
            a[:, mhd.BX + c, :] = wl @ T[:, c, :]
    return a


def side_means(S, m):
    """Neighbour means per cell, axis and side (0: -axis, 1: +axis). Uniform
    mesh: the face neighbour; octree: the average of the leaves across the
    side (one of the same level or coarser, or the finer ones), the neighbour
    mean the octree TVB procedure uses (limiter.mean_differences)."""
    if not hasattr(S, "faces"):
        return np.stack([np.stack([m[S.nbr_minus[ax]], m[S.nbr_plus[ax]]], 1) for ax in range(S.D)], 1)
    acc = np.zeros((S.C, S.D, 2, m.shape[1]))
    cnt = np.zeros((S.C, S.D, 2))
    for cL, cR, ax, kind, sub in S.faces:
        acc[cR, ax, 0] += m[cL]     # cR sees cL on its -axis side
        cnt[cR, ax, 0] += 1
        acc[cL, ax, 1] += m[cR]
        cnt[cL, ax, 1] += 1
    return acc / cnt[..., None]


def features(S, w):
    a = coefficients(S, w)
    m = S.means(w)[:, :8]
    nb = side_means(S, m)
    dmax = np.zeros_like(m)
    ratios = []
    for ax in range(S.D):
        for side in (0, 1):
            dmax = np.maximum(dmax, np.abs(nb[:, ax, side] - m))
            ratios.append(nb[:, ax, side, 0] / m[:, 0] - 1.0)
    s = np.abs(m) + dmax + 1e-12
    X = (a / s[:, :, None]).reshape(S.C, -1)
    deg1 = [S.modes.index(tuple(1 if i == ax else 0 for i in range(S.D))) for ax in range(S.D)]
    dx = S.dxc[:, None] if hasattr(S, "faces") else S.dx
    sl = np.concatenate([a[:, :, deg1[ax]] for ax in range(S.D)], -1) / (S.P.Mtilde * dx)
    return np.concatenate([X, np.stack(ratios, -1), sl], -1)


def forward(theta, X):
    nin = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(theta, nin)
    Z1 = X @ W1.T + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2.T + b2
    A2 = np.maximum(Z2, 0.0)
    z3 = A2 @ w3 + b3
    return z3, (Z1, A1, Z2, A2)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def loss_and_grad(theta, X, y, pos_weight=1.0):
    """Mean weighted BCE loss -(pw y log p + (1 - y) log(1 - p)) and its
    gradient w.r.t. theta (backpropagation)."""
    nin = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(theta, nin)
    z3, (Z1, A1, Z2, A2) = forward(theta, X)
    p = sigmoid(z3)
    eps = 1e-12
    loss = -np.mean(pos_weight * y * np.log(p + eps) + (1 - y) * np.log(1 - p + eps))
    n = len(y)
    d3 = (pos_weight * y * (p - 1) + (1 - y) * p) / n
    gw3 = A2.T @ d3
    gb3 = d3.sum()
    d2 = np.outer(d3, w3) * (Z2 > 0)
    gW2 = d2.T @ A1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (Z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
