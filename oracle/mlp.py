"""FP64 CPU oracle of the learned warm start and block-preconditioner
correction (test infrastructure; only tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use it).

The paper has no learned part; the method here is specified by its
interface: per camera i a small MLP maps features of the block-Jacobi block
M_i (the damped diagonal block of the reduced camera system, Sec. 5.4) and
of the right-hand side g_i to
  * a warm start  x0_i = (M_i^-1 g_i) * (1 + tanh(o_i))      (elementwise), and
  * a correction of the block preconditioner
        B_i = L_i^-T (I + E_i)(I + E_i)^T L_i^-1,   M_i = L_i L_i^T,
    with E_i lower triangular; diag(I + E_i) = 1 + 0.9 tanh(e_ii) > 0.1,
    so B_i is symmetric positive definite by construction and E_i = 0
    gives B_i = M_i^-1 (plain block Jacobi).

Features (19 per camera): log of the 9 diagonal entries of M_i, the
direction of the whitened right-hand side w_i = L_i^-1 g_i (w_i / |w_i|),
and log of the camera's observation count (at least 1).

Training loss per camera, with x*_i the camera block of a tight solve of the
reduced system and z*_i = L_i^T x*_i:
    ( |L^T x0 - z*|^2 + |F F^T w - z*|^2 ) / ( |z*|^2 + 1e-30 ),  F = I + E,
i.e. the M_i-norm errors |x0 - x*|_M^2 and |B g - x*|_M^2 (the second term
makes the corrected preconditioner map the first residual, g for a zero
start, to the true error), normalised per camera; the batch loss is the
mean.  The MLP is 19 -> 256 -> 256 -> 256 -> 54, GELU (exact, erf form)
after every hidden layer; outputs 0..8 are o, 9..53 the lower triangle of
E row by row.

Parity pinned against: finite differences of the loss, the closed forms
E = 0 => B = M^-1 and o = 0 => x0 = M^-1 g, positive definiteness of B, the
whitened loss against the direct M-norm form, and tabulated GELU values.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SIZES = (19, 256, 256, 256, 54)
N_OUT = 54
TRI = [(i, j) for i in range(9) for j in range(i + 1)]  # lower triangle, row by row


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(rng, sizes=SIZES):
    """He-style normal init for hidden layers, zeros for the output layer
    (so the untrained model is plain block Jacobi from M^-1 g)."""
    params = []
    for li in range(len(sizes) - 1):
        fan_in, fan_out = sizes[li], sizes[li + 1]
        if li == len(sizes) - 2:
            W = np.zeros((fan_out, fan_in))
        else:
            W = rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in)
        params.append((W, np.zeros(fan_out)))
    return params


def features(M, g, count):
    """M (n,9,9) SPD, g (n,9), count (n,) -> feats (n,19), L, w, s."""
    M = np.asarray(M, np.float64)
    g = np.asarray(g, np.float64)
    L = np.linalg.cholesky(M)
    w = np.linalg.solve(L, g[..., None])[..., 0]
    s = np.linalg.solve(M, g[..., None])[..., 0]
    nw = np.linalg.norm(w, axis=1, keepdims=True)
    wd = np.where(nw > 0, w / np.where(nw > 0, nw, 1.0), 0.0)
    cnt = np.maximum(np.asarray(count, np.float64), 1.0)  # a camera without observations counts as one
    f = np.concatenate([np.log(np.einsum("nii->ni", M)), wd, np.log(cnt)[:, None]], axis=1)
    return f, L, w, s


def forward(params, X):
    """Returns Y and the pre-activations of every layer."""
    h = np.asarray(X, np.float64)
    zs = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = gelu(z) if li < len(params) - 1 else z
    return h, zs


def _F(e):
    n = e.shape[0]
    F = np.zeros((n, 9, 9))
    for t, (i, j) in enumerate(TRI):
        if i == j:
            F[:, i, i] = 1.0 + 0.9 * np.tanh(e[:, t])
        else:
            F[:, i, j] = e[:, t]
    return F


def head_apply(Y, L, s):
    """Inference head: x0 (n,9) and B (n,9,9)."""
    o, e = Y[:, :9], Y[:, 9:N_OUT]
    x0 = s * (1.0 + np.tanh(o))
    F = _F(e)
    Li = np.linalg.inv(L)
    B = np.einsum("nki,nkl,njl,njm->nim", Li, F, F, Li)
    return x0, B


def head_loss(Y, L, w, s, zs):
    """Per-camera normalised loss and its gradient with respect to Y."""
    n = Y.shape[0]
    o, e = Y[:, :9], Y[:, 9:N_OUT]
    th = np.tanh(o)
    x0 = s * (1.0 + th)
    den = np.einsum("ni,ni->n", zs, zs) + 1e-30
    R1 = np.einsum("nki,nk->ni", L, x0) - zs          # L^T x0 - z*
    F = _F(e)
    u = np.einsum("nki,nk->ni", F, w)                  # F^T w
    v = np.einsum("nij,nj->ni", F, u)                  # F F^T w
    R2 = v - zs
    loss = (np.einsum("ni,ni->n", R1, R1) + np.einsum("ni,ni->n", R2, R2)) / den
    dY = np.zeros((n, Y.shape[1]))
    # term 1: d/dx0 = 2 L R1 / den, x0 = s (1 + tanh o)
    gx = 2.0 * np.einsum("nik,nk->ni", L, R1) / den[:, None]
    dY[:, :9] = gx * s * (1.0 - th * th)
    # term 2: dF_ij = 2 (R2_i u_j + w_i q_j) / den, q = F^T R2
    q = np.einsum("nki,nk->ni", F, R2)
    dF = 2.0 * (R2[:, :, None] * u[:, None, :] + w[:, :, None] * q[:, None, :]) / den[:, None, None]
    for t, (i, j) in enumerate(TRI):
        if i == j:
            te = np.tanh(e[:, t])
            dY[:, 9 + t] = dF[:, i, i] * 0.9 * (1.0 - te * te)
        else:
            dY[:, 9 + t] = dF[:, i, j]
    return loss, dY


def head_loss_direct(Y, M, g, xstar):
    """The same loss written with M-norms in the original coordinates (a
    second, independent form used to pin head_loss)."""
    L = np.linalg.cholesky(M)
    s = np.linalg.solve(M, g[..., None])[..., 0]
    x0, B = head_apply(Y, L, s)
    d1 = x0 - xstar
    d2 = np.einsum("nij,nj->ni", B, g) - xstar
    den = np.einsum("ni,nij,nj->n", xstar, M, xstar) + 1e-30
    return (np.einsum("ni,nij,nj->n", d1, M, d1) + np.einsum("ni,nij,nj->n", d2, M, d2)) / den


def loss_and_grads(params, X, L, w, s, zs):
    """Mean loss over the batch and the gradients of every (W, b)."""
    Y, zl = forward(params, X)
    loss, dY = head_loss(Y, L, w, s, zs)
    n = X.shape[0]
    dz = dY / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h_in = np.asarray(X, np.float64) if li == 0 else gelu(zl[li - 1])
        grads[li] = (dz.T @ h_in, dz.sum(axis=0))
        if li > 0:
            dz = (dz @ params[li][0]) * gelu_grad(zl[li - 1])
    return float(loss.mean()), grads


def training_sample(M, g, xstar, count):
    """Per-camera training tuple from a solve: features and the head inputs."""
    f, L, w, s = features(M, g, count)
    zs = np.einsum("nki,nk->ni", L, np.asarray(xstar, np.float64))
    return f, L, w, s, zs
