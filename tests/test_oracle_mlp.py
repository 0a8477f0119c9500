"""Pins of the FP64 oracle of the learned warm start / preconditioner
correction (oracle/mlp.py) against values fixed by the mathematics:
tabulated GELU values, closed forms of the head, positive definiteness,
an independent direct M-norm form of the loss, and central finite
differences of the loss and of the full MLP gradient."""
import math

import numpy as np

from oracle import mlp


def _spd(rng, n):
    A = rng.standard_normal((n, 9, 9))
    D = np.exp(rng.uniform(-3, 6, size=(n, 9)))  # widely different scales, like camera parameters
    M = np.einsum("nij,nkj->nik", A, A) + np.einsum("ni,ij->nij", D, np.eye(9))
    return M


def test_gelu_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208
    np.testing.assert_allclose(mlp.gelu(np.array([0.0, 1.0, -1.0, 2.0])),
                               [0.0, 0.8413447460685429, -0.15865525393145707, 1.9544997361036416], rtol=1e-14)
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5


def test_head_closed_forms():
    rng = np.random.default_rng(0)
    M = _spd(rng, 5)
    g = rng.standard_normal((5, 9))
    f, L, w, s = mlp.features(M, g, np.arange(1, 6))
    x0, B = mlp.head_apply(np.zeros((5, 54)), L, s)
    np.testing.assert_allclose(x0, np.linalg.solve(M, g[..., None])[..., 0], rtol=1e-12)
    np.testing.assert_allclose(B, np.linalg.inv(M), rtol=1e-9, atol=1e-12 * np.abs(np.linalg.inv(M)).max())
    # features: log diag, unit whitened direction, log count
    np.testing.assert_allclose(f[:, :9], np.log(np.einsum("nii->ni", M)))
    np.testing.assert_allclose(np.linalg.norm(f[:, 9:18], axis=1), 1.0)
    np.testing.assert_allclose(f[:, 18], np.log(np.arange(1, 6)))
    f0, _, _, _ = mlp.features(M[:1], g[:1], [0])
    assert f0[0, 18] == 0.0  # a camera without observations counts as one
    np.testing.assert_allclose(np.einsum("nij,nj->ni", L, w), g, rtol=1e-10)


def test_corrected_preconditioner_is_spd():
    rng = np.random.default_rng(1)
    M = _spd(rng, 8)
    g = rng.standard_normal((8, 9))
    _, L, _, s = mlp.features(M, g, np.ones(8))
    Y = rng.standard_normal((8, 54))  # far from the untrained model
    _, B = mlp.head_apply(Y, L, s)
    np.testing.assert_allclose(B, np.transpose(B, (0, 2, 1)), rtol=1e-10, atol=1e-12 * np.abs(B).max())
    assert np.all(np.linalg.eigvalsh(B) > 0)
    np.linalg.cholesky(B)
    # however large the raw outputs, diag(I + E) stays above 0.1 (F invertible)
    F = mlp._F(rng.standard_normal((8, 45)) * 100.0)
    assert np.all(np.einsum("nii->ni", F) > 0.1 - 1e-12)


def test_whitened_loss_equals_direct_m_norms():
    rng = np.random.default_rng(2)
    M = _spd(rng, 6)
    g = rng.standard_normal((6, 9))
    xs = rng.standard_normal((6, 9))
    Y = rng.standard_normal((6, 54))
    f, L, w, s, zs = mlp.training_sample(M, g, xs, np.ones(6))
    loss, _ = mlp.head_loss(Y, L, w, s, zs)
    np.testing.assert_allclose(loss, mlp.head_loss_direct(Y, M, g, xs), rtol=1e-9)


def test_head_gradient_finite_differences():
    rng = np.random.default_rng(3)
    M = _spd(rng, 3)
    g = rng.standard_normal((3, 9))
    xs = rng.standard_normal((3, 9))
    Y = rng.standard_normal((3, 54)) * 0.5
    _, L, w, s, zs = mlp.training_sample(M, g, xs, np.ones(3))
    _, dY = mlp.head_loss(Y, L, w, s, zs)
    h = 1e-6
    for c in range(54):
        Yp, Ym = Y.copy(), Y.copy()
        Yp[:, c] += h
        Ym[:, c] -= h
        fd = (mlp.head_loss(Yp, L, w, s, zs)[0] - mlp.head_loss(Ym, L, w, s, zs)[0]) / (2 * h)
        np.testing.assert_allclose(dY[:, c], fd, rtol=1e-5, atol=1e-7)


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(4)
    sizes = (19, 8, 8, 8, 54)
    params = [(rng.standard_normal((o, i)) * 0.3, rng.standard_normal(o) * 0.1)
              for i, o in zip(sizes[:-1], sizes[1:])]
    M = _spd(rng, 4)
    g = rng.standard_normal((4, 9))
    xs = rng.standard_normal((4, 9))
    X, L, w, s, zs = mlp.training_sample(M, g, xs, np.arange(2, 6))
    loss, grads = mlp.loss_and_grads(params, X, L, w, s, zs)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (r, c) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, 3)]:
            Wp = [(x.copy(), y.copy()) for x, y in params]
            Wm = [(x.copy(), y.copy()) for x, y in params]
            Wp[li][0][r, c] += h
            Wm[li][0][r, c] -= h
            fd = (mlp.loss_and_grads(Wp, X, L, w, s, zs)[0] - mlp.loss_and_grads(Wm, X, L, w, s, zs)[0]) / (2 * h)
            assert math.isclose(grads[li][0][r, c], fd, rel_tol=1e-5, abs_tol=1e-8), (li, r, c)
        Bp = [(x.copy(), y.copy()) for x, y in params]
        Bm = [(x.copy(), y.copy()) for x, y in params]
        Bp[li][1][1] += h
        Bm[li][1][1] -= h
        fd = (mlp.loss_and_grads(Bp, X, L, w, s, zs)[0] - mlp.loss_and_grads(Bm, X, L, w, s, zs)[0]) / (2 * h)
        assert math.isclose(grads[li][1][1], fd, rel_tol=1e-5, abs_tol=1e-8), li


def test_untrained_model_is_block_jacobi():
    rng = np.random.default_rng(5)
    params = mlp.init_params(rng)
    M = _spd(rng, 4)
    g = rng.standard_normal((4, 9))
    X, L, w, s = mlp.features(M, g, np.ones(4))
    Y, _ = mlp.forward(params, X)
    assert np.all(Y == 0.0)
    x0, B = mlp.head_apply(Y, L, s)
    np.testing.assert_allclose(x0, s)
