"""The identity the Gram-form block-Jacobi preconditioner rests on, checked
with numpy on random landmark blocks (no oracle, no GPU).

For a landmark block [J_p | J_l | r] with the damping rows [0 | sqrt(lambda) D_l | 0]
appended (Sec. 5.3), an orthogonal Q with Q^T [J_l; sqrt(lambda) D_l] = [R1; 0]
splits the pose and residual columns into the top rows [T | t] and the rest
[A | c].  Q is orthogonal, so the Gram matrix of those columns is unchanged:
    J_p^T J_p = T^T T + A^T A,     J_p^T r = T^T t + A^T c,
and per observation s (its 9 pose columns) the diagonal block of the reduced
camera system is (A^T A)_ss = J_s^T J_s - T_s^T T_s with J_s the observation's
two Jacobian rows (Eq. red_H / red_b)."""
import numpy as np
import pytest


def _block(rng, k, lam):
    jp = np.zeros((2 * k, 9 * k))
    for s in range(k):
        jp[2 * s:2 * s + 2, 9 * s:9 * s + 9] = rng.normal(size=(2, 9))
    jl = rng.normal(size=(2 * k, 3))
    r = rng.normal(size=2 * k)
    d = np.sqrt(np.sum(jl * jl, axis=0))
    big = np.zeros((2 * k + 3, 9 * k + 4))
    big[:2 * k, :9 * k] = jp
    big[:2 * k, 9 * k:9 * k + 3] = jl
    big[:2 * k, -1] = r
    big[2 * k:, 9 * k:9 * k + 3] = np.sqrt(lam) * np.diag(d)
    return jp, jl, r, d, big


@pytest.mark.parametrize("k,lam", [(2, 1e-4), (3, 1.0), (7, 1e-2), (20, 1e2)])
def test_gram_identity_per_observation(k, lam):
    rng = np.random.default_rng(k)
    jp, jl, r, d, big = _block(rng, k, lam)
    q, _ = np.linalg.qr(big[:, 9 * k:9 * k + 3], mode="complete")
    rot = q.T @ big
    assert np.allclose(rot[3:, 9 * k:9 * k + 3], 0.0, atol=1e-10)  # landmark columns eliminated
    top, rest = rot[:3], rot[3:]
    T, t = top[:, :9 * k], top[:, -1]
    A, c = rest[:, :9 * k], rest[:, -1]
    # reduced system from the explicit damped Schur complement
    H_ll = jl.T @ jl + lam * np.diag(d * d)
    S = jp.T @ jp - jp.T @ jl @ np.linalg.solve(H_ll, jl.T @ jp)
    b = jp.T @ r - jp.T @ jl @ np.linalg.solve(H_ll, jl.T @ r)
    np.testing.assert_allclose(A.T @ A, S, atol=1e-9 * np.abs(S).max())
    np.testing.assert_allclose(A.T @ c, b, atol=1e-9 * np.abs(b).max())
    for s in range(k):
        cols = slice(9 * s, 9 * s + 9)
        js = jp[2 * s:2 * s + 2, cols]
        gram = js.T @ js - T[:, cols].T @ T[:, cols]
        rhs = js.T @ r[2 * s:2 * s + 2] - T[:, cols].T @ t
        np.testing.assert_allclose(gram, (A.T @ A)[cols, cols], atol=1e-9 * np.abs(js.T @ js).max())
        np.testing.assert_allclose(rhs, (A.T @ c)[cols], atol=1e-9 * np.abs(js.T @ r[2 * s:2 * s + 2]).max())


def test_gram_identity_fails_for_a_wrong_top_row():
    """A plausible mistake (one top row dropped) breaks the identity."""
    rng = np.random.default_rng(5)
    k, lam = 4, 1e-2
    jp, jl, r, d, big = _block(rng, k, lam)
    q, _ = np.linalg.qr(big[:, 9 * k:9 * k + 3], mode="complete")
    rot = q.T @ big
    T, A = rot[:2, :9 * k], rot[3:, :9 * k]  # row 2 of the top rows left out
    js = jp[0:2, 0:9]
    assert not np.allclose(js.T @ js - T[:, 0:9].T @ T[:, 0:9], (A.T @ A)[0:9, 0:9], atol=1e-6)
