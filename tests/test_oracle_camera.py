"""Pins of the oracle's camera model (Sec. 6.2, BAL Snavely camera).

Each check compares the oracle with something other than itself: scipy's
rotation routines, a hand-computed worked example, the scene generator's
independent matrix-form projection, and finite differences.
"""
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2103_01843_gb300.synth import make_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "camera_worked_example.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, *nums = line.split()
        vals[key] = np.array([float(x) for x in nums])
    return vals


def test_worked_example_residual_and_derivatives():
    g = _golden()
    r, Jp, Jl = oracle.residual(g["cam"], g["point"], g["obs"])
    np.testing.assert_allclose(r, g["residual"], rtol=1e-12)
    np.testing.assert_allclose(Jp[:, 6], g["d_f"], rtol=1e-12)
    np.testing.assert_allclose(Jp[:, 7], g["d_k1"], rtol=1e-12)
    np.testing.assert_allclose(Jp[:, 8], g["d_k2"], rtol=1e-12)
    np.testing.assert_allclose(Jp[0, 3], g["d_tx_row0"][0], rtol=1e-12)
    # with R = I the landmark Jacobian equals d pixel / d P = the translation block
    np.testing.assert_allclose(Jl, Jp[:, 3:6], rtol=1e-14)


@pytest.mark.parametrize("scale", [0.0, 1e-12, 1e-9, 1e-5, 0.3, 2.0, 3.1])
def test_rodrigues_matches_scipy(scale):
    rng = np.random.default_rng(1)
    for _ in range(20):
        w = rng.normal(size=3)
        w = scale * w / np.linalg.norm(w)
        np.testing.assert_allclose(oracle.rotmat(w), Rotation.from_rotvec(w).as_matrix(),
                                   atol=1e-14)


def test_compose_matches_scipy_product():
    rng = np.random.default_rng(2)
    for _ in range(50):
        w = rng.normal(size=3) * rng.uniform(0, 3.0)
        dw = rng.normal(size=3) * rng.uniform(0, 0.5)
        out = oracle.compose(dw, w)
        ref = (Rotation.from_rotvec(dw) * Rotation.from_rotvec(w)).as_matrix()
        np.testing.assert_allclose(oracle.rotmat(out), ref, atol=1e-12)
        assert np.linalg.norm(out) <= np.pi + 1e-12


def test_noise_free_ground_truth_has_zero_cost():
    # the generator projects with rotation matrices built by look-at; the
    # oracle projects from axis-angle with Rodrigues: two independent codes
    s = make_scene("tiny", 0, noise_px=0.0, perturb=False)
    assert oracle.cost(s) < 1e-16 * s.n_obs
    s = make_scene("tiny", 3, noise_px=0.0)
    assert oracle.cost(s, s.cams_gt, s.pts_gt) < 1e-16 * s.n_obs


def test_noisy_ground_truth_cost_is_chi_square():
    s = make_scene("tiny", 0, noise_px=1.0)
    e = oracle.cost(s, s.cams_gt, s.pts_gt)
    n = 2 * s.n_obs  # sum of 2 n_obs squared N(0, 1) draws
    assert abs(e - n) < 5 * np.sqrt(2 * n)


def _fd_jacobians(cam, X, z, h_rel=1e-6):
    Jp = np.zeros((2, 9))
    for c in range(9):
        h = h_rel * max(1.0, abs(cam[c])) if c >= 3 else 1e-6
        cp, cm = cam.copy(), cam.copy()
        if c < 3:  # left-multiplicative rotation increment
            e = np.zeros(3)
            e[c] = h
            cp[:3] = oracle.compose(e, cam[:3])
            cm[:3] = oracle.compose(-e, cam[:3])
        else:
            cp[c] += h
            cm[c] -= h
        Jp[:, c] = (oracle.residual(cp, X, z)[0] - oracle.residual(cm, X, z)[0]) / (2 * h)
    Jl = np.zeros((2, 3))
    for c in range(3):
        h = h_rel * max(1.0, abs(X[c]))
        Xp, Xm = X.copy(), X.copy()
        Xp[c] += h
        Xm[c] -= h
        Jl[:, c] = (oracle.residual(cam, Xp, z)[0] - oracle.residual(cam, Xm, z)[0]) / (2 * h)
    return Jp, Jl


def test_analytic_jacobians_match_central_differences(tiny_scene):
    s = tiny_scene
    rng = np.random.default_rng(5)
    for o in rng.choice(s.n_obs, 40, replace=False):
        cam, X, z = s.cams[s.obs_cam[o]], s.pts[s.obs_pt[o]], s.obs_xy[o]
        _, Jp, Jl = oracle.residual(cam, X, z)
        Fp, Fl = _fd_jacobians(cam, X, z)
        for A, F in ((Jp, Fp), (Jl, Fl)):
            err = np.abs(A - F) / np.maximum(np.abs(F).max(), 1e-12)
            assert err.max() < 1e-6, (o, err.max())


def test_update_is_left_multiplicative_and_additive():
    rng = np.random.default_rng(6)
    cams = rng.normal(size=(3, 9))
    pts = rng.normal(size=(4, 3))
    dc = rng.normal(size=(3, 9)) * 0.1
    dp = rng.normal(size=(4, 3))
    co, po = oracle.apply_update(cams, dc, pts, dp)
    np.testing.assert_allclose(po, pts + dp, rtol=0, atol=1e-15)
    np.testing.assert_allclose(co[:, 3:], cams[:, 3:] + dc[:, 3:], atol=1e-15)
    for i in range(3):
        ref = Rotation.from_rotvec(dc[i, :3]) * Rotation.from_rotvec(cams[i, :3])
        np.testing.assert_allclose(oracle.rotmat(co[i, :3]), ref.as_matrix(), atol=1e-12)
