"""Parity at the full sizes of the medium and large workloads, in the launch
configuration bench.py times (autotuned matvec plan), on outputs the FP64
oracle can compute one by one:

  * sampled landmark blocks: A_j^T A_j and A_j^T c_j against the landmark's
    damped Schur-complement pieces (Eq. red_H / red_b), R1^T R1 against
    H_ll + lambda D_l^2, ||c_j||^2 (the heaviest and lightest landmarks are
    always among the samples);
  * medium: the whole block diagonal of H~ and g (K3) and two matvecs (K4)
    against the oracle's assembled reduced camera system;
  * large: matvec rows of sampled cameras, assembled from the oracle's
    per-landmark Schur complements of every landmark the camera sees, and
    the device memory footprint (blocks of 72 sum k^2 bytes, total within
    1.6x of it).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.synth import make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_01843_gb300 as pkg
    pkg.lib()
    return pkg


def Rounded(s):
    return dataclasses.replace(s, cams=s.cams.astype(np.float32).astype(np.float64),
                               pts=s.pts.astype(np.float32).astype(np.float64))


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


class _Groups:
    """Observation rows of every landmark (for one-landmark sub-problems)."""

    def __init__(self, s):
        self.order = np.argsort(s.obs_pt, kind="stable")
        self.off = np.searchsorted(s.obs_pt[self.order], np.arange(s.n_pt + 1))

    def sub(self, s, j):
        rows = self.order[self.off[j]:self.off[j + 1]]
        return dataclasses.replace(s, pts=s.pts[j:j + 1], obs_cam=s.obs_cam[rows],
                                   obs_pt=np.zeros(rows.size, s.obs_pt.dtype), obs_xy=s.obs_xy[rows])


def _landmark_sc(s, groups, lam, j):
    # the landmark's damped Schur-complement pieces depend only on its own
    # observations, the cameras and its point: the oracle works on that
    # one-landmark sub-problem
    return oracle.landmark_sc(groups.sub(s, j), lam, 0)


def _check_landmark(s, groups, blk, lam, j, tol):
    k = blk["k"]
    A, c, top = blk["a"].astype(np.float64), blk["c"].astype(np.float64), blk["top"].astype(np.float64)
    S, bts, Hll, cc = _landmark_sc(s, groups, lam, j)
    assert S.shape == (9 * k, 9 * k)
    assert rel_fro(A.T @ A, S) < tol, (j, k, rel_fro(A.T @ A, S))
    assert np.linalg.norm(A.T @ c - bts) <= tol * (np.linalg.norm(A) * np.linalg.norm(c) + np.linalg.norm(bts))
    R = top[:, 9 * k:9 * k + 3]
    assert rel_fro(R.T @ R, Hll) < 1e-5
    rr = cc + top[:, -1] @ top[:, -1]
    assert abs(c @ c - cc) <= 1e-5 * rr + 1e-4 * cc


def _samples(s, n, seed):
    k = s.k_per_point()
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(s.n_pt, n, replace=False).tolist())
    pick |= set(np.argsort(k)[-4:].tolist()) | set(np.nonzero(k == k.min())[0][:2].tolist())
    return sorted(pick)


@pytest.fixture(scope="module")
def medium():
    return make_scene("medium", 0)


def test_medium_full_size(pkg, medium):
    s = Rounded(medium)
    lam = 1e-4
    with pkg.Problem.from_scene(medium, autotune=1) as p:
        p.linearize()
        p.marginalize_qr(lam)
        p.autotune()  # the plan bench.py times
        groups = _Groups(s)
        for j in _samples(medium, 30, 0):
            _check_landmark(s, groups, p.export_landmark(j, k_cap=64), lam, j, tol=1e-4)
        p.pcg_solve()
        M, g = p.export_rcs_diag()
        V = np.random.default_rng(3).normal(size=(2, 9 * s.n_cam)).astype(np.float32)
        Y = np.stack([p.matvec(v) for v in V])
    Mref, bt = oracle.rcs_diag(s, lam)
    assert rel_fro(M, Mref) < 1e-4, rel_fro(M, Mref)
    assert rel_fro(g, -bt) < 1e-4, rel_fro(g, -bt)
    assert rel_fro(Y, oracle.rcs_matvec(s, lam, V)) < 1e-4


def test_large_full_size(pkg):
    sc = make_scene("large", 0)
    s = Rounded(sc)
    lam = 1e-3
    k = sc.k_per_point()
    with pkg.Problem.from_scene(sc, autotune=1) as p:
        info = p.info()
        blocks = 4 * info["a_pool_floats"]
        assert blocks >= 72 * info["sum_k2"]
        assert info["device_bytes"] <= 1.6 * blocks, (info["device_bytes"], blocks)
        p.linearize()
        p.marginalize_qr(lam)
        p.autotune()
        groups = _Groups(s)
        for j in _samples(sc, 12, 1):
            _check_landmark(s, groups, p.export_landmark(j, k_cap=256), lam, j, tol=2e-4)
        v = np.random.default_rng(4).normal(size=9 * s.n_cam).astype(np.float32)
        y = p.matvec(v)
        dp2, _ = p.export_damping()
    # rows of two cameras: sum of the damped per-landmark Schur complements
    # (Eq. red_H) of every landmark the camera sees, plus lambda D_p^2 v
    rng = np.random.default_rng(5)
    v64 = v.astype(np.float64)
    for cam in rng.choice(s.n_cam, 2, replace=False):
        ref = np.zeros(9)
        for j in np.unique(s.obs_pt[s.obs_cam == cam]):
            S, _, _, _ = _landmark_sc(s, groups, lam, int(j))
            cams_j = np.sort(groups.sub(s, int(j)).obs_cam)
            slot = int(np.nonzero(cams_j == cam)[0][0])
            vj = np.concatenate([v64[9 * c:9 * c + 9] for c in cams_j])
            ref += (S @ vj)[9 * slot:9 * slot + 9]
        ref += lam * dp2[cam].astype(np.float64) * v64[9 * cam:9 * cam + 9]
        got = y[9 * cam:9 * cam + 9].astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), (cam, got, ref)
    assert k.max() == 200
