"""Seeded synthetic bundle-adjustment scenes (input generation only).

This module builds problem instances for both the CUDA path and the FP64
oracle.  It holds none of the solver's arithmetic: no residual, Jacobian,
QR, damping, conjugate-gradient or Levenberg-Marquardt step.  To synthesise
pixel observations it needs a forward camera model; it uses its own
matrix formulation (rotation matrices built by look-at / yaw construction)
of the 9-parameter BAL "Snavely" camera (Sec. 6.2 of the paper: one focal
length, two radial distortion parameters), so the solver sides never share
code with it.  Axis-angle conversion goes through scipy.

Recipe (the paper's preprocessing, Sec. 6.2, applied to synthetic data):
  1. ground truth in metres (cameras, points), per-config geometry below;
  2. observations = projection of ground truth + N(0, sigma_px^2) pixel noise;
     a camera observes a point only if the point is in front of it (depth >
     0.5 m), projects inside the 1000 x 1000 px image (|u|, |v| < 500) and
     lies inside the field of view (|P_x / P_z|, |P_y / P_z| < 1.2);
  3. initial state = ground truth perturbed (rotation Exp(N(0, 0.01^2 I)) R,
     translation + N(0, 0.05^2), points + N(0, 0.1^2)); observations whose
     point has depth < 1 m or |P_xy / P_z| >= 1.5 in the perturbed state are
     removed, then landmarks with fewer than two observations (Sec. 6.2);
  4. gauge normalisation of the initial state: points centred at their
     per-axis median and scaled so that the median L1 deviation is 100;
     cameras transformed consistently (pixels are unchanged by this
     similarity transform).  Ground truth is mapped by the same transform.

BAL conventions: camera = [axis-angle (3), t (3), f, k1, k2]; P = R X + t;
points in front have P_z < 0; p = -P_xy / P_z; pixel = f (1 + k1|p|^2 +
k2|p|^4) p.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial.transform import Rotation

IMAGE_HALF = 500.0  # image is 2*500 x 2*500 px, principal point at 0


@dataclasses.dataclass
class Scene:
    cams: np.ndarray      # (n_cam, 9) float64 initial state, BAL order
    pts: np.ndarray       # (n_pt, 3) float64 initial state
    obs_cam: np.ndarray   # (n_obs,) int32
    obs_pt: np.ndarray    # (n_obs,) int32
    obs_xy: np.ndarray    # (n_obs, 2) float64 pixels
    cams_gt: np.ndarray   # ground truth in the normalised gauge
    pts_gt: np.ndarray
    name: str = ""
    seed: int = 0

    @property
    def n_cam(self):
        return int(self.cams.shape[0])

    @property
    def n_pt(self):
        return int(self.pts.shape[0])

    @property
    def n_obs(self):
        return int(self.obs_cam.shape[0])

    def k_per_point(self):
        return np.bincount(self.obs_pt, minlength=self.n_pt)

    def sum_k2(self):
        k = self.k_per_point().astype(np.int64)
        return int((k * k).sum())


# ----------------------------------------------------------------------------
# forward camera model in matrix form (scene synthesis only)
# ----------------------------------------------------------------------------

def _project_mat(Rm, t, f, k1, k2, X):
    """Project points X (..., 3) with rotation matrices Rm (..., 3, 3).

    Returns (pixels (..., 2), depth (...,)) where depth = -P_z (> 0 in front).
    """
    pix, depth, _ = _project_mat_p(Rm, t, f, k1, k2, X)
    return pix, depth


def _project_mat_p(Rm, t, f, k1, k2, X):
    P = np.einsum("...ij,...j->...i", Rm, X) + t
    depth = -P[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        p = P[..., :2] / depth[..., None]
    r2 = (p * p).sum(-1)
    d = 1.0 + k1 * r2 + k2 * r2 * r2
    return (f * d)[..., None] * p, depth, p


def _visible(Rm, t, f, k1, k2, X):
    """In front (depth > 0.5 m), inside the image, and inside the field of
    view in normalised coordinates (|p| < 1.2), so that radial distortion
    cannot fold a point far outside the view back into the image."""
    pix, depth, p = _project_mat_p(Rm, t, f, k1, k2, X)
    with np.errstate(invalid="ignore"):
        return (depth > 0.5) & (np.abs(pix) < IMAGE_HALF).all(-1) & (np.abs(p) < 1.2).all(-1)


def _look_at(center, target, up=np.array([0.0, 0.0, 1.0])):
    """Rows x, y, z of R with z = -forward (BAL: visible points have P_z < 0)."""
    fwd = target - center
    fwd = fwd / np.linalg.norm(fwd)
    z = -fwd
    x = np.cross(up, z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z])


def _yaw_frame(yaw):
    """Camera looking horizontally along heading `yaw` (z up)."""
    c = np.array([np.cos(yaw), np.sin(yaw), 0.0])
    return _look_at(np.zeros(3), c)


def _intrinsics(rng, n, f_range=None, dist_sigma=1e-3):
    """f ~ N(500, 20) px (or log-uniform over f_range), k1, k2 ~ N(0, dist_sigma^2)."""
    if f_range is None:
        f = rng.normal(500.0, 20.0, n)
    else:
        f = np.exp(rng.uniform(np.log(f_range[0]), np.log(f_range[1]), n))
    k1 = rng.normal(0.0, dist_sigma, n)
    k2 = rng.normal(0.0, dist_sigma, n)
    return f, k1, k2


def _choose_subsets(rng, valid, k_target):
    """Pick min(k, #valid) distinct valid candidates per row, uniformly.

    valid: (m, c) bool; k_target: (m,) int.  Returns (m, c) bool selection.
    """
    keys = rng.random(valid.shape)
    keys[~valid] = np.inf
    order = np.argsort(keys, axis=1)
    ranks = np.empty_like(order)
    rows = np.arange(valid.shape[0])[:, None]
    ranks[rows, order] = np.arange(valid.shape[1])[None, :]
    k_eff = np.minimum(k_target, valid.sum(1))
    return (ranks < k_eff[:, None]) & valid


# ----------------------------------------------------------------------------
# per-config ground truth
# ----------------------------------------------------------------------------

def _ring_cameras(rng, n_cam, radius, height_sigma, target_sigma):
    ang = np.linspace(0.0, 2.0 * np.pi, n_cam, endpoint=False)
    ang = ang + rng.normal(0.0, 0.25 * 2.0 * np.pi / n_cam, n_cam)
    C = np.stack([radius * np.cos(ang), radius * np.sin(ang),
                  rng.normal(0.0, height_sigma, n_cam)], 1)
    R = np.stack([_look_at(C[i], rng.normal(0.0, target_sigma, 3))
                  for i in range(n_cam)])
    t = -np.einsum("nij,nj->ni", R, C)
    return R, t


def _gt_ring(rng, n_cam, n_pt, radius, box_half, k_sampler, window=None,
             height_sigma=0.0, target_sigma=0.0, chunk=20000, f_range=None, dist_sigma=1e-3):
    """Cameras on a ring facing the centre, points uniform in a box.

    Each point draws k and then k distinct cameras uniformly from a window
    of consecutive ring cameras (all of them when window is None); the
    geometry keeps every point visible from every camera, and a point whose
    chosen views are not all valid is re-drawn (rejection sampling).
    """
    R, t = _ring_cameras(rng, n_cam, radius, height_sigma, target_sigma)
    f, k1, k2 = _intrinsics(rng, n_cam, f_range, dist_sigma)
    X = rng.uniform(-box_half, box_half, (n_pt, 3))
    win = n_cam if (window is None or window >= n_cam) else window
    obs_cam, obs_pt = [], []
    todo = np.arange(n_pt)
    while todo.size:
        nxt = []
        for c0 in range(0, todo.size, chunk):
            idx = todo[c0:c0 + chunk]
            m = idx.size
            kt = np.minimum(k_sampler(rng, m), win)
            start = rng.integers(0, n_cam, m) if win < n_cam else np.zeros(m, np.int64)
            sel = _choose_subsets(rng, np.ones((m, win), bool), kt)
            rows, cols = np.nonzero(sel)
            cams = (start[rows] + cols) % n_cam
            ok_pair = _visible(R[cams], t[cams], f[cams], k1[cams], k2[cams], X[idx[rows]])
            ok = np.ones(m, bool)
            ok[rows[~ok_pair]] = False
            keep = ok[rows]
            obs_pt.append(idx[rows[keep]])
            obs_cam.append(cams[keep])
            bad = idx[~ok]
            X[bad] = rng.uniform(-box_half, box_half, (bad.size, 3))
            nxt.append(bad)
        todo = np.concatenate(nxt)
    return R, t, f, k1, k2, X, np.concatenate(obs_cam), np.concatenate(obs_pt)


def _gt_walk(rng, n_cam, n_pt, k_sampler, window=80, step_sigma=0.5, depth_range=(2.0, 20.0)):
    """Cameras along a random-walk trajectory with drifting heading."""
    yaw = np.cumsum(rng.normal(0.0, 0.05, n_cam))
    step = rng.normal(0.0, step_sigma, (n_cam, 3))
    step[:, 2] *= 0.1
    C = np.cumsum(step, 0)
    R = np.stack([_yaw_frame(y) for y in yaw])
    t = -np.einsum("nij,nj->ni", R, C)
    f, k1, k2 = _intrinsics(rng, n_cam)
    X = np.empty((n_pt, 3))
    obs_cam, obs_pt = [], []
    todo = np.arange(n_pt)
    chunk = 20000
    while todo.size:
        nxt = []
        for c0 in range(0, todo.size, chunk):
            idx = todo[c0:c0 + chunk]
            m = idx.size
            anchor = rng.integers(0, n_cam, m)
            uv = rng.uniform(-0.9 * IMAGE_HALF, 0.9 * IMAGE_HALF, (m, 2))
            depth = rng.uniform(depth_range[0], depth_range[1], m)
            Pc = np.concatenate([uv / f[anchor, None] * depth[:, None],
                                 -depth[:, None]], 1)
            X[idx] = np.einsum("nji,nj->ni", R[anchor], Pc - t[anchor])
            cand = anchor[:, None] + np.arange(-window, window + 1)[None, :]
            inr = (cand >= 0) & (cand < n_cam)
            cand = np.clip(cand, 0, n_cam - 1)
            valid = inr & _visible(R[cand], t[cand], f[cand], k1[cand], k2[cand],
                                   X[idx][:, None, :])
            sel = _choose_subsets(rng, valid, k_sampler(rng, m))
            ok = sel.sum(1) >= 2
            rows, cols = np.nonzero(sel & ok[:, None])
            obs_pt.append(idx[rows])
            obs_cam.append(cand[rows, cols])
            nxt.append(idx[~ok])
        todo = np.concatenate(nxt)
    return R, t, f, k1, k2, X, np.concatenate(obs_cam), np.concatenate(obs_pt)


def _geom0(p, cap):
    """k = min(cap, 2 + G), G ~ Geometric(p) counting failures (support >= 0)."""
    def sampler(rng, m):
        return np.minimum(cap, 2 + (rng.geometric(p, m) - 1))
    return sampler


def _pareto_floor(alpha, cap):
    """k = min(cap, 2 + floor(X)), X ~ classic Pareto(x_m = 1, alpha)."""
    def sampler(rng, m):
        x = 1.0 + rng.pareto(alpha, m)
        return np.minimum(cap, 2 + np.floor(x).astype(np.int64))
    return sampler


# ----------------------------------------------------------------------------
# assembly: observations, perturbation, gauge normalisation
# ----------------------------------------------------------------------------

def _finish(rng, name, seed, R, t, f, k1, k2, X, obs_cam, obs_pt,
            noise_px, perturb, outlier_frac=0.0):
    order = np.lexsort((obs_cam, obs_pt))  # tidy (pt, cam) order; any order is legal input
    obs_cam = obs_cam[order].astype(np.int32)
    obs_pt = obs_pt[order].astype(np.int32)
    pix, depth = _project_mat(R[obs_cam], t[obs_cam], f[obs_cam],
                              k1[obs_cam], k2[obs_cam], X[obs_pt])
    assert (depth > 0).all()
    obs_xy = pix + rng.normal(0.0, noise_px, pix.shape) if noise_px > 0 else pix.copy()
    if outlier_frac > 0:
        # gross outliers: a fraction of the measurements replaced by pixels drawn
        # uniformly over the image (a separate stream, so the inliers are unchanged)
        orng = np.random.default_rng([seed, 7919])
        bad = orng.random(obs_xy.shape[0]) < outlier_frac
        obs_xy[bad] = orng.uniform(-IMAGE_HALF, IMAGE_HALF, (int(bad.sum()), 2))

    # perturbed initial state (metres)
    n_cam = R.shape[0]
    if perturb:
        dR = Rotation.from_rotvec(rng.normal(0.0, 0.01, (n_cam, 3))).as_matrix()
        R0 = np.einsum("nij,njk->nik", dR, R)
        t0 = t + rng.normal(0.0, 0.05, t.shape)
        X0 = X + rng.normal(0.0, 0.1, X.shape)
    else:
        R0, t0, X0 = R.copy(), t.copy(), X.copy()

    # Sec. 6.2: drop observations with small or negative z in the camera frame
    # of the perturbed state (read as depth < 1 m or |P_xy / P_z| >= 1.5), then
    # landmarks left with fewer than two observations (points re-indexed)
    _, dep0, p0 = _project_mat_p(R0[obs_cam], t0[obs_cam], f[obs_cam], k1[obs_cam],
                                 k2[obs_cam], X0[obs_pt])
    with np.errstate(invalid="ignore"):
        keep = (dep0 > 1.0) & (np.abs(p0) < 1.5).all(-1)
    cnt = np.bincount(obs_pt[keep], minlength=X.shape[0])
    keep &= cnt[obs_pt] >= 2
    if not keep.all():
        obs_cam, obs_pt, obs_xy = obs_cam[keep], obs_pt[keep], obs_xy[keep]
        used = np.unique(obs_pt)
        remap = np.full(X.shape[0], -1, np.int64)
        remap[used] = np.arange(used.size)
        obs_pt = remap[obs_pt].astype(np.int32)
        X, X0 = X[used], X0[used]

    # gauge normalisation from the initial state
    center = np.median(X0, axis=0)
    mad = np.median(np.abs(X0 - center).sum(1))
    s = 100.0 / mad

    def to_gauge(Rm, tv, Xp):
        C = -np.einsum("nji,nj->ni", Rm, tv)           # camera centres
        Cn = s * (C - center)
        tn = -np.einsum("nij,nj->ni", Rm, Cn)
        return tn, s * (Xp - center)

    t0n, X0n = to_gauge(R0, t0, X0)
    tgn, Xgn = to_gauge(R, t, X)

    def pack(Rm, tv):
        aa = Rotation.from_matrix(Rm).as_rotvec()
        return np.concatenate([aa, tv, f[:, None], k1[:, None], k2[:, None]], 1)

    return Scene(cams=pack(R0, t0n), pts=X0n, obs_cam=obs_cam, obs_pt=obs_pt,
                 obs_xy=obs_xy, cams_gt=pack(R, tgn), pts_gt=Xgn,
                 name=name, seed=seed)


CONFIGS = ("tiny", "medium", "large", "small", "batched_member", "walk")


def degenerate_scene(seed=0, n_pt=300, noise_px=1.0):
    """A small ring scene plus landmarks on which the method's degenerate
    branches run (no gauge normalisation; the special cameras and landmarks
    keep their exact ground-truth state).

    Cameras 0..7 form a ring of radius 10 m facing the origin (perturbed
    initial state).  Camera 8 (axis-angle exactly 0, centre (0, 0, 10)) and
    camera 9 (axis-angle 0, centre (0, 0, 14)) look down the z axis; camera 10
    shares camera 8's centre and is tilted by 0.2 rad.  Landmarks:
      n_pt regular points in a 5 m cube, seen by the cameras that see them;
      `axis`: (0, 0, 0.5), seen by cameras 8 and 9 only: both project it onto
        their optical axis (P_x = P_y = 0 exactly), so the depth column of its
        landmark Jacobian is exactly zero (rank 2, a zero sub-column in the
        third Householder step);
      `same_centre`: seen by cameras 8 and 10 only, which share a centre: the
        ray direction is a null vector of its landmark Jacobian (rank 2 in
        exact arithmetic);
      `near`: 0.08 m in front of camera 8 (and seen by camera 9 from 4.08 m):
        a near-zero depth with Jacobian entries of order f / depth.
    Returns (scene, dict of the special landmark indices)."""
    rng = np.random.default_rng(seed)
    n_ring = 8
    Rr, tr = _ring_cameras(rng, n_ring, 10.0, 0.3, 0.0)
    fr, k1r, k2r = _intrinsics(rng, n_ring)
    tilt = Rotation.from_rotvec([0.2, 0.0, 0.0]).as_matrix()
    Rs = np.stack([np.eye(3), np.eye(3), tilt])
    Cs = np.array([[0.0, 0.0, 10.0], [0.0, 0.0, 14.0], [0.0, 0.0, 10.0]])
    ts = -np.einsum("nij,nj->ni", Rs, Cs)
    R = np.concatenate([Rr, Rs])
    t = np.concatenate([tr, ts])
    f = np.concatenate([fr, [500.0, 520.0, 480.0]])
    k1 = np.concatenate([k1r, [0.0, 0.0, 0.0]])
    k2 = np.concatenate([k2r, [0.0, 0.0, 0.0]])
    n_cam = R.shape[0]
    X = rng.uniform(-2.5, 2.5, (n_pt, 3))
    vis = _visible(R[None], t[None], f[None], k1[None], k2[None], X[:, None, :])
    keep = vis.sum(1) >= 2
    X, vis = X[keep], vis[keep]
    obs_pt, obs_cam = np.nonzero(vis)
    # the direction that camera 10 sees at pixel (40, -30), from the common centre
    d10 = np.array([40.0 / 480.0, -30.0 / 480.0, -1.0])
    X_same = Cs[0] + 6.0 * (tilt.T @ d10)
    special = np.array([[0.0, 0.0, 0.5], X_same, [0.0005, -0.0004, 9.92]])
    views = [(8, 9), (8, 10), (8, 9)]
    base = X.shape[0]
    X = np.concatenate([X, special])
    for i, cams in enumerate(views):
        obs_pt = np.concatenate([obs_pt, np.full(len(cams), base + i)])
        obs_cam = np.concatenate([obs_cam, np.array(cams)])
    order = np.lexsort((obs_cam, obs_pt))
    obs_cam = obs_cam[order].astype(np.int32)
    obs_pt = obs_pt[order].astype(np.int32)
    pix, depth = _project_mat(R[obs_cam], t[obs_cam], f[obs_cam], k1[obs_cam], k2[obs_cam], X[obs_pt])
    assert (depth > 0).all()
    obs_xy = pix + rng.normal(0.0, noise_px, pix.shape)
    # perturbed initial state of the ring cameras and the regular points only
    dR = Rotation.from_rotvec(rng.normal(0.0, 0.01, (n_ring, 3))).as_matrix()
    R0 = R.copy()
    R0[:n_ring] = np.einsum("nij,njk->nik", dR, R[:n_ring])
    t0 = t.copy()
    t0[:n_ring] += rng.normal(0.0, 0.05, (n_ring, 3))
    X0 = X.copy()
    X0[:base] += rng.normal(0.0, 0.1, (base, 3))

    def pack(Rm, tv):
        aa = Rotation.from_matrix(Rm).as_rotvec()
        aa[n_ring:n_ring + 2] = 0.0  # exactly zero for the axis cameras
        return np.concatenate([aa, tv, f[:, None], k1[:, None], k2[:, None]], 1)

    sc = Scene(cams=pack(R0, t0), pts=X0, obs_cam=obs_cam, obs_pt=obs_pt, obs_xy=obs_xy,
               cams_gt=pack(R, t), pts_gt=X, name="degenerate", seed=seed)
    return sc, dict(axis=base, same_centre=base + 1, near=base + 2, n_cam=n_cam)


def make_scene(name="tiny", seed=0, noise_px=1.0, perturb=True, outlier_frac=0.0, **kw):
    """Build one seeded synthetic scene.

    tiny   : 16 cams on a 10 m circle facing a 5 m cube of 500 points,
             k = min(16, 2 + Geom0(0.4)).
    medium : 500 cams along a random walk (step N(0, 0.5 m), heading drift
             0.05 rad), 100k points placed in front of anchor cameras at
             depth U[2, 20] m, k = min(64, 2 + Geom0(0.2)), visible cameras
             searched within +-80 trajectory neighbours.
    large  : 1800 cams on a 30 m ring, 1M points in a 12 m cube,
             k = min(200, 2 + floor(Pareto(1.5))), cameras drawn from a
             window of 600 ring neighbours (heavy-tailed, venice-like).
    small  : tiny-like ring with n_cam / n_pt / p given by keywords
             (defaults 32 cams, 2000 points, p = 0.3, cap 32); f_range =
             (lo, hi) draws focal lengths log-uniformly, dist_sigma sets the
             spread of k1, k2 (ill-conditioned camera sets).
    outlier_frac > 0 (any config) replaces that fraction of the pixel
    measurements by gross outliers uniform over the image (the robust-norm
    experiments of Sec. 6.2; the BAL data are not available here).
    batched_member : member `seed` of the 256-problem batch: cams U[8, 64],
             points U[200, 5000], k = 2 + Geom0(0.3) capped at n_cam.
    walk   : medium-shaped (the medium generator and k distribution) with
             n_cam / n_pt given by keywords (defaults 100 cams, 20000
             points); the training and evaluation scenes of the learned
             warm start.  step_sigma (m) and depth = (lo, hi) (m) set the
             baselines and point depths (short baselines to far points make
             the landmark blocks ill-conditioned).
    """
    rng = np.random.default_rng(seed)
    if name == "tiny":
        gt = _gt_ring(rng, 16, 500, 10.0, 2.5, _geom0(0.4, 16))
    elif name == "medium":
        gt = _gt_walk(rng, 500, 100_000, _geom0(0.2, 64))
    elif name == "large":
        gt = _gt_ring(rng, 1800, 1_000_000, 30.0, 6.0, _pareto_floor(1.5, 200),
                      window=600, height_sigma=2.0, target_sigma=1.0)
    elif name == "small":
        n_cam = kw.get("n_cam", 32)
        n_pt = kw.get("n_pt", 2000)
        gt = _gt_ring(rng, n_cam, n_pt, 10.0, 2.5,
                      _geom0(kw.get("p", 0.3), kw.get("cap", 32)),
                      height_sigma=0.5, f_range=kw.get("f_range"),
                      dist_sigma=kw.get("dist_sigma", 1e-3))
    elif name == "walk":
        gt = _gt_walk(rng, kw.get("n_cam", 100), kw.get("n_pt", 20_000), _geom0(0.2, 64),
                      step_sigma=kw.get("step_sigma", 0.5), depth_range=kw.get("depth", (2.0, 20.0)))
    elif name == "batched_member":
        n_cam = int(rng.integers(8, 65))
        n_pt = int(rng.integers(200, 5001))
        gt = _gt_ring(rng, n_cam, n_pt, 10.0, 2.5, _geom0(0.3, n_cam),
                      height_sigma=0.5)
    else:
        raise ValueError(f"unknown scene config {name!r}")
    return _finish(rng, name, seed, *gt, noise_px=noise_px, perturb=perturb, outlier_frac=outlier_frac)
