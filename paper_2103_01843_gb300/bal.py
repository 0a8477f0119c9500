"""Reader and writer of the BAL text format ("Bundle Adjustment in the Large"),
the input format of the paper's experiments (Sec. 6.2), for users who supply
their own BAL files (the datasets themselves are not part of this package).

Layout of a BAL file (whitespace separated, one record per line):
    n_cam n_pt n_obs
    n_obs lines:  camera_index point_index x y
    9 n_cam values: per camera axis-angle (3), translation (3), f, k1, k2
    3 n_pt values:  per point X, Y, Z
The camera model and sign conventions are the ones the library uses (the
"Snavely" model: P = R(w) X + t, p = -P_xy / P_z, pixel = f (1 + k1 |p|^2 +
k2 |p|^4) p), so the arrays are passed to ba_create unchanged.  Files ending
in .bz2 or .gz are decompressed on the fly.
"""
from __future__ import annotations

import bz2
import gzip
import io

import numpy as np

from .synth import Scene


def _open(path, mode):
    if str(path).endswith(".bz2"):
        return bz2.open(path, mode + "t")
    if str(path).endswith(".gz"):
        return gzip.open(path, mode + "t")
    return open(path, mode)


def read_bal(path_or_text):
    """Scene (cams, pts, obs_cam, obs_pt, obs_xy; the *_gt fields hold the
    file's values too) from a BAL file path, or from BAL text when the
    argument contains a newline.  Raises ValueError on a malformed file."""
    if isinstance(path_or_text, str) and "\n" in path_or_text:
        f = io.StringIO(path_or_text)
    else:
        f = _open(path_or_text, "r")
    with f:
        tokens = f.read().split()
    if len(tokens) < 3:
        raise ValueError("BAL: missing header")
    try:
        n_cam, n_pt, n_obs = (int(t) for t in tokens[:3])
    except ValueError as e:
        raise ValueError("BAL: malformed header") from e
    if n_cam < 1 or n_pt < 1 or n_obs < 1:
        raise ValueError("BAL: empty problem")
    need = 3 + 4 * n_obs + 9 * n_cam + 3 * n_pt
    if len(tokens) != need:
        raise ValueError(f"BAL: expected {need} values, found {len(tokens)}")
    obs = np.array(tokens[3:3 + 4 * n_obs], dtype=np.float64).reshape(n_obs, 4)
    cam_idx, pt_idx = obs[:, 0], obs[:, 1]
    if not (np.all(cam_idx == np.round(cam_idx)) and np.all(pt_idx == np.round(pt_idx))):
        raise ValueError("BAL: non-integer index")
    obs_cam = cam_idx.astype(np.int32)
    obs_pt = pt_idx.astype(np.int32)
    if obs_cam.min() < 0 or obs_cam.max() >= n_cam or obs_pt.min() < 0 or obs_pt.max() >= n_pt:
        raise ValueError("BAL: observation index out of range")
    o = 3 + 4 * n_obs
    cams = np.array(tokens[o:o + 9 * n_cam], dtype=np.float64).reshape(n_cam, 9)
    pts = np.array(tokens[o + 9 * n_cam:], dtype=np.float64).reshape(n_pt, 3)
    return Scene(cams=cams, pts=pts, obs_cam=obs_cam, obs_pt=obs_pt, obs_xy=obs[:, 2:4].copy(),
                 cams_gt=cams.copy(), pts_gt=pts.copy(), name="bal", seed=0)


def write_bal(scene, path):
    """Writes a scene (any object with cams, pts, obs_cam, obs_pt, obs_xy) in
    the BAL format; values are written with 17 significant digits, so that
    read_bal gives back the same doubles."""
    cams = np.asarray(scene.cams, np.float64)
    pts = np.asarray(scene.pts, np.float64)
    oc = np.asarray(scene.obs_cam)
    op = np.asarray(scene.obs_pt)
    xy = np.asarray(scene.obs_xy, np.float64)
    with _open(path, "w") as f:
        f.write(f"{cams.shape[0]} {pts.shape[0]} {oc.shape[0]}\n")
        for c, p, (x, y) in zip(oc, op, xy):
            f.write(f"{int(c)} {int(p)} {x:.17g} {y:.17g}\n")
        for v in cams.ravel():
            f.write(f"{v:.17g}\n")
        for v in pts.ravel():
            f.write(f"{v:.17g}\n")
