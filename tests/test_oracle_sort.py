"""Pins of the oracle's grouping of observations by landmark (Sec. 5.1)."""
import numpy as np

import oracle
from paper_2103_01843_gb300.synth import make_scene


def test_sort_matches_numpy_lexsort():
    s = make_scene("small", 1, n_cam=12, n_pt=300)
    rng = np.random.default_rng(0)
    sh = rng.permutation(s.n_obs)
    oc, op = s.obs_cam[sh], s.obs_pt[sh]
    rc, perm, pt_off, cam_off, cam_list = oracle.sort_obs(s.n_cam, s.n_pt, oc, op)
    assert rc == 0
    np.testing.assert_array_equal(perm, np.lexsort((oc, op)))
    np.testing.assert_array_equal(pt_off, np.concatenate([[0], np.cumsum(np.bincount(op, minlength=s.n_pt))]))
    np.testing.assert_array_equal(cam_off, np.concatenate([[0], np.cumsum(np.bincount(oc, minlength=s.n_cam))]))
    sorted_cam = oc[perm]
    for i in range(s.n_cam):
        np.testing.assert_array_equal(cam_list[cam_off[i]:cam_off[i + 1]], np.nonzero(sorted_cam == i)[0])


def test_sort_rejects_invalid_input():
    oc = np.array([0, 1, 0, 1], np.int32)
    op = np.array([0, 0, 1, 1], np.int32)
    assert oracle.sort_obs(2, 2, oc, op)[0] == 0
    assert oracle.sort_obs(2, 2, np.array([0, 1, 0, 0], np.int32), op)[0] != 0   # duplicate
    assert oracle.sort_obs(2, 3, oc, op)[0] != 0                                 # landmark with 0 obs
    assert oracle.sort_obs(2, 2, np.array([0, 1, 0, 2], np.int32), op)[0] != 0   # camera out of range
    assert oracle.sort_obs(2, 2, oc, np.array([0, 0, 1, -1], np.int32))[0] != 0  # landmark out of range
