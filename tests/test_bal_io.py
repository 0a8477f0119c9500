"""The BAL text reader and writer (the input format of the paper's
experiments, Sec. 6.2): a hand-written two-camera file
(tests/golden/bal_two_cameras.txt, made up for this test, not a BAL
problem), a round trip of a synthetic scene through .txt and .bz2, and the
rejection of malformed files."""
import os

import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.bal import read_bal, write_bal
from paper_2103_01843_gb300.synth import make_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bal_two_cameras.txt")


def test_hand_written_file():
    s = read_bal(GOLDEN)
    assert (s.n_cam, s.n_pt, s.n_obs) == (2, 3, 5)
    np.testing.assert_array_equal(s.obs_cam, [0, 1, 0, 1, 0])
    np.testing.assert_array_equal(s.obs_pt, [0, 0, 1, 1, 2])
    np.testing.assert_array_equal(s.obs_xy[3], [-7.125, 1.0])
    np.testing.assert_array_equal(s.cams[0], [0.01, -0.02, 0.03, 0.1, 0.2, -5.0, 500.0, 0.001, -0.0005])
    np.testing.assert_array_equal(s.cams[1, 3:7], [1.0, 0.0, -6.0, 520.0])
    np.testing.assert_array_equal(s.pts[2], [0.0, 0.0, -1.0])
    # the arrays feed the solver's camera model unchanged
    r, _, _ = oracle.residual(s.cams[0], s.pts[0], s.obs_xy[0])
    assert np.all(np.isfinite(r))


@pytest.mark.parametrize("ext", [".txt", ".bz2"])
def test_round_trip(tmp_path, ext):
    s = make_scene("tiny", 1)
    path = str(tmp_path / ("scene" + ext))
    write_bal(s, path)
    t = read_bal(path)
    for key in ("cams", "pts", "obs_cam", "obs_pt", "obs_xy"):
        np.testing.assert_array_equal(getattr(t, key), getattr(s, key))
    assert oracle.cost(t) == oracle.cost(s)


@pytest.mark.parametrize("text", [
    "2 1",                                             # short header
    "1 1 1\n0 0 1.0 2.0\n" + "0\n" * 9,               # point values missing
    "1 1 1\n1 0 1.0 2.0\n" + "0\n" * 12,              # camera index out of range
    "1 1 1\n0 0.5 1.0 2.0\n" + "0\n" * 12,            # fractional index
    "0 1 1\n0 0 1.0 2.0\n" + "0\n" * 3,               # empty
])
def test_malformed_files_are_rejected(text):
    with pytest.raises(ValueError):
        read_bal(text + "\n")
