"""Pins of the oracle's robust norm (Sec. 6.2: Huber with a 1 px parameter;
reading: the Huber function of s = ||r_ij||^2 applied by iteratively
reweighted least squares).

* Limits: a parameter above every residual norm gives the squared norm
  exactly; any parameter gives a cost at or below the squared norm.
* First-order exactness of the reweighted model: along the LM step the
  decrease the model predicts, E - L, and the true decrease of the robust
  cost agree to first order in the step, so their relative difference halves
  when the damping doubles.  A wrong weight (w instead of sqrt(w) on the
  rows, or an unweighted model) leaves a constant relative error instead.
* The robust solution of a scene with gross outliers lies closer to the
  ground truth than the squared-norm solution (median landmark error).
"""
import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.synth import make_scene


@pytest.fixture(scope="module")
def outliers():
    return make_scene("tiny", 0, outlier_frac=0.05)


def test_limits_of_the_huber_cost(outliers):
    plain = oracle.cost(outliers)
    assert oracle.cost(outliers, huber_delta=1e12) == plain
    costs = [oracle.cost(outliers, huber_delta=d) for d in (0.5, 1.0, 4.0, 64.0)]
    assert all(c < plain for c in costs)
    assert all(a < b for a, b in zip(costs, costs[1:]))  # increasing in the parameter
    st0 = oracle.linear_step(outliers, 1e-3, dense=True)
    st1 = oracle.linear_step(outliers, 1e-3, dense=True, huber_delta=1e12)
    np.testing.assert_array_equal(st0["dp"], st1["dp"])
    assert st0["model_cost"] == st1["model_cost"]


def test_reweighted_model_is_first_order_exact(outliers):
    rel = []
    for lam in (1e5, 2e5, 4e5):
        st = oracle.linear_step(outliers, lam, dense=True, huber_delta=1.0)
        c, p = oracle.apply_update(outliers.cams, st["dp"], outliers.pts, st["dl"])
        E, L = st["cost"], st["model_cost"]
        En = oracle.cost(outliers, c, p, huber_delta=1.0)
        assert E == pytest.approx(oracle.cost(outliers, huber_delta=1.0), rel=1e-12)
        rel.append(abs((E - En) - (E - L)) / (E - L))
    assert rel[0] < 1e-4
    for a, b in zip(rel, rel[1:]):
        assert 0.4 < b / a < 0.6, rel


def test_robust_solution_is_closer_to_ground_truth():
    s = make_scene("tiny", 2, outlier_frac=0.05)
    err = {}
    for name, delta in (("plain", 0.0), ("huber", 1.0)):
        _, pts, log = oracle.lm(s, max_iters=30, dense=True, huber_delta=delta)
        assert log[-1]["accepted"] or any(e["accepted"] for e in log)
        # median point error in the gauge of the ground truth (a landmark seen
        # twice, once by an outlier, is not determined by either norm)
        err[name] = float(np.median(np.linalg.norm(pts - s.pts_gt, axis=1)))
    assert err["huber"] < 0.2 * err["plain"], err
