"""Pins of the oracle's LM and CG rules against results fixed outside the oracle.

* The CG stop (Sec. 6.1, "forcing sequence"; reading: the truncated-Newton test of
  Nash and Sofer, i (Q_i - Q_{i-1}) / Q_i < eta).  PCG iterate i minimises
  Q(x) = 1/2 x^T H x - g^T x over the Krylov space K_i(M^-1 H, M^-1 g).  The test
  computes those minimisers with a dense projected solve on an Arnoldi basis (no CG
  recursion), predicts the stop iteration of the rule for several eta, and checks
  that the oracle stops there with the same Q_i and the same iterate.  The eta set
  is chosen so that two plausible misreadings of the rule (dropping the factor i,
  dividing by Q_{i-1}) would stop elsewhere.
* The damping update (Sec. 6.1; reading: Nielsen's rule) against a sequence of
  decisions worked by hand (tests/golden/nielsen_lambda_steps.txt).
* The oracle's block-sparse products with H~ against its dense assembly, which
  the brute-force solves of test_oracle_solver.py pin.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.synth import make_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nielsen_lambda_steps.txt")


def _spd(n_blk, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    n = 9 * n_blk
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(rng.uniform(0.0, math.log(cond), n))
    H = (Q * lam) @ Q.T
    return 0.5 * (H + H.T), rng.standard_normal(n)


def _block_jacobi_inverse(H, n_blk):
    Minv = np.zeros_like(H)
    for b in range(n_blk):
        s = slice(9 * b, 9 * b + 9)
        Minv[s, s] = np.linalg.inv(H[s, s])
    return Minv


def _krylov_q(H, g, n_blk, imax):
    """Q(x_i) and x_i for the minimisers over K_i(M^-1 H, M^-1 g), i = 0..imax."""
    Minv = _block_jacobi_inverse(H, n_blk)
    B = Minv @ H
    v = Minv @ g
    basis = [v / np.linalg.norm(v)]
    qs, xs = [0.0], [np.zeros_like(g)]
    for i in range(1, imax + 1):
        V = np.stack(basis, axis=1)
        y = np.linalg.solve(V.T @ H @ V, V.T @ g)
        x = V @ y
        xs.append(x)
        qs.append(0.5 * x @ H @ x - g @ x)
        w = B @ basis[-1]
        for _ in range(2):  # Gram-Schmidt, twice
            w = w - V @ (V.T @ w)
        basis.append(w / np.linalg.norm(w))
    return np.array(qs), xs


def _stop(ratios, eta):
    """First i >= 1 with ratios[i] < eta (ratios[0] unused), else None."""
    for i in range(1, len(ratios)):
        if ratios[i] < eta:
            return i
    return None


def _eta_set(ns, imax):
    """eta values on a log grid whose stop is unambiguous: every ratio up to the
    predicted stop lies at least 0.2 % away from eta (the Q_i are exact to ~1e-12)."""
    etas = []
    for eta in np.geomspace(0.05, 1.5, 120):
        i = _stop(ns, eta)
        if i is None:
            continue
        if all(abs(ns[j] - eta) > 2e-3 * eta for j in range(1, i + 1)):
            etas.append(float(eta))
    return etas


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nash_sofer_stop_matches_krylov_minimisers(seed):
    n_blk, imax = 4, 18
    H, g = _spd(n_blk, seed)
    q, xs = _krylov_q(H, g, n_blk, imax)
    i = np.arange(imax + 1)
    ns = np.full(imax + 1, np.inf)
    ns[1:] = i[1:] * (q[1:] - q[:-1]) / q[1:]
    etas = _eta_set(ns, imax)
    assert len({_stop(ns, e) for e in etas}) >= 4, ns
    # the eta set separates the rule from two misreadings of it
    no_i = np.full(imax + 1, np.inf)
    no_i[1:] = (q[1:] - q[:-1]) / q[1:]
    prev_den = np.full(imax + 1, np.inf)
    prev_den[2:] = i[2:] * (q[2:] - q[1:-1]) / q[1:-1]
    for wrong in (no_i, prev_den):
        assert any(_stop(wrong, e) != _stop(ns, e) for e in etas)
    for eta in etas:
        want = _stop(ns, eta)
        x, it, Q, st = oracle.pcg_dense(H, g, max_it=imax, eta=eta)
        assert st == 0
        assert it == want, (eta, it, want, ns)
        np.testing.assert_allclose(Q, q[: it + 1], rtol=1e-9, atol=0)
        np.testing.assert_allclose(x, xs[it], rtol=0, atol=1e-9 * np.abs(xs[it]).max())


def test_pcg_iteration_limit_and_residual_stop():
    H, g = _spd(3, 7)
    # eta = 0: the Nash-Sofer test never fires, the limit ends the run
    _, it, _, st = oracle.pcg_dense(H, g, max_it=5, eta=0.0)
    assert (it, st) == (5, 0)
    # block-diagonal H: block Jacobi is exact, the residual vanishes after one step
    Hb = np.zeros_like(H)
    for b in range(3):
        s = slice(9 * b, 9 * b + 9)
        Hb[s, s] = H[s, s]
    x, it, _, st = oracle.pcg_dense(Hb, g, max_it=50, eta=0.0)
    assert (it, st) == (1, 0)
    np.testing.assert_allclose(Hb @ x, g, rtol=0, atol=1e-10 * np.abs(g).max())


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            lhs, rhs = ln.split("|")
            E, En, L, lam, nu, tol, target = (float(t) for t in lhs.split())
            acc, stop, lam_after, nu_after = rhs.split()
            rows.append(((E, En, L, lam, nu, tol, target),
                         (bool(int(acc)), bool(int(stop)), float(lam_after), float(nu_after))))
    return rows


def test_nielsen_update_matches_hand_worked_steps():
    rows = _golden_rows()
    assert len(rows) == 18
    for n, ((E, En, L, lam, nu, tol, target), (acc, stop, lam_after, nu_after)) in enumerate(rows):
        d = oracle.lm_decide(E, En, L, lam, nu, func_tol=tol, target_cost=target)
        assert (d["accepted"], d["stop"]) == (acc, stop), (n, d)
        assert d["lam"] == pytest.approx(lam_after, rel=1e-12), (n, d)
        assert d["nu"] == nu_after, (n, d)
    # rows 1-10 chain: each starts from the previous decision's damping
    for (a, ra), (b, _) in zip(rows[:9], rows[1:10]):
        assert b[3] == pytest.approx(ra[2], rel=1e-15) and b[4] == ra[3]


def test_lm_log_follows_the_decision_rule(tiny_scene):
    """The LM loop takes its damping from the pinned decision routine."""
    _, _, log = oracle.lm(tiny_scene, max_iters=20, dense=True)
    lam, nu = 1e-4, 2.0
    for e in log:
        assert e["lam"] == lam
        d = oracle.lm_decide(e["cost"], e["new_cost"], e["model_cost"], lam, nu)
        assert d["accepted"] == e["accepted"]
        lam, nu = d["lam"], d["nu"]


def test_rcs_matvec_equals_dense_assembly():
    s = make_scene("small", 3, n_cam=6, n_pt=120)
    rng = np.random.default_rng(5)
    for lam in (1e-4, 1.0):
        H, _ = oracle.rcs_dense(s, lam)
        V = rng.standard_normal((3, H.shape[0]))
        Y = oracle.rcs_matvec(s, lam, V)
        np.testing.assert_allclose(Y, V @ H.T, rtol=0, atol=1e-10 * np.abs(V @ H.T).max())
