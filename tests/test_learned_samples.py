"""Host-side filter of the learned model's training samples
(paper_2103_01843_gb300.learned.clean_samples): which samples it drops and
why, checked against closed forms (||L^-1 g||^2 = g^T M^-1 g and
||L^T x||^2 = x^T M x for M = L L^T) rather than against its own Cholesky."""
import numpy as np

from paper_2103_01843_gb300.learned import clean_samples


def _spd(rng, n):
    A = rng.standard_normal((n, 9, 9))
    return A @ A.transpose(0, 2, 1) + 0.5 * np.eye(9)


def test_filter_counts_and_kept_samples():
    rng = np.random.default_rng(0)
    n = 40
    M = _spd(rng, n)
    g = rng.standard_normal((n, 9))
    x = np.linalg.solve(M, g[:, :, None])[:, :, 0] + 0.1 * rng.standard_normal((n, 9))
    M[0, 3, 3] = np.nan                       # non-finite block
    g[1, 2] = np.inf                          # non-finite right-hand side
    M[2] = -np.eye(9)                         # not positive definite
    M[3, 0, 1] = M[3, 1, 0] = 10.0 * np.sqrt(M[3, 0, 0] * M[3, 1, 1])  # indefinite
    x[4] = 0.0                                # zero target
    x[5] *= 1e-5                              # block-Jacobi term 1e10 x the target: dropped
    x[6] *= 1e-2                              # 1e4 x: kept
    data = dict(M=M.reshape(n, 81).astype(np.float32), g=g.astype(np.float32),
                xstar=x.astype(np.float32), count=np.arange(n, dtype=np.int32))
    out, counts = clean_samples(data, chunk=16)
    assert counts == dict(total=n, non_finite=2, not_pd=2, zero_target=1, ratio=1, kept=n - 6)
    np.testing.assert_array_equal(out["count"], np.arange(6, n, dtype=np.int32))
    for k in ("M", "g", "xstar"):
        assert out[k].dtype == np.float32 and out[k].shape[0] == n - 6


def test_ratio_threshold_matches_the_closed_form():
    rng = np.random.default_rng(1)
    n = 200
    M = _spd(rng, n)
    g = rng.standard_normal((n, 9))
    x = rng.standard_normal((n, 9)) * 10.0 ** rng.uniform(-5, 1, size=(n, 1))
    data = dict(M=M.reshape(n, 81).astype(np.float32), g=g.astype(np.float32),
                xstar=x.astype(np.float32), count=np.ones(n, np.int32))
    M64 = data["M"].reshape(n, 9, 9).astype(np.float64)
    g64, x64 = data["g"].astype(np.float64), data["xstar"].astype(np.float64)
    w2 = np.einsum("ni,ni->n", g64, np.linalg.solve(M64, g64[:, :, None])[:, :, 0])
    z2 = np.einsum("ni,nij,nj->n", x64, M64, x64)
    ratio = w2 / z2
    assert np.all(np.abs(np.log(ratio / 1e3)) > 1e-3)  # no sample at the threshold itself
    out, counts = clean_samples(data, max_ratio=1e3)
    assert 0 < counts["ratio"] < n
    assert counts["ratio"] == int((ratio > 1e3).sum())
    np.testing.assert_array_equal(out["xstar"], data["xstar"][ratio <= 1e3])
