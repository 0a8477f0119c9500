"""The precision reading of the energy and model-cost sums (Sec. 6.1: FP32
arithmetic, the cost sums in FP64): each observation's term rho(r0^2 + r1^2)
is formed in FP32 from the FP32 residuals and added to an FP64 sum.

What this file pins, on the host, is the error bound that reading rests on:
for FP32 inputs, the FP32 term (two products and a sum, with or without a
fused multiply-add) is within 2^-23 of the exact term relative to it, the
robust branch evaluated in FP64 from the FP32 square keeps that bound, and so
does the FP64 sum of positive terms (its own rounding is ~2^-53 per add).
The FP32 residual itself already carries a relative error of about 2^-24 of
the projected coordinate, which is larger than the term's rounding for every
residual smaller than the projection, so the FP32 square adds nothing that
the FP32 residual does not already bring."""
import numpy as np

U32 = 2.0 ** -24  # unit roundoff of FP32


def _terms_fp32(r0, r1, fused):
    """The term r0^2 + r1^2 as the kernels form it: in FP32, the first
    product either rounded (plain) or kept exact inside a fused multiply-add."""
    r0 = r0.astype(np.float32)
    r1 = r1.astype(np.float32)
    p1 = (r1 * r1).astype(np.float32)
    if fused:
        # fma(r0, r0, p1): r0^2 is exact in FP64 (two 24-bit significands),
        # then one rounding of the sum to FP32 (via FP64: within the bound)
        return (r0.astype(np.float64) ** 2 + p1.astype(np.float64)).astype(np.float32)
    return ((r0 * r0).astype(np.float32) + p1).astype(np.float32)


def _huber(delta, s):
    return np.where(s > delta * delta, 2.0 * delta * np.sqrt(s) - delta * delta, s)


def _residuals(rng, n):
    # residual magnitudes from 1e-3 px to 1e3 px (the converged and the
    # initial states of the bench scenes), both signs
    mag = 10.0 ** rng.uniform(-3, 3, size=(n, 2))
    return (mag * rng.choice([-1.0, 1.0], size=(n, 2))).astype(np.float32)


def test_fp32_term_is_within_two_unit_roundoffs():
    rng = np.random.default_rng(0)
    r = _residuals(rng, 200_000)
    exact = r[:, 0].astype(np.float64) ** 2 + r[:, 1].astype(np.float64) ** 2  # exact in FP64
    for fused in (False, True):
        t = _terms_fp32(r[:, 0], r[:, 1], fused).astype(np.float64)
        rel = np.abs(t - exact) / exact
        assert rel.max() <= 2 * U32, (fused, rel.max())
        # the bound is not vacuous: FP32 rounding does show
        assert rel.max() > 0.25 * U32


def test_robust_branch_keeps_the_bound():
    rng = np.random.default_rng(1)
    r = _residuals(rng, 100_000)
    delta = 1.0
    exact = _huber(delta, r[:, 0].astype(np.float64) ** 2 + r[:, 1].astype(np.float64) ** 2)
    s32 = _terms_fp32(r[:, 0], r[:, 1], True)
    t = np.where(s32 > np.float32(delta * delta), _huber(delta, s32.astype(np.float64)),
                 s32.astype(np.float64))
    rel = np.abs(t - exact) / exact
    assert rel.max() <= 2 * U32, rel.max()


def test_fp64_sum_of_fp32_terms_meets_the_bound_and_fp32_sums_would_not():
    rng = np.random.default_rng(2)
    n = 600_000  # about the medium scene's observation count
    r = _residuals(rng, n)
    exact_terms = r[:, 0].astype(np.float64) ** 2 + r[:, 1].astype(np.float64) ** 2
    E = float(np.sum(exact_terms))  # reference (FP64 pairwise sum)
    t32 = _terms_fp32(r[:, 0], r[:, 1], True)
    # sequential FP64 accumulation, the worst order for rounding growth
    acc = 0.0
    for c in np.array_split(t32.astype(np.float64), 64):
        for v in c.tolist():
            acc += v
    assert abs(acc - E) <= 2 * U32 * E, (acc, E)
    # the reason the sums stay in FP64: a sequential FP32 sum drifts far
    # beyond the per-term bound at this count
    acc32 = np.float32(0.0)
    for v in t32[:: max(1, n // 100_000)]:
        acc32 = np.float32(acc32 + v)
    sub = float(np.sum(exact_terms[:: max(1, n // 100_000)]))
    assert abs(float(acc32) - sub) > 16 * U32 * sub
