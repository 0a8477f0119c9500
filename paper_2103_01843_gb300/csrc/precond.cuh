// The per-camera finish of K3 (block-Jacobi preconditioner, Sec. 5.4 / 6.1),
// shared by the square-root forms (pcg.cu) and the explicit Schur complement
// (schur.cu).
#pragma once

#include "common.cuh"

namespace sqrtba {

// Second half of K3, one warp per camera: the 54 sums (upper triangle of
// sum_j A_ji^T A_ji and sum_j A_ji^T c_j) are expanded, lambda D_p^2 is added,
// the 9x9 block is factored by Cholesky (lanes over the rows below the
// pivot) and inverted column by column (lane c solves L L^T x = e_c).
// sM, sL: 81 floats of shared memory each.
__device__ inline void precond_finish_warp(int cam, const float* tot, const float* __restrict__ dp2, float lam,
                                  float* __restrict__ mdiag, float* __restrict__ minv, float* __restrict__ g,
                                  uint32_t* err, float* sM, float* sL, int lane) {
    for (int i = lane; i < 81; i += 32) {
        const int u = i / 9, v = i - 9 * u;
        const int lo = u < v ? u : v, hi = u < v ? v : u;
        float m = tot[9 * lo - lo * (lo - 1) / 2 + (hi - lo)];
        if (u == v) m += lam * dp2[9 * cam + u];
        sM[i] = m;
        sL[i] = 0.f;
        mdiag[81 * (int64_t)cam + i] = m;
    }
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < 9; ++j) {
        float s = sM[j * 9 + j];
        for (int m = 0; m < j; ++m) s -= sL[j * 9 + m] * sL[j * 9 + m];
        ok = ok && s > 0.f;
        const float l = s > 0.f ? sqrtf(s) : 1.f;
        if (lane > j && lane < 9) {
            float t = sM[lane * 9 + j];
            for (int m = 0; m < j; ++m) t -= sL[lane * 9 + m] * sL[j * 9 + m];
            sL[lane * 9 + j] = t / l;
        }
        if (lane == 0) sL[j * 9 + j] = l;
        __syncwarp();
    }
    if (lane < 9) {
        const int c = lane;
        float x[9];
        if (ok) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float t = i == c ? 1.f : 0.f;
#pragma unroll
                for (int m = 0; m < i; ++m) t -= sL[i * 9 + m] * x[m];
                x[i] = t / sL[i * 9 + i];
            }
#pragma unroll
            for (int i = 8; i >= 0; --i) {
                float t = x[i];
#pragma unroll
                for (int m = i + 1; m < 9; ++m) t -= sL[m * 9 + i] * x[m];
                x[i] = t / sL[i * 9 + i];
            }
        } else {
            // not positive definite in FP32: fall back to the diagonal (Jacobi)
#pragma unroll
            for (int i = 0; i < 9; ++i) x[i] = 0.f;
            const float d = sM[c * 9 + c];
#pragma unroll
            for (int i = 0; i < 9; ++i)
                if (i == c) x[i] = d > 0.f ? 1.f / d : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) minv[81 * (int64_t)cam + i * 9 + c] = x[i];
        g[9 * cam + c] = -tot[45 + c];
    }
    if (!ok && lane == 0) {
        atomicOr(err, ERRBIT_PRECOND);
        atomicAdd(err + 1, 1u);  // blocks replaced by their diagonal (read back by the host)
    }
}

}  // namespace sqrtba
