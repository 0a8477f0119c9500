// K2: landmark damping folded into the marginalised landmark blocks with six
// Givens rotations (Sec. 5.3, Fig. 3).
//
// The three damping rows [0 | sqrt(lambda) D_l | 0] are attached below the
// block (they are the last three rows of A_j); rotation m acts on the pair
// (R1 row c, damping row d) for (d, c) = (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
// and zeroes the damping row's entry in landmark column c:
//     rho = hypot(a, b), cos = a / rho, sin = b / rho  (a = pivot, b = damping entry)
//     pivot_row' = cos pivot_row + sin damp_row,  damp_row' = -sin pivot_row + cos damp_row.
// The rotations are stored individually; re-damping first applies the
// transposed rotations in reverse order and zeroes the damping rows
// (Fig. 3c), which restores the undamped block up to rounding, then applies
// the new damping.  One warp per landmark; every lane owns whole columns.
#include "problem.cuh"

namespace sqrtba {

namespace {

__constant__ int kRotC[6] = {0, 1, 2, 1, 2, 2};
__constant__ int kRotD[6] = {0, 0, 0, 1, 1, 2};

__global__ void __launch_bounds__(128)
k_damp(int n_pt, const int32_t* __restrict__ pt_off, const int64_t* __restrict__ a_off,
       float* __restrict__ tpool, float* __restrict__ apool, float* __restrict__ cpool,
       const int32_t* __restrict__ c_off,
       const float* __restrict__ dl2, float* __restrict__ rot, float sqrt_lambda, int undo) {
    __shared__ float sh_rot[4][24];  // per warp: old (12) and new (12) rotations
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n_pt) return;
    const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
    const int ncol = 9 * k, nr = 2 * k;
    float* top = tpool + top_offset(s0, j);
    float* damp = apool + a_off[j] + (int64_t)(nr - 3) * ncol;  // damping rows of A_j
    float* cd = cpool + c_off[j] + (nr - 3);                     // their residual entries
    float* rs = sh_rot[w];

    if (lane == 0) {
        float R[3][3], D[3][3];
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) {
                R[i][c] = top[i * (ncol + 4) + ncol + c];
                D[i][c] = 0.f;
            }
        if (undo) {
            for (int m = 0; m < 12; ++m) rs[m] = rot[12 * (int64_t)j + m];
            for (int m = 5; m >= 0; --m) {
                const int c = kRotC[m], d = kRotD[m];
                const float cs = rs[2 * m], sn = rs[2 * m + 1];
                for (int col = 0; col < 3; ++col) {
                    const float u = R[c][col], v = D[d][col];
                    R[c][col] = cs * u - sn * v;
                    D[d][col] = sn * u + cs * v;
                }
            }
            for (int i = 0; i < 3; ++i)
                for (int c = 0; c < 3; ++c) D[i][c] = 0.f;
        }
        for (int d = 0; d < 3; ++d) D[d][d] = sqrt_lambda * sqrtf(dl2[3 * j + d]);
        for (int m = 0; m < 6; ++m) {
            const int c = kRotC[m], d = kRotD[m];
            const float a = R[c][c], b = D[d][c];
            const float rho = hypotf(a, b);
            float cs = 1.f, sn = 0.f;
            if (rho > 0.f) {
                cs = a / rho;
                sn = b / rho;
            }
            for (int col = c; col < 3; ++col) {
                const float u = R[c][col], v = D[d][col];
                R[c][col] = cs * u + sn * v;
                D[d][col] = -sn * u + cs * v;
            }
            D[d][c] = 0.f;
            rs[12 + 2 * m] = cs;
            rs[12 + 2 * m + 1] = sn;
        }
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) top[i * (ncol + 4) + ncol + c] = c >= i ? R[i][c] : 0.f;
        for (int m = 0; m < 12; ++m) rot[12 * (int64_t)j + m] = rs[12 + m];
    }
    __syncwarp();

    float oc[6], os[6], nc[6], ns[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        oc[m] = undo ? rs[2 * m] : 1.f;
        os[m] = undo ? rs[2 * m + 1] : 0.f;
        nc[m] = rs[12 + 2 * m];
        ns[m] = rs[12 + 2 * m + 1];
    }
    // pose columns and the residual column (index ncol)
    for (int col = lane; col <= ncol; col += 32) {
        const int tc = col < ncol ? col : ncol + 3;
        float u[3], v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            u[i] = top[i * (ncol + 4) + tc];
            v[i] = 0.f;
        }
        if (undo) {
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] = col < ncol ? damp[(int64_t)i * ncol + col] : cd[i];
#pragma unroll
            for (int m = 5; m >= 0; --m) {
                const int c = m < 3 ? m : (m < 5 ? m - 2 : 2);
                const int d = m < 3 ? 0 : (m < 5 ? 1 : 2);
                const float a = u[c], b = v[d];
                u[c] = oc[m] * a - os[m] * b;
                v[d] = os[m] * a + oc[m] * b;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int c = m < 3 ? m : (m < 5 ? m - 2 : 2);
            const int d = m < 3 ? 0 : (m < 5 ? 1 : 2);
            const float a = u[c], b = v[d];
            u[c] = nc[m] * a + ns[m] * b;
            v[d] = -ns[m] * a + nc[m] * b;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            top[i * (ncol + 4) + tc] = u[i];
            if (col < ncol) damp[(int64_t)i * ncol + col] = v[i];
            else cd[i] = v[i];
        }
    }
}

}  // namespace

void launch_damp(Problem& p, bool undo_old, float lambda) {
    count_launches(p, 1);
    k_damp<<<ceil_div((int64_t)p.n_pt * 32, 128), 128, 0, p.stream>>>(
        p.n_pt, p.pt_off, p.a_off, p.tpool, p.apool, p.cpool, p.c_off, p.dl2, p.rot, sqrtf(lambda),
        undo_old ? 1 : 0);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
