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
// the new damping.
//
// In a batch of problems each landmark takes the damping of its problem.
//
// Layout of the work: a CTA takes DB landmarks.  Phase 1, one landmark per
// thread: undo/redo on the 3x3 landmark part and the new rotations.  Phase 2:
// the CTA's (landmark, column) pairs, flattened through a prefix sum over the
// landmarks' 9k + 1 columns, one pair per thread at a time, so that
// consecutive threads touch consecutive columns of the six rows.
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int DB = 128;  // landmarks (and threads) per CTA

__device__ __forceinline__ void rot_pair(int m, int& c, int& d) {
    c = m < 3 ? m : (m < 5 ? m - 2 : 2);
    d = m < 3 ? 0 : (m < 5 ? 1 : 2);
}

__global__ void __launch_bounds__(DB)
k_damp(int n_pt, const int32_t* __restrict__ pt_off, const int64_t* __restrict__ a_off,
       const int32_t* __restrict__ c_off, float* __restrict__ tpool, float* __restrict__ apool,
       float* __restrict__ cpool, const float* __restrict__ dl2, float* __restrict__ rot, float sqrt_lambda,
       const float* __restrict__ lam_prob, const int32_t* __restrict__ lm_prob, int undo) {
    __shared__ float s_rot[DB][24];  // old (12) and new (12) rotations
    __shared__ int s_off[DB + 1];    // prefix of the column counts 9k + 1
    __shared__ int s_k[DB];
    __shared__ int64_t s_top[DB], s_damp[DB];
    __shared__ int s_cd[DB];
    __shared__ int s_w[DB / 32];
    const int tid = threadIdx.x;
    const int j = blockIdx.x * DB + tid;
    int ncols = 0;
    if (j < n_pt) {
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        const int ncol = 9 * k, nr = 2 * k;
        const int64_t toff = top_offset(s0, j);
        float* top = tpool + toff;
        s_k[tid] = k;
        s_top[tid] = toff;
        s_damp[tid] = a_off[j] + (int64_t)(nr - 3) * ncol;
        s_cd[tid] = c_off[j] + (nr - 3);
        ncols = ncol + 1;
        float R[3][3], D[3][3];
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) {
                R[i][c] = top[i * (ncol + 4) + ncol + c];
                D[i][c] = 0.f;
            }
        float* rs = s_rot[tid];
        if (undo) {
            for (int m = 0; m < 12; ++m) rs[m] = rot[12 * (int64_t)j + m];
            for (int m = 5; m >= 0; --m) {
                int c, d;
                rot_pair(m, c, d);
                const float cs = rs[2 * m], sn = rs[2 * m + 1];
                for (int col = 0; col < 3; ++col) {
                    const float u = R[c][col], v = D[d][col];
                    R[c][col] = cs * u - sn * v;
                    D[d][col] = sn * u + cs * v;
                }
            }
            for (int i = 0; i < 3; ++i)
                for (int c = 0; c < 3; ++c) D[i][c] = 0.f;
        } else {
            for (int m = 0; m < 12; m += 2) {
                rs[m] = 1.f;
                rs[m + 1] = 0.f;
            }
        }
        const float sl = lam_prob ? sqrtf(lam_prob[lm_prob[j]]) : sqrt_lambda;
        for (int d = 0; d < 3; ++d) D[d][d] = sl * sqrtf(dl2[3 * j + d]);
        for (int m = 0; m < 6; ++m) {
            int c, d;
            rot_pair(m, c, d);
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
    // exclusive prefix of the column counts (block scan)
    {
        const int lane = tid & 31, w = tid >> 5;
        int inc = ncols;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_w[w] = inc;
        __syncthreads();
        int base = 0;
        for (int q = 0; q < w; ++q) base += s_w[q];
        s_off[tid] = base + inc - ncols;
        if (tid == DB - 1) s_off[DB] = base + inc;
        __syncthreads();
    }
    const int total = s_off[DB];
    int l = 0;
    for (int item = tid; item < total; item += DB) {
        while (s_off[l + 1] <= item) ++l;  // items are visited in increasing order
        const int col = item - s_off[l];
        const int ncol = 9 * s_k[l];
        float* top = tpool + s_top[l];
        const int tc = col < ncol ? col : ncol + 3;
        const float* rs = s_rot[l];
        float u[3], v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            u[i] = top[i * (ncol + 4) + tc];
            v[i] = 0.f;
        }
        if (undo) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
                v[i] = col < ncol ? apool[s_damp[l] + (int64_t)i * ncol + col] : cpool[s_cd[l] + i];
#pragma unroll
            for (int m = 5; m >= 0; --m) {
                int c, d;
                rot_pair(m, c, d);
                const float a = u[c], b = v[d];
                u[c] = rs[2 * m] * a - rs[2 * m + 1] * b;
                v[d] = rs[2 * m + 1] * a + rs[2 * m] * b;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            int c, d;
            rot_pair(m, c, d);
            const float a = u[c], b = v[d];
            u[c] = rs[12 + 2 * m] * a + rs[13 + 2 * m] * b;
            v[d] = -rs[13 + 2 * m] * a + rs[12 + 2 * m] * b;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            top[i * (ncol + 4) + tc] = u[i];
            if (col < ncol) apool[s_damp[l] + (int64_t)i * ncol + col] = v[i];
            else cpool[s_cd[l] + i] = v[i];
        }
    }
}

}  // namespace

void launch_damp(Problem& p, bool undo_old, float lambda) {
    count_launches(p, 1);
    k_damp<<<ceil_div(p.n_pt, DB), DB, 0, p.stream>>>(p.n_pt, p.pt_off, p.a_off, p.c_off, p.tpool, p.apool, p.cpool,
                                                      p.dl2, p.rot, sqrtf(lambda), p.batch.lam, p.batch.lm_prob,
                                                      undo_old ? 1 : 0);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
