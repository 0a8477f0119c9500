// K2: landmark damping folded into the marginalised landmark blocks with six
// Givens rotations (Sec. 5.3, Fig. 3).
//
// The three damping rows [0 | sqrt(lambda) D_l | 0] are attached below the
// block (they are the last three rows of A_j); rotation m acts on the pair
// (R1 row c, damping row d) for (d, c) = (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
// and zeroes the damping row's entry in landmark column c:
//     rho = sqrt(a^2 + b^2), cos = a / rho, sin = b / rho  (a = pivot, b = damping entry)
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
// one warp per landmark, lanes over its 9k + 1 columns, so that consecutive
// lanes touch consecutive columns of the six rows; 8 warps per CTA keep many
// landmarks' loads in flight per SM (the kernel is latency-bound otherwise).
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int DB = 64;   // landmarks per CTA (phase 1: one thread each)
constexpr int DT = 256;  // threads per CTA (phase 2: 8 warps, DB / 8 landmarks each)


__global__ void __launch_bounds__(DT)
k_damp(int n_pt, const int32_t* __restrict__ pt_off, const int64_t* __restrict__ a_off,
       const int32_t* __restrict__ c_off, float* __restrict__ tpool, float* __restrict__ apool,
       float* __restrict__ cpool, const float* __restrict__ dl2, float* __restrict__ rot, float sqrt_lambda,
       const float* __restrict__ lam_prob, const int32_t* __restrict__ lm_prob, int undo_all,
       const BatchLm* __restrict__ blm) {
    __shared__ float s_rot[DB][24];  // old (12) and new (12) rotations
    __shared__ int s_k[DB];          // k, or -1: a stopped problem's landmark (skipped)
    __shared__ int s_undo[DB];
    __shared__ int64_t s_top[DB], s_damp[DB];
    __shared__ int s_cd[DB];
    const int tid = threadIdx.x;
    const int j = blockIdx.x * DB + tid;
    if (tid < DB && j < n_pt && blm && !batch_active(blm, lm_prob[j])) {
        s_k[tid] = -1;
    } else if (tid < DB && j < n_pt) {
        // a batch undoes the damping of the problems that kept their linearisation
        const int undo = blm ? (batch_relin(blm, lm_prob[j]) ? 0 : 1) : undo_all;
        s_undo[tid] = undo;
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        const int ncol = 9 * k, nr = 2 * k;
        const int64_t toff = top_offset(s0, j);
        float* top = tpool + toff;
        s_k[tid] = k;
        s_top[tid] = toff;
        s_damp[tid] = a_off[j] + (int64_t)(nr - 3) * ncol;
        s_cd[tid] = c_off[j] + (nr - 3);
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
                givens_pair(m, c, d);
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
            givens_pair(m, c, d);
            const float a = R[c][c], b = D[d][c];
            const float r2 = a * a + b * b;
            float cs = 1.f, sn = 0.f;
            if (r2 > 0.f) {
                const float inv = rsqrtf(r2);
                cs = a * inv;
                sn = b * inv;
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
    __syncthreads();
    // Phase 2, one warp per landmark: lanes over the 9k + 1 columns of the
    // six rows (three top rows, three damping rows; coalesced row segments)
    const int lane = tid & 31, w = tid >> 5;
    for (int l = w; l < DB; l += DT / 32) {
        if (blockIdx.x * DB + l >= n_pt) break;
        if (s_k[l] < 0) continue;
        const int undo = s_undo[l];
        const int ncol = 9 * s_k[l];
        float* __restrict__ top = tpool + s_top[l];
        float* __restrict__ dmp = apool + s_damp[l];
        float* __restrict__ cdm = cpool + s_cd[l];
        float ro[12], rn[12];
#pragma unroll
        for (int m = 0; m < 12; ++m) {
            ro[m] = s_rot[l][m];
            rn[m] = s_rot[l][12 + m];
        }
        // two columns per lane and step, loads of both issued first (the
        // kernel is bound by the latency of these loads)
        for (int col0 = lane; col0 <= ncol; col0 += 64) {
            float u[2][3], v[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = col0 + 32 * h;
                const int tc = col < ncol ? col : ncol + 3;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    u[h][i] = col <= ncol ? top[i * (ncol + 4) + tc] : 0.f;
                    v[h][i] = (undo && col <= ncol) ? (col < ncol ? dmp[(int64_t)i * ncol + col] : cdm[i]) : 0.f;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (undo) {
#pragma unroll
                    for (int m = 5; m >= 0; --m) {
                        int c, d;
                        givens_pair(m, c, d);
                        const float a = u[h][c], b = v[h][d];
                        u[h][c] = ro[2 * m] * a - ro[2 * m + 1] * b;
                        v[h][d] = ro[2 * m + 1] * a + ro[2 * m] * b;
                    }
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) v[h][i] = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    int c, d;
                    givens_pair(m, c, d);
                    const float a = u[h][c], b = v[h][d];
                    u[h][c] = rn[2 * m] * a + rn[2 * m + 1] * b;
                    v[h][d] = -rn[2 * m + 1] * a + rn[2 * m] * b;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = col0 + 32 * h;
                if (col > ncol) continue;
                const int tc = col < ncol ? col : ncol + 3;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    top[i * (ncol + 4) + tc] = u[h][i];
                    if (col < ncol) dmp[(int64_t)i * ncol + col] = v[h][i];
                    else cdm[i] = v[h][i];
                }
            }
        }
    }
}

// The implicit storage keeps no top rows; its landmark record holds the
// undamped R1, Q1^T r = t and P (K1).  One lane per landmark (storage
// position) computes the same six rotations from R1 and sqrt(lambda) D_l,
// applies them also to [I; 0] (the map from the undamped top rows to the six
// rotated rows, G[:, 0:3] = [G_tt; G_dt]), and stores S = G_dt^T G_dt, G_tt,
// G_tt P, G_tt t and the damped R.  No undo is needed: every call starts from
// the undamped R1.  A warp takes 32 consecutive 256-byte records: their input
// fields (floats 40..63) are loaded and their outputs (floats 6..39) stored
// cooperatively through shared memory, so that consecutive lanes touch
// consecutive 16-byte words instead of one word per record each.
constexpr int DI_WARPS = 4;
constexpr int DI_OUT = 37;  // shared floats per record for floats 6..39 (odd stride)

__global__ void __launch_bounds__(32 * DI_WARPS)
k_damp_implicit(int n_pt, float* __restrict__ lmrec, float sqrt_lambda, const int32_t* __restrict__ lm_by_k,
                const float* __restrict__ lam_prob, const int32_t* __restrict__ lm_prob,
                const BatchLm* __restrict__ blm) {
    __shared__ float4 sin[DI_WARPS][32 * 6];
    __shared__ float sout[DI_WARPS][32 * DI_OUT];
    __shared__ int sact[DI_WARPS][32];
    static_assert(LR_R1 == 40 && LR_DL2 == 46 && LR_T == 49 && LR_P == 52, "input fields: float4s 10..15");
    static_assert(LR_S == 6 && LR_GP == 12 && LR_GT == 21 && LR_G == 24 && LR_RD == 33, "outputs: floats 6..39");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pos0 = (blockIdx.x * DI_WARPS + w) * 32;
    if (pos0 >= n_pt) return;  // whole warp
    const int nrec = min(32, n_pt - pos0);
    float4* L4 = reinterpret_cast<float4*>(lmrec + (int64_t)LM_REC * pos0);
    for (int q = lane; q < nrec * 6; q += 32) {
        const int r = q / 6;
        sin[w][q] = L4[16 * r + 10 + (q - 6 * r)];
    }
    const int pos = pos0 + lane;
    const bool act = lane < nrec && (!blm || batch_active(blm, lm_prob[lm_by_k[pos]]));
    sact[w][lane] = act ? 1 : 0;
    __syncwarp();
    if (act) {
        const float4* in = &sin[w][6 * lane];
        const float4 q0 = in[0], q1 = in[1], q2 = in[2], p0 = in[3], p1 = in[4], p2 = in[5];
        float R[3][3] = {{q0.x, q0.y, q0.z}, {0.f, q0.w, q1.x}, {0.f, 0.f, q1.y}};
        const float dl2[3] = {q1.z, q1.w, q2.x};
        const float t[3] = {q2.y, q2.z, q2.w};
        const float P[3][3] = {{p0.x, p0.y, p0.z}, {p0.w, p1.x, p1.y}, {p1.z, p1.w, p2.x}};
        float D[3][3], E[6][3];
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) {
                D[i][c] = 0.f;
                E[i][c] = i == c ? 1.f : 0.f;
                E[3 + i][c] = 0.f;
            }
        const float sl = lam_prob ? sqrtf(lam_prob[lm_prob[lm_by_k[pos]]]) : sqrt_lambda;
        for (int d = 0; d < 3; ++d) D[d][d] = sl * sqrtf(dl2[d]);
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            int c, d;
            givens_pair(m, c, d);
            const float a = R[c][c], b = D[d][c];
            const float r2 = a * a + b * b;
            float cs = 1.f, sn = 0.f;
            if (r2 > 0.f) {
                const float inv = rsqrtf(r2);
                cs = a * inv;
                sn = b * inv;
            }
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                if (col < c) continue;
                const float u = R[c][col], v = D[d][col];
                R[c][col] = cs * u + sn * v;
                D[d][col] = -sn * u + cs * v;
            }
            D[d][c] = 0.f;
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                const float u = E[c][col], v = E[3 + d][col];
                E[c][col] = cs * u + sn * v;
                E[3 + d][col] = -sn * u + cs * v;
            }
        }
        // floats 6..39 of the record: S (6), G_tt P (9), G_tt t (3), G_tt (9), damped R (6), pad
        float* o = &sout[w][DI_OUT * lane];
        int q = 0;
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = u; v < 3; ++v) o[q++] = E[3][u] * E[3][v] + E[4][u] * E[4][v] + E[5][u] * E[5][v];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int b = 0; b < 3; ++b) o[6 + 3 * i + b] = E[i][0] * P[0][b] + E[i][1] * P[1][b] + E[i][2] * P[2][b];
#pragma unroll
        for (int i = 0; i < 3; ++i) o[15 + i] = E[i][0] * t[0] + E[i][1] * t[1] + E[i][2] * t[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) o[18 + 3 * i + c] = E[i][c];
        o[27] = R[0][0];
        o[28] = R[0][1];
        o[29] = R[0][2];
        o[30] = R[1][1];
        o[31] = R[1][2];
        o[32] = R[2][2];
        o[33] = 0.f;
    }
    __syncwarp();
    // floats 8..39 as 8 float4 per record, floats 6..7 as one float2
    for (int q = lane; q < nrec * 8; q += 32) {
        const int r = q >> 3, m = q & 7;
        if (!sact[w][r]) continue;
        const float* o = &sout[w][DI_OUT * r + 2 + 4 * m];
        L4[16 * r + 2 + m] = make_float4(o[0], o[1], o[2], o[3]);
    }
    if (act)
        *reinterpret_cast<float2*>(lmrec + (int64_t)LM_REC * pos + LR_S) =
            make_float2(sout[w][DI_OUT * lane], sout[w][DI_OUT * lane + 1]);
}

}  // namespace

void launch_damp(Problem& p, bool undo_old, float lambda) {
    if (p.schur) {  // the explicit Schur complement is re-formed at every damping
        launch_schur_assemble(p, lambda);
        return;
    }
    count_launches(p, 1);
    if (p.implicit) {
        k_damp_implicit<<<ceil_div(p.n_pt, 32 * DI_WARPS), 32 * DI_WARPS, 0, p.stream>>>(
            p.n_pt, p.lmrec, sqrtf(lambda), p.lm_by_k, p.batch.lam, p.batch.lm_prob,
            p.batch.n_prob > 0 ? p.batch.lm : nullptr);
        BA_LAUNCH_CHECK();
        return;
    }
    k_damp<<<ceil_div(p.n_pt, DB), DT, 0, p.stream>>>(p.n_pt, p.pt_off, p.a_off, p.c_off, p.tpool, p.apool, p.cpool,
                                                      p.dl2, p.rot, sqrtf(lambda), p.batch.lam, p.batch.lm_prob,
                                                      undo_old ? 1 : 0, p.batch.n_prob > 0 ? p.batch.lm : nullptr);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
