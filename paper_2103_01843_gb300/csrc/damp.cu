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
// undamped R1, Q1^T r = t and P (K1).  One thread per landmark (storage
// position) computes the same six rotations from R1 and sqrt(lambda) D_l,
// applies them also to [I; 0] (the map from the undamped top rows to the six
// rotated rows, G[:, 0:3] = [G_tt; G_dt]), and stores S = G_dt^T G_dt, G_tt,
// G_tt P, G_tt t and the damped R.  No undo is needed: every call starts from
// the undamped R1.
__global__ void __launch_bounds__(128)
k_damp_implicit(int n_pt, float* __restrict__ lmrec, float sqrt_lambda, const int32_t* __restrict__ lm_by_k,
                const float* __restrict__ lam_prob, const int32_t* __restrict__ lm_prob,
                const BatchLm* __restrict__ blm) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n_pt) return;
    if (blm && !batch_active(blm, lm_prob[lm_by_k[pos]])) return;
    float* L = lmrec + (int64_t)LM_REC * pos;
    // R1 (upper), D_l^2, t and P from the landmark record (K1), 16-byte loads
    static_assert(LR_DL2 == LR_R1 + 6 && LR_T == LR_R1 + 9 && LR_P == LR_R1 + 12 && LR_R1 % 4 == 0, "record");
    const float4 q0 = *reinterpret_cast<const float4*>(L + LR_R1), q1 = *reinterpret_cast<const float4*>(L + LR_R1 + 4),
                 q2 = *reinterpret_cast<const float4*>(L + LR_R1 + 8), p0 = *reinterpret_cast<const float4*>(L + LR_P),
                 p1 = *reinterpret_cast<const float4*>(L + LR_P + 4);
    const float p8 = L[LR_P + 8];
    float R[3][3] = {{q0.x, q0.y, q0.z}, {0.f, q0.w, q1.x}, {0.f, 0.f, q1.y}};
    const float dl2[3] = {q1.z, q1.w, q2.x};
    const float t[3] = {q2.y, q2.z, q2.w};
    const float P[3][3] = {{p0.x, p0.y, p0.z}, {p0.w, p1.x, p1.y}, {p1.z, p1.w, p8}};
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
    // S = G_dt^T G_dt (upper: 00 01 02 11 12 22), G_tt P, G_tt t, G_tt, damped R
    // (upper): 16-byte stores
    float S[6], GP[9], Gt[3];
    int q = 0;
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = u; v < 3; ++v) S[q++] = E[3][u] * E[3][v] + E[4][u] * E[4][v] + E[5][u] * E[5][v];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Gt[i] = E[i][0] * t[0] + E[i][1] * t[1] + E[i][2] * t[2];
#pragma unroll
        for (int b = 0; b < 3; ++b) GP[3 * i + b] = E[i][0] * P[0][b] + E[i][1] * P[1][b] + E[i][2] * P[2][b];
    }
    static_assert(LR_S == 6 && LR_GP == 12 && LR_GT == 21 && LR_G == 24 && LR_RD == 33, "record");
    *reinterpret_cast<float2*>(L + 6) = make_float2(S[0], S[1]);
    *reinterpret_cast<float4*>(L + 8) = make_float4(S[2], S[3], S[4], S[5]);
    *reinterpret_cast<float4*>(L + 12) = make_float4(GP[0], GP[1], GP[2], GP[3]);
    *reinterpret_cast<float4*>(L + 16) = make_float4(GP[4], GP[5], GP[6], GP[7]);
    *reinterpret_cast<float4*>(L + 20) = make_float4(GP[8], Gt[0], Gt[1], Gt[2]);
    *reinterpret_cast<float4*>(L + 24) = make_float4(E[0][0], E[0][1], E[0][2], E[1][0]);
    *reinterpret_cast<float4*>(L + 28) = make_float4(E[1][1], E[1][2], E[2][0], E[2][1]);
    *reinterpret_cast<float4*>(L + 32) = make_float4(E[2][2], R[0][0], R[0][1], R[0][2]);
    *reinterpret_cast<float4*>(L + 36) = make_float4(R[1][1], R[1][2], R[2][2], 0.f);
}

}  // namespace

void launch_damp(Problem& p, bool undo_old, float lambda) {
    if (p.schur) {  // the explicit Schur complement is re-formed at every damping
        launch_schur_assemble(p, lambda);
        return;
    }
    count_launches(p, 1);
    if (p.implicit) {
        k_damp_implicit<<<ceil_div(p.n_pt, 128), 128, 0, p.stream>>>(
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
