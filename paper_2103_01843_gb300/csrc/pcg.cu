// K3-K5: block-Jacobi preconditioned CG on the reduced camera system
// (Sec. 5.4, Eq. cg_mult, Sec. 6.1), working only on the stored landmark
// blocks A_j = Q2^T J_p (2k x 9k, the last three rows being the rotated
// landmark-damping rows) and c_j = Q2^T r.
//
//   K3  M_i = sum_j A_ji^T A_ji + lambda D_p,i^2,  g_i = -sum_j A_ji^T c_j,
//       Cholesky-inverted per camera (the block diagonal of H~, Sec. 6.1):
//       by default each term from the Gram identity (below) per chunk of a
//       camera's observations; optionally from per-observation records of
//       the tile pipeline (matvec.cu); summed per camera in a fixed order
//   K4  y = sum_j P_j^T A_j^T (A_j P_j v) (matvec.cu) + lambda D_p^2 v, the pose
//       damping added only in the product (Sec. 5.3), inside K5
//   K5  the CG recursion with the Nash-Sofer stop
//       i (Q_i - Q_{i-1}) / Q_i < eta, Q(x) = 1/2 x^T H~ x - g^T x = -1/2 x^T (g + r).
#include <algorithm>

#include "camera.cuh"
#include "precond.cuh"
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int PC_WARPS = 16;
constexpr int REC_SUMS = 54;  // upper triangle of a 9 x 9 block (45) and a 9-vector

// ---------------------------------------------------------------------------
// K3: per-camera preconditioner block and right-hand side
// ---------------------------------------------------------------------------
// from per-observation records (56 floats apart): a warp reads two records
// at a time, lanes 0-13 and 16-29 one float4 each, four record pairs in
// flight per warp; the camera's records are summed in a fixed order
__global__ void __launch_bounds__(32 * PC_WARPS)
k_precond_reduce(int n_cam, const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list_st,
                 const float* __restrict__ rec, const float* __restrict__ dp2, float lam,
                 const float* __restrict__ lam_prob, const int32_t* __restrict__ cam_prob,
                 float* __restrict__ mdiag, float* __restrict__ minv, float* __restrict__ g, uint32_t* err) {
    constexpr int U = 4;
    __shared__ float4 part[2 * PC_WARPS][14];
    __shared__ float tot[56], sM[81], sL[81];
    const int cam = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int half = lane >> 4, q = lane & 15;
    float4 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < 14) {
        const int e0 = cam_off[cam], e1 = cam_off[cam + 1];
        const float4* r4 = reinterpret_cast<const float4*>(rec) + q;
        for (int e = e0 + 2 * w + half; e < e1; e += 2 * PC_WARPS * U) {
            int st[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int eu = e + 2 * PC_WARPS * u;
                st[u] = eu < e1 ? __ldg(cam_list_st + eu) : -1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (st[u] >= 0) {
                    const float4 r = __ldg(r4 + (int64_t)st[u] * 14);
                    acc[u].x += r.x;
                    acc[u].y += r.y;
                    acc[u].z += r.z;
                    acc[u].w += r.w;
                }
            }
        }
#pragma unroll
        for (int u = 1; u < U; ++u) {
            acc[0].x += acc[u].x;
            acc[0].y += acc[u].y;
            acc[0].z += acc[u].z;
            acc[0].w += acc[u].w;
        }
        part[2 * w + half][q] = acc[0];
    }
    __syncthreads();
    if (threadIdx.x < 14) {
        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m = 0; m < 2 * PC_WARPS; ++m) {
            const float4 t = part[m][threadIdx.x];
            s4.x += t.x;
            s4.y += t.y;
            s4.z += t.z;
            s4.w += t.w;
        }
        tot[4 * threadIdx.x] = s4.x;
        tot[4 * threadIdx.x + 1] = s4.y;
        tot[4 * threadIdx.x + 2] = s4.z;
        tot[4 * threadIdx.x + 3] = s4.w;
    }
    __syncthreads();
    if (lam_prob) lam = lam_prob[cam_prob[cam]];
    if (w == 0) precond_finish_warp(cam, tot, dp2, lam, mdiag, minv, g, err, sM, sL, lane);
}

// K3 in Gram form.  The orthogonal transforms of K1 and K2 preserve the Gram
// matrix of the pose and residual columns of a landmark block (the damping
// rows have zero pose and residual entries), so for observation s of
// landmark j
//   (A_j^T A_j)_ss = J_s^T J_s - T_s^T T_s,   (A_j^T c_j)_s = J_s^T r_s - T_s^T t,
// with J_s, r_s the observation's two Jacobian rows and residuals (recomputed
// here) and T_s, t the camera's 3 x 9 slice and the residual column of the
// landmark's damped top rows [Q1^T J_p | R1 | Q1^T r]: 30 floats read per
// observation instead of the 18 k floats of its columns of A_j.  The implicit
// storage keeps no top rows: there T_s = C_s J_s with the 3 x 2 matrix
// C_s = G_tt D'_s - (G_tt P) V_s^T (V_s the observation's two Householder
// rows, 8 floats read; G_tt P and G_tt t from the landmark record, 12 floats,
// G_tt too for the slots 0 and 1, whose D'_s is non-zero), and the two sums
// become J_s^T (I - C_s^T C_s) J_s and J_s^T (r_s - C_s^T G_tt t).
// First pass: one CTA per chunk of up to PG_CHUNK observations of one camera
// (threads over the observations, each summing its own in order, then a
// fixed-order CTA reduction) writes the chunk's 54 partial sums.
constexpr int PG_T = 128;
template <bool IMPLICIT>
__global__ void __launch_bounds__(PG_T)
k_precond_gram(const int32_t* __restrict__ chunk_cam, const int32_t* __restrict__ chunk_off,
               const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list,
               const int32_t* __restrict__ obs_pt_s, const float2* __restrict__ obs_xy_s,
               const int32_t* __restrict__ pt_off, const float* __restrict__ frames, const float* __restrict__ pts,
               const float* __restrict__ tpool, float* __restrict__ part_out, const float* __restrict__ lmrec,
               const int32_t* __restrict__ lm_pos, const int32_t* __restrict__ c_off,
               const float4* __restrict__ ipool, int64_t n_obs, const int4* __restrict__ k3rec,
               const float2* __restrict__ k3xy, float huber, const BatchLm* __restrict__ blm,
               const int32_t* __restrict__ cam_prob) {
    __shared__ float part[PG_T / 32][REC_SUMS + 1];
    const int ch = blockIdx.x, cam = chunk_cam[ch];
    if (blm && !batch_active(blm, cam_prob[cam])) return;  // a stopped problem of a batch
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e0 = cam_off[cam] + (ch - chunk_off[cam]) * PG_CHUNK;
    const int e1 = min(cam_off[cam + 1], e0 + PG_CHUNK);
    float acc[REC_SUMS + 1];  // + sum of ||J_s||_F^2 (the cancellation guard of the finish)
#pragma unroll
    for (int q = 0; q <= REC_SUMS; ++q) acc[q] = 0.f;
    const float* fr = frames + FRAME * cam;  // global (load_frame reads it with __ldg)
    for (int e = e0 + threadIdx.x; e < e1; e += PG_T) {
        int s = 0, j, s0 = 0, k = 0;
        float2 z;
        int4 rec = make_int4(0, 0, 0, 0);
        if constexpr (IMPLICIT) {  // the camera-ordered record: landmark, storage index, position | slot
            rec = __ldg(k3rec + e);
            z = __ldg(k3xy + e);
            j = rec.x;
        } else {
            s = cam_list[e];
            j = obs_pt_s[s];
            s0 = pt_off[j];
            k = pt_off[j + 1] - s0;
            z = obs_xy_s[s];
        }
        float r[2], Jp[18], Jl[6];
        frame_jacobians(fr, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r, Jp, Jl);
        huber_scale_rows(huber, r, Jp, Jl);  // the rows K1 factored
#pragma unroll
        for (int u = 0; u < 18; ++u) acc[REC_SUMS] += Jp[u] * Jp[u];
        if constexpr (IMPLICIT) {
            // T_s = C J_s with C = G_tt D'_s - (G_tt P) V_s^T (3 x 2; D'_s picks
            // J_s's rows 0, 1 into top rows 0, 1 for slot 0, row 0 into top row 2
            // for slot 1), so J_s^T J_s - T_s^T T_s = J_s^T W J_s, W = I - C^T C,
            // and J_s^T r_s - T_s^T t = J_s^T (r_s - C^T G_tt t)
            const int slot = (int)((unsigned)rec.z >> 30);     // 0, 1 or 2 (>= 2)
            const int64_t so = (int64_t)(unsigned)rec.y;
            const int pos = rec.z & 0x3fffffff;
            const float4 c4 = __ldg(ipool + 4 * n_obs + so), c5 = __ldg(ipool + 5 * n_obs + so);
            const float va[3] = {c4.z, c4.w, c5.x}, vb[3] = {c5.y, c5.z, c5.w};  // V rows 2 slot, 2 slot + 1
            const float4* Lr = reinterpret_cast<const float4*>(lmrec + (int64_t)LM_REC * pos);
            static_assert(LR_GP == 12 && LR_GT == 21 && LR_G == 24, "record");
            const float4 g0 = __ldg(Lr + 3), g1 = __ldg(Lr + 4), g2 = __ldg(Lr + 5);
            const float GP[9] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g2.x};
            const float Gt[3] = {g2.y, g2.z, g2.w};
            float C[3][2];
#pragma unroll
            for (int row = 0; row < 3; ++row) {
                C[row][0] = -(GP[3 * row] * va[0] + GP[3 * row + 1] * va[1] + GP[3 * row + 2] * va[2]);
                C[row][1] = -(GP[3 * row] * vb[0] + GP[3 * row + 1] * vb[1] + GP[3 * row + 2] * vb[2]);
            }
            if (slot < 2) {
                const float4 h0 = __ldg(Lr + 6), h1 = __ldg(Lr + 7), h2 = __ldg(Lr + 8);
                const float G[9] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w, h2.x};
#pragma unroll
                for (int row = 0; row < 3; ++row) {
                    C[row][0] += slot == 0 ? G[3 * row] : G[3 * row + 2];
                    C[row][1] += slot == 0 ? G[3 * row + 1] : 0.f;
                }
            }
            const float w00 = 1.f - (C[0][0] * C[0][0] + C[1][0] * C[1][0] + C[2][0] * C[2][0]);
            const float w01 = -(C[0][0] * C[0][1] + C[1][0] * C[1][1] + C[2][0] * C[2][1]);
            const float w11 = 1.f - (C[0][1] * C[0][1] + C[1][1] * C[1][1] + C[2][1] * C[2][1]);
            const float q0 = r[0] - (C[0][0] * Gt[0] + C[1][0] * Gt[1] + C[2][0] * Gt[2]);
            const float q1 = r[1] - (C[0][1] * Gt[0] + C[1][1] * Gt[1] + C[2][1] * Gt[2]);
            float y0[9], y1[9];  // W J_s
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                y0[c] = w00 * Jp[c] + w01 * Jp[9 + c];
                y1[c] = w01 * Jp[c] + w11 * Jp[9 + c];
            }
            int q = 0;
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                acc[45 + u] += Jp[u] * q0 + Jp[9 + u] * q1;
#pragma unroll
                for (int v = u; v < 9; ++v) acc[q++] += Jp[u] * y0[v] + Jp[9 + u] * y1[v];
            }
        } else {
            int q = 0;
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                acc[45 + u] += Jp[u] * r[0] + Jp[9 + u] * r[1];
#pragma unroll
                for (int v = u; v < 9; ++v) acc[q++] += Jp[u] * Jp[v] + Jp[9 + u] * Jp[9 + v];
            }
            // the camera's 3 x 9 slice of the damped top rows and the residual column
            const int stride = 9 * k + 4;
            const float* top = tpool + top_offset(s0, j) + 9 * (s - s0);
#pragma unroll
            for (int row = 0; row < 3; ++row) {
                float T[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) T[c] = __ldg(top + row * stride + c);
                const float t = __ldg(top + row * stride + 9 * (k - (s - s0)) + 3);
                q = 0;
#pragma unroll
                for (int u = 0; u < 9; ++u) {
                    acc[45 + u] -= T[u] * t;
#pragma unroll
                    for (int v = u; v < 9; ++v) acc[q++] -= T[u] * T[v];
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q <= REC_SUMS; ++q) {
        const float v = warp_sum(acc[q]);
        if (lane == 0) part[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x <= REC_SUMS) {
        float v = 0.f;
#pragma unroll
        for (int m = 0; m < PG_T / 32; ++m) v += part[m][threadIdx.x];
        part_out[56LL * ch + threadIdx.x] = v;
    }
}

// The camera-ordered record of every observation (entry e of the camera
// lists) for the implicit K3: landmark, storage index, landmark storage
// position with the slot (0, 1, or 2 for any later slot) in its top two bits,
// and the measurement.  Static per problem (built at create).
__global__ void k_k3_records(int64_t n_obs, const int32_t* __restrict__ cam_list, const int32_t* __restrict__ obs_pt_s,
                             const int32_t* __restrict__ pt_off, const int32_t* __restrict__ c_off,
                             const int32_t* __restrict__ lm_pos, const float2* __restrict__ obs_xy_s,
                             int4* __restrict__ rec, float2* __restrict__ xy) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_obs; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = cam_list[e];
        const int j = obs_pt_s[s];
        const int slot = s - pt_off[j];
        const int so = (c_off[j] >> 1) + slot;
        rec[e] = make_int4(j, so, (int)((unsigned)lm_pos[j] | ((unsigned)min(slot, 2) << 30)), 0);
        xy[e] = obs_xy_s[s];
    }
}

// The Gram form's FP32 error is about eps * sum_s ||J_s||_F^2 per block, while
// a block's size is about tr(M_i): where the landmark elimination removes
// most of a camera's Jacobian energy (a point very close to the camera, or
// seen from nearly one centre) the subtraction cancels.  Above this ratio
// (error bound ~1e-5 relative) the camera's sums come from the stored
// square-root blocks instead; synthetic scenes of every shape tested stay
// below 10, a landmark at 0.08 m depth reaches ~900.
constexpr float GRAM_KAPPA_MAX = 64.f;

// The 54 sums of one camera taken from the stored blocks, one warp: for each
// of its observations s (landmark j, slot q), (A_j^T A_j)_ss and (A_j^T c_j)_s
// over all 2k rows of A_j (including the rotated damping rows), lanes over
// the rows, then a fixed-order warp reduction.
__device__ void exact_sums_warp(int cam, const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list,
                                const int32_t* __restrict__ obs_pt_s, const int32_t* __restrict__ pt_off,
                                const int64_t* __restrict__ a_off, const int32_t* __restrict__ c_off,
                                const float* __restrict__ apool, const float* __restrict__ cpool, float* tot,
                                int lane) {
    float acc[REC_SUMS];
#pragma unroll
    for (int q = 0; q < REC_SUMS; ++q) acc[q] = 0.f;
    for (int e = cam_off[cam]; e < cam_off[cam + 1]; ++e) {
        const int s = cam_list[e];
        const int j = obs_pt_s[s];
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        const int64_t nc = 9LL * k;
        const float* A = apool + a_off[j] + 9 * (s - s0);
        const float* c = cpool + c_off[j];
        for (int r = lane; r < 2 * k; r += 32) {
            float a[9];
#pragma unroll
            for (int u = 0; u < 9; ++u) a[u] = __ldg(A + r * nc + u);
            const float cr = __ldg(c + r);
            int q = 0;
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                acc[45 + u] += a[u] * cr;
#pragma unroll
                for (int v = u; v < 9; ++v) acc[q++] += a[u] * a[v];
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < REC_SUMS; ++q) {
        const float v = warp_sum(acc[q]);
        if (lane == 0) tot[q] = v;
    }
    __syncwarp();
}

// The 54 sums of one camera in the implicit storage, one warp: for each of
// its observations s (landmark j, slot q) the columns of A_j for s are formed
// from the stored factorisation, x_c = Q^T e_c restricted to the landmark's
// rows with e_c = J_p column c (two non-zeros, rows 2q, 2q+1):
// x_c[i] = J_p[i][c] - V_i . t_c with t_c = Tm^T (V^T J_p[:, c]), and
// c_j[i] = r_i - V_i . Tm^T (V^T r); rows >= 3 enter with weight one, the
// top rows through S (the damping rows keep G_dt times the top entries).
__device__ void exact_sums_warp_implicit(int cam, const int32_t* __restrict__ cam_off,
                                         const int32_t* __restrict__ cam_list, const int32_t* __restrict__ obs_pt_s,
                                         const int32_t* __restrict__ pt_off, const int32_t* __restrict__ c_off,
                                         const int32_t* __restrict__ lm_pos, const float4* __restrict__ ipool,
                                         int64_t n_obs, const float* __restrict__ rpool,
                                         const float* __restrict__ lmrec, float* tot, int lane) {
    auto rec = [&](int64_t so, float (&f)[24]) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float4 c = __ldg(ipool + m * n_obs + so);
            f[4 * m] = c.x;
            f[4 * m + 1] = c.y;
            f[4 * m + 2] = c.z;
            f[4 * m + 3] = c.w;
        }
    };
    float acc[REC_SUMS];
#pragma unroll
    for (int q = 0; q < REC_SUMS; ++q) acc[q] = 0.f;
    for (int e = cam_off[cam]; e < cam_off[cam + 1]; ++e) {
        const int s = cam_list[e];
        const int j = obs_pt_s[s];
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0, qs = s - s0;
        const int64_t so0 = c_off[j] >> 1;
        const float* L = lmrec + (int64_t)LM_REC * lm_pos[j];
        const float T00 = L[0], T01 = L[1], T02 = L[2], T11 = L[3], T12 = L[4], T22 = L[5];
        const float S[3][3] = {{L[6], L[7], L[8]}, {L[7], L[9], L[10]}, {L[8], L[10], L[11]}};
        float fq[24];
        rec(so0 + qs, fq);
        float tc[9][3];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float a0 = fq[18] * fq[c] + fq[21] * fq[9 + c];
            const float a1 = fq[19] * fq[c] + fq[22] * fq[9 + c];
            const float a2 = fq[20] * fq[c] + fq[23] * fq[9 + c];
            tc[c][0] = T00 * a0;
            tc[c][1] = T01 * a0 + T11 * a1;
            tc[c][2] = T02 * a0 + T12 * a1 + T22 * a2;
        }
        float p0 = 0.f, p1 = 0.f, p2 = 0.f;
        for (int t = lane; t < k; t += 32) {
            float f[24];
            rec(so0 + t, f);
            const float r0 = __ldg(rpool + 2 * (so0 + t)), r1 = __ldg(rpool + 2 * (so0 + t) + 1);
            p0 += f[18] * r0 + f[21] * r1;
            p1 += f[19] * r0 + f[22] * r1;
            p2 += f[20] * r0 + f[23] * r1;
        }
        p0 = warp_sum(p0);
        p1 = warp_sum(p1);
        p2 = warp_sum(p2);
        const float h0 = T00 * p0, h1 = T01 * p0 + T11 * p1, h2 = T02 * p0 + T12 * p1 + T22 * p2;
        float xt[2][10];  // this lane's top rows (lane 0: rows 0, 1; lane 1: row 2), columns and c
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int c = 0; c < 10; ++c) xt[rr][c] = 0.f;
        for (int t = lane; t < k; t += 32) {
            float f[24];
            rec(so0 + t, f);
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const float v0 = f[18 + 3 * rr], v1 = f[19 + 3 * rr], v2 = f[20 + 3 * rr];
                const float ci = __ldg(rpool + 2 * (so0 + t) + rr) - (v0 * h0 + v1 * h1 + v2 * h2);
                float x[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    x[c] = (t == qs ? fq[9 * rr + c] : 0.f) - (v0 * tc[c][0] + v1 * tc[c][1] + v2 * tc[c][2]);
                }
                const int i = 2 * t + rr;
                if (i >= 3) {
                    int q = 0;
#pragma unroll
                    for (int u = 0; u < 9; ++u) {
                        acc[45 + u] += x[u] * ci;
#pragma unroll
                        for (int v = u; v < 9; ++v) acc[q++] += x[u] * x[v];
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 9; ++c) xt[rr][c] = x[c];
                    xt[rr][9] = ci;
                }
            }
        }
        // the top rows through S, on lane 0 (row 2 comes from lane 1)
        float row2[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) row2[c] = __shfl_sync(0xffffffffu, xt[0][c], 1);
        if (lane == 0) {
            float X[3][10];
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                X[0][c] = xt[0][c];
                X[1][c] = xt[1][c];
                X[2][c] = row2[c];
            }
            float SX[3][10];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 10; ++c) SX[a][c] = S[a][0] * X[0][c] + S[a][1] * X[1][c] + S[a][2] * X[2][c];
            int q = 0;
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                acc[45 + u] += X[0][u] * SX[0][9] + X[1][u] * SX[1][9] + X[2][u] * SX[2][9];
#pragma unroll
                for (int v = u; v < 9; ++v) acc[q++] += X[0][u] * SX[0][v] + X[1][u] * SX[1][v] + X[2][u] * SX[2][v];
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < REC_SUMS; ++q) {
        const float v = warp_sum(acc[q]);
        if (lane == 0) tot[q] = v;
    }
    __syncwarp();
}

// The CG start folded into the finish (a single problem without the learned
// correction): each camera's warp writes x = 0, r = g, q = 0 and p = z = M^-1 g
// for its camera and its partials of g^T g and r^T z; the last warp to finish
// (an atomic ticket) sums the partials in camera order (deterministic) and
// sets the CG scalars as k_pcg_init does.
struct PcgInit {
    PcgScalars* S;      // null: no fused start
    float *x, *r, *z, *p, *q;
    float* part;        // 2 per camera
    uint32_t* ticket;   // zero between calls (the last warp resets it)
    float eta;
    int max_it;
};

__device__ void pcg_init_fused(int cam, int n_cam, const float* __restrict__ minv, const float* g, const PcgInit& in,
                               float lam, int lane) {
    __syncwarp();  // minv and g of this camera, written by the warp's lanes
    float gg = 0.f, rz = 0.f;
    if (lane < 9) {
        const int64_t o = 9LL * cam;
        const float* M = minv + 81LL * cam + 9 * lane;
        float zi = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) zi += M[c] * g[o + c];
        const float gi = g[o + lane];
        in.x[o + lane] = 0.f;
        in.r[o + lane] = gi;
        in.q[o + lane] = 0.f;
        in.z[o + lane] = zi;
        in.p[o + lane] = zi;
        gg = gi * gi;
        rz = gi * zi;
    }
    gg = warp_sum(gg);
    rz = warp_sum(rz);
    unsigned last = 0;
    if (lane == 0) {
        in.part[2 * cam] = gg;
        in.part[2 * cam + 1] = rz;
        __threadfence();
        last = atomicAdd(in.ticket, 1u) == (unsigned)(n_cam - 1);
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
    float sg = 0.f, sr = 0.f;
    for (int c = lane; c < n_cam; c += 32) {
        sg += __ldcg(in.part + 2 * c);
        sr += __ldcg(in.part + 2 * c + 1);
    }
    sg = warp_sum(sg);
    sr = warp_sum(sr);
    if (lane == 0) {
        const bool done = !(sg > 0.f && sr > 0.f);
        PcgScalars* S = in.S;
        S->rho = sr;
        S->q_prev = 0.f;
        S->gnorm = sqrtf(sg);
        S->rnorm = sqrtf(sg);
        S->lambda = lam;
        S->eta = in.eta;
        S->it = 0;
        S->max_it = in.max_it;
        S->done = done ? 1 : 0;
        S->stop = done ? 4 : -1;
        S->warm = 0;
        *in.ticket = 0u;
    }
}

// Second pass, one warp per camera: its chunks' sums in chunk order, then
// the 9 x 9 block as in the record path.
__global__ void __launch_bounds__(32)
k_precond_gram_finish(const int32_t* __restrict__ chunk_off, const float* __restrict__ part,
                      const float* __restrict__ dp2, float lam, const float* __restrict__ lam_prob,
                      const int32_t* __restrict__ cam_prob, float* __restrict__ mdiag, float* __restrict__ minv,
                      float* __restrict__ g, uint32_t* err, const int32_t* __restrict__ cam_off,
                      const int32_t* __restrict__ cam_list, const int32_t* __restrict__ obs_pt_s,
                      const int32_t* __restrict__ pt_off, const int64_t* __restrict__ a_off,
                      const int32_t* __restrict__ c_off, const float* __restrict__ apool,
                      const float* __restrict__ cpool, const int32_t* __restrict__ lm_pos,
                      const float4* __restrict__ ipool, int64_t n_obs, const float* __restrict__ rpool,
                      const float* __restrict__ lmrec, int force_exact, const BatchLm* __restrict__ blm,
                      PcgInit init) {
    __shared__ float tot[56], sM[81], sL[81];
    const int cam = blockIdx.x, lane = threadIdx.x;
    if (blm && !batch_active(blm, cam_prob[cam])) return;  // a stopped problem of a batch
    for (int q = lane; q <= REC_SUMS; q += 32) {
        float v = 0.f;
        for (int c = chunk_off[cam]; c < chunk_off[cam + 1]; ++c) v += part[56LL * c + q];
        tot[q] = v;
    }
    __syncwarp();
    if (lam_prob) lam = lam_prob[cam_prob[cam]];
    float trM = 0.f;
#pragma unroll
    for (int u = 0; u < 9; ++u) trM += tot[9 * u - u * (u - 1) / 2] + lam * dp2[9 * cam + u];
    if (force_exact || tot[REC_SUMS] > GRAM_KAPPA_MAX * trM) {
        if (lmrec)
            exact_sums_warp_implicit(cam, cam_off, cam_list, obs_pt_s, pt_off, c_off, lm_pos, ipool, n_obs, rpool,
                                     lmrec, tot, lane);
        else
            exact_sums_warp(cam, cam_off, cam_list, obs_pt_s, pt_off, a_off, c_off, apool, cpool, tot, lane);
        if (lane == 0) atomicAdd(err + 2, 1u);  // cameras summed from the stored blocks (read back by the host)
    }
    precond_finish_warp(cam, tot, dp2, lam, mdiag, minv, g, err, sM, sL, lane);
    if (init.S) pcg_init_fused(cam, gridDim.x, minv, g, init, lam, lane);
}

// ---------------------------------------------------------------------------
// K5: the CG recursion.  One CTA works on the camera range [c0, c1) of one
// problem (9 floats per camera): a single problem uses one CTA of 1024
// threads; a batch of independent problems one CTA of 256 threads per
// problem, with the problem's own scalars and damping.
// ---------------------------------------------------------------------------
constexpr int PCG_T = 1024;
constexpr int BPCG_T = 256;

template <int T>
__device__ __forceinline__ float precond_apply(int c0, int c1, const float* __restrict__ minv,
                                               const float* __restrict__ r, float* __restrict__ z) {
    float rz = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        const int cam = i / 9, row = i - 9 * cam;
        const float* Mi = minv + 81 * (int64_t)cam + 9 * row;
        const float* rc = r + 9 * cam;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) s += Mi[c] * rc[c];
        z[i] = s;
        rz += r[i] * s;
    }
    return rz;
}

// x = 0, r = g, z = M^-1 r, p = z; returns true if there is nothing to solve
// (zero right-hand side, or skip)
template <int T>
__device__ bool pcg_init_range(int c0, int c1, const float* __restrict__ g, const float* __restrict__ minv,
                               float* x, float* r, float* z, float* p, float* q, PcgScalars* S, float lambda,
                               float eta, int max_it, bool skip, float* red) {
    float gg = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        const float gi = skip ? 0.f : g[i];
        x[i] = 0.f;
        r[i] = gi;
        q[i] = 0.f;
        gg += gi * gi;
    }
    __syncthreads();
    float rz = precond_apply<T>(c0, c1, minv, r, z);
    gg = block_sum(gg, red);
    rz = block_sum(rz, red);
    __syncthreads();
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) p[i] = z[i];
    const bool done = !(gg > 0.f && rz > 0.f);
    if (threadIdx.x == 0) {
        S->rho = rz;
        S->q_prev = 0.f;
        S->gnorm = sqrtf(gg);
        S->rnorm = sqrtf(gg);
        S->lambda = lambda;
        S->eta = eta;
        S->it = 0;
        S->max_it = max_it;
        S->done = done ? 1 : 0;
        S->stop = done ? 4 : -1;
        S->warm = 0;
    }
    return done;
}

// one CG iteration after q = A^T A p (the matvec); adds the pose damping
// lambda D_p^2 p to q.  Returns true if a stop rule fired in this call.
// pq_part (non-null, n_part of them): the matvec's per-CTA sums of
// ||A_j p||^2, so that p^T (A^T A + lambda D_p^2) p is formed as a sum of
// squares (positive unless p = 0), not as p^T q from the rounded product
template <int T>
__device__ bool pcg_update_range(int c0, int c1, const float* __restrict__ g, const float* __restrict__ dp2,
                                 const float* __restrict__ minv, float* x, float* r, float* z, float* p, float* q,
                                 PcgScalars* S, float* red, const float* __restrict__ pq_part = nullptr,
                                 int n_part = 0) {
    const float lam = S->lambda;
    const float rho = S->rho;
    float pq = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        const float di = lam * dp2[i] * p[i];
        const float qi = q[i] + di;
        q[i] = qi;
        pq += pq_part ? p[i] * di : p[i] * qi;
    }
    if (pq_part)
        for (int c = threadIdx.x; c < n_part; c += T) pq += pq_part[c];
    pq = block_sum(pq, red);
    if (!(pq > 0.f)) {
        if (threadIdx.x == 0) {
            S->done = 1;
            S->stop = 3;
        }
        return true;
    }
    const float alpha = rho / pq;
    float rr = 0.f, xgr = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        const float xi = x[i] + alpha * p[i];
        const float ri = r[i] - alpha * q[i];
        x[i] = xi;
        r[i] = ri;
        rr += ri * ri;
        xgr += xi * (g[i] + ri);
    }
    rr = block_sum(rr, red);
    xgr = block_sum(xgr, red);
    const int it = S->it + 1;
    const float q1 = -0.5f * xgr;
    const float rn = sqrtf(rr);
    int stop = -1;
    if (rn <= 1e-10f * S->gnorm) stop = 1;
    else if ((float)it * (q1 - S->q_prev) / q1 < S->eta) stop = 0;
    else if (it >= S->max_it) stop = 2;
    __syncthreads();
    if (threadIdx.x == 0) {
        S->it = it;
        S->q_prev = q1;
        S->rnorm = rn;
        if (stop >= 0) {
            S->done = 1;
            S->stop = stop;
        }
    }
    if (stop >= 0) return true;
    float rz = precond_apply<T>(c0, c1, minv, r, z);
    rz = block_sum(rz, red);
    const float beta = rz / rho;
    __syncthreads();
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        p[i] = z[i] + beta * p[i];
        q[i] = 0.f;
    }
    if (threadIdx.x == 0) S->rho = rz;
    return false;
}

// Warm start (learned): x = x0 is given and q = (A^T A) x0 from the matvec;
// r = g - q - lambda D_p^2 x0 and Q(x0) = -1/2 x0^T (g + r).  The true
// residual judges the warm start: unless Q(x0) < 0 (a decrease of the
// quadratic model from the zero start) it is dropped and CG starts from 0.
template <int T>
__device__ bool pcg_init_warm_range(int c0, int c1, const float* __restrict__ g, const float* __restrict__ dp2,
                                    const float* __restrict__ minv, float* x, float* r, float* z, float* p,
                                    float* q, PcgScalars* S, float lambda, float eta, int max_it, float* red) {
    float gg = 0.f, xgr = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        const float gi = g[i], xi = x[i];
        const float ri = gi - q[i] - lambda * dp2[i] * xi;
        r[i] = ri;
        gg += gi * gi;
        xgr += xi * (gi + ri);
    }
    gg = block_sum(gg, red);
    xgr = block_sum(xgr, red);
    const float q0 = -0.5f * xgr;
    const bool keep = q0 < 0.f;
    __syncthreads();
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) {
        if (!keep) {
            x[i] = 0.f;
            r[i] = g[i];
        }
        q[i] = 0.f;
    }
    __syncthreads();
    float rz = precond_apply<T>(c0, c1, minv, r, z);
    float rr = 0.f;
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) rr += r[i] * r[i];
    rz = block_sum(rz, red);
    rr = block_sum(rr, red);
    __syncthreads();
    for (int i = 9 * c0 + threadIdx.x; i < 9 * c1; i += T) p[i] = z[i];
    const float rn = sqrtf(rr), gn = sqrtf(gg);
    const bool done = !(gg > 0.f && rz > 0.f) || rn <= 1e-10f * gn;
    if (threadIdx.x == 0) {
        S->rho = rz;
        S->q_prev = keep ? q0 : 0.f;
        S->gnorm = gn;
        S->rnorm = rn;
        S->lambda = lambda;
        S->eta = eta;
        S->it = 0;
        S->max_it = max_it;
        S->done = done ? 1 : 0;
        S->stop = done ? (gg > 0.f ? 1 : 4) : -1;
        S->warm = keep ? 1 : 0;
    }
    return done;
}

__global__ void __launch_bounds__(PCG_T)
k_pcg_init_warm(int n_cam, const float* __restrict__ g, const float* __restrict__ dp2,
                const float* __restrict__ minv, float* x, float* r, float* z, float* p, float* q, PcgScalars* S,
                float lambda, float eta, int max_it) {
    __shared__ float red[32];
    pcg_init_warm_range<PCG_T>(0, n_cam, g, dp2, minv, x, r, z, p, q, S, lambda, eta, max_it, red);
}

__global__ void __launch_bounds__(PCG_T)
k_pcg_init(int n_cam, const float* __restrict__ g, const float* __restrict__ minv, float* x, float* r,
           float* z, float* p, float* q, PcgScalars* S, float lambda, float eta, int max_it) {
    __shared__ float red[32];
    pcg_init_range<PCG_T>(0, n_cam, g, minv, x, r, z, p, q, S, lambda, eta, max_it, false, red);
}

// `cond`: when the iterations run inside a conditional WHILE node of a CUDA
// graph (cond_on != 0), the kernel ends the loop by setting the node's
// condition to 0 once the CG has stopped; the only writer is thread 0.
__global__ void __launch_bounds__(PCG_T)
k_pcg_update(int n_cam, const float* __restrict__ g, const float* __restrict__ dp2,
             const float* __restrict__ minv, float* x, float* r, float* z, float* p, float* q,
             PcgScalars* S, cudaGraphConditionalHandle cond, int cond_on, const float* __restrict__ pq_part,
             int n_part) {
    __shared__ float red[32];
    if (S->done) {
        if (cond_on && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const bool fin = pcg_update_range<PCG_T>(0, n_cam, g, dp2, minv, x, r, z, p, q, S, red, pq_part, n_part);
    if (fin && cond_on && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
}

// batch: a problem that finishes bumps the counter; the last one marks the
// batch-wide scalars done (read by the matvec to skip the remaining work)
__device__ __forceinline__ void batch_problem_done(int n_prob, int32_t* n_done, PcgScalars* S_all, int it) {
    atomicMax(&S_all->it, it);
    if (atomicAdd(n_done, 1) == n_prob - 1) S_all->done = 1;
}

__global__ void k_set_max_it(PcgScalars* S, int max_it) { S->max_it = max_it; }

__global__ void __launch_bounds__(BPCG_T)
k_bpcg_init(int n_prob, const int32_t* __restrict__ prob_cam_off, const BatchLm* __restrict__ lm,
            const float* __restrict__ lam, const float* __restrict__ g, const float* __restrict__ minv, float* x,
            float* r, float* z, float* p, float* q, PcgScalars* Sb, PcgScalars* S_all, int32_t* n_done, float eta,
            int max_it) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    const bool done = pcg_init_range<BPCG_T>(prob_cam_off[b], prob_cam_off[b + 1], g, minv, x, r, z, p, q, Sb + b,
                                             lam[b], eta, max_it, !lm[b].active, red);
    if (done && threadIdx.x == 0) batch_problem_done(n_prob, n_done, S_all, 0);
}

// In a WHILE node the loop is ended by CTA 0 alone, at the start of the
// iteration after the batch-wide done flag was set (one writer, no race), or
// once the iterations exceed max_it + 2 (a guard: every problem stops at
// max_it by itself).
__global__ void __launch_bounds__(BPCG_T)
k_bpcg_update(int n_prob, const int32_t* __restrict__ prob_cam_off, const float* __restrict__ g,
              const float* __restrict__ dp2, const float* __restrict__ minv, float* x, float* r, float* z, float* p,
              float* q, PcgScalars* Sb, PcgScalars* S_all, int32_t* n_done, cudaGraphConditionalHandle cond,
              int cond_on) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    if (cond_on && b == 0 && threadIdx.x == 0) {
        const int loops = ++S_all->pad;
        if (S_all->done || loops > S_all->max_it + 2) {
            S_all->done = 1;
            cudaGraphSetConditional(cond, 0);
        }
    }
    PcgScalars* S = Sb + b;
    if (S->done) return;
    const bool fin = pcg_update_range<BPCG_T>(prob_cam_off[b], prob_cam_off[b + 1], g, dp2, minv, x, r, z, p, q, S, red);
    if (fin && threadIdx.x == 0) batch_problem_done(n_prob, n_done, S_all, S->it);
}

}  // namespace

void build_k3_records(Problem& p) {
    p.k3rec = dalloc<int4>(p, std::max<int64_t>(1, p.n_obs));
    p.k3xy = dalloc<float2>(p, std::max<int64_t>(1, p.n_obs));
    if (p.n_obs > 0)
        k_k3_records<<<p.sm_count * 8, 256, 0, p.stream>>>(p.n_obs, p.cam_list, p.obs_pt_s, p.pt_off, p.c_off, p.lm_pos,
                                                          p.obs_xy_s, p.k3rec, p.k3xy);
    BA_LAUNCH_CHECK();
}

bool launch_precond_rhs(Problem& p, bool fuse_init) {
    if (p.schur) {
        launch_schur_precond(p);
        return false;
    }
    if (!p.opt.precond_from_blocks || p.implicit) {
        // (implicit storage with precond_from_blocks: every camera's sums from
        // the factorisation, in the finish kernel)
        const float* lmrec = p.implicit ? p.lmrec : nullptr;
        count_launches(p, p.pg_chunks > 0 ? 2 : 1);
        if (p.pg_chunks > 0)
            (p.implicit ? k_precond_gram<true> : k_precond_gram<false>)<<<p.pg_chunks, PG_T, 0, p.stream>>>(
                p.pg_chunk_cam, p.pg_chunk_off, p.cam_off, p.cam_list, p.obs_pt_s, p.obs_xy_s, p.pt_off, p.frames,
                p.pts, p.tpool, p.pg_part, lmrec, p.lm_pos, p.c_off, reinterpret_cast<const float4*>(p.ipool),
                p.n_obs, p.k3rec, p.k3xy, (float)p.opt.huber_delta, p.batch.n_prob > 0 ? p.batch.lm : nullptr,
                p.batch.cam_prob);
        const bool fuse = fuse_init && p.batch.n_prob == 0;
        if (fuse && !p.init_part) {
            p.init_part = dalloc<float>(p, 2LL * p.n_cam);
            p.init_ticket = dalloc<uint32_t>(p, 1);
        }
        if (fuse) BA_CUDA_TRY(cudaMemsetAsync(p.init_ticket, 0, sizeof(uint32_t), p.stream));
        const PcgInit init{fuse ? p.pcg : nullptr, p.x, p.r, p.z, p.p, p.q, p.init_part, p.init_ticket,
                           (float)p.opt.cg_eta, p.opt.max_cg_iters};
        k_precond_gram_finish<<<p.n_cam, 32, 0, p.stream>>>(
            p.pg_chunk_off, p.pg_part, p.dp2, (float)p.lambda_damped, p.batch.lam, p.batch.cam_prob, p.mdiag, p.minv,
            p.g, p.err, p.cam_off, p.cam_list, p.obs_pt_s, p.pt_off, p.a_off, p.c_off, p.apool, p.cpool, p.lm_pos,
            reinterpret_cast<const float4*>(p.ipool), p.n_obs, p.rpool, lmrec,
            p.implicit && p.opt.precond_from_blocks ? 1 : 0, p.batch.n_prob > 0 ? p.batch.lm : nullptr, init);
        BA_LAUNCH_CHECK();
        return fuse;
    }
    launch_precond_records(p);
    count_launches(p, 2 + (p.pc_plan.n_obs_split > 0 ? 1 : 0));
    k_precond_reduce<<<p.n_cam, 32 * PC_WARPS, 0, p.stream>>>(p.n_cam, p.cam_off, p.cam_list_st, p.prec, p.dp2,
                                                             (float)p.lambda_damped, p.batch.lam, p.batch.cam_prob,
                                                             p.mdiag, p.minv, p.g, p.err);
    BA_LAUNCH_CHECK();
    return false;
}

// the block inverses the CG applies: plain block Jacobi, or the learned
// correction B_i when the learned mode is active for this solve
const float* active_minv(const Problem& p) { return p.learned_active ? p.minv_l : p.minv; }

void launch_pcg_init(Problem& p) {
    if (p.batch.n_prob > 0) {
        BatchState& B = p.batch;
        count_launches(p, 1);
        BA_CUDA_TRY(cudaMemsetAsync(p.pcg, 0, sizeof(PcgScalars), p.stream));
        BA_CUDA_TRY(cudaMemsetAsync(B.n_done, 0, sizeof(int32_t), p.stream));
        k_set_max_it<<<1, 1, 0, p.stream>>>(p.pcg, p.opt.max_cg_iters);
        k_bpcg_init<<<B.n_prob, BPCG_T, 0, p.stream>>>(B.n_prob, B.prob_cam_off, B.lm, B.lam, p.g, p.minv, p.x, p.r,
                                                      p.z, p.p, p.q, B.pcg, p.pcg, B.n_done, (float)p.opt.cg_eta,
                                                      p.opt.max_cg_iters);
        BA_LAUNCH_CHECK();
        return;
    }
    count_launches(p, 1);
    k_pcg_init<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, active_minv(p), p.x, p.r, p.z, p.p, p.q, p.pcg,
                                          (float)p.lambda_damped, (float)p.opt.cg_eta, p.opt.max_cg_iters);
    BA_LAUNCH_CHECK();
}

void launch_pcg_init_warm(Problem& p) {
    count_launches(p, 1);
    k_pcg_init_warm<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, p.dp2, active_minv(p), p.x, p.r, p.z, p.p, p.q, p.pcg,
                                               (float)p.lambda_damped, (float)p.opt.cg_eta, p.opt.max_cg_iters);
    BA_LAUNCH_CHECK();
}

void launch_pcg_iteration(Problem& p, cudaEvent_t mv_begin, cudaEvent_t mv_end, bool in_while,
                          cudaGraphConditionalHandle cond) {
    count_launches(p, 2);
    auto record = [&](cudaEvent_t ev) {
        if (!ev) return;
        if (p.capturing) BA_CUDA_TRY(cudaEventRecordWithFlags(ev, p.stream, cudaEventRecordExternal));
        else BA_CUDA_TRY(cudaEventRecord(ev, p.stream));
    };
    // the implicit storage's matvec also forms p^T A^T A p as a sum of squares (a single problem)
    const bool sq = p.implicit && p.batch.n_prob == 0;
    record(mv_begin);
    if (sq) launch_matvec_implicit(p, p.p, p.q, p.pcg, p.pq_part);
    else launch_matvec_raw(p, p.p, p.q, p.pcg);
    record(mv_end);
    if (p.batch.n_prob > 0) {
        BatchState& B = p.batch;
        k_bpcg_update<<<B.n_prob, BPCG_T, 0, p.stream>>>(B.n_prob, B.prob_cam_off, p.g, p.dp2, p.minv, p.x, p.r, p.z,
                                                        p.p, p.q, B.pcg, p.pcg, B.n_done, cond, in_while ? 1 : 0);
    } else {
        k_pcg_update<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, p.dp2, active_minv(p), p.x, p.r, p.z, p.p, p.q,
                                                p.pcg, cond, in_while ? 1 : 0, sq ? p.pq_part : nullptr,
                                                sq ? implicit_matvec_grid(p) : 0);
    }
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
