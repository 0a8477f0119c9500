// K6: landmark back substitution (Eq. backsub_nm, damped form of Sec. 5.3):
//     dx_l = -R1^-1 (Q1^T r + Q1^T J_p dx_p)
// from the three top rows of each landmark block (one warp per landmark),
// followed by the Gauss-Newton model cost L(dx) = ||r + J_p dx_p + J_l dx_l||^2
// (undamped) evaluated per observation (one thread each) from the camera
// model, each observation's term in FP32, the sum in FP64.
//
// K7 (same file): candidate state x (+) dx (rotation Exp(dw) R, everything
// else additive) and the energy E = sum ||r||^2 (Eq. ba_energy), FP32 terms
// accumulated in FP64.  All FP64 sums are deterministic: fixed per-block
// partials reduced in a fixed order.
#include <algorithm>

#include "camera.cuh"
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int BS_WARPS = 8;

// dl_j for one landmark per team of BS_TEAM lanes, landmarks in storage order
// (neighbouring teams have equal or similar k): lane t takes observations
// t, t + BS_TEAM, ...: its camera's dx_p (9 values) against its 3 x 9 slice of
// the top rows (three contiguous 36-byte runs), then a team sum of the three
// partial dot products and the 3x3 triangular solve on the team's first lane.
constexpr int BS_TEAM = 8;
__global__ void __launch_bounds__(32 * BS_WARPS)
k_backsub_dl(int n_pt, const int32_t* __restrict__ lm_by_k, const int32_t* __restrict__ pt_off,
             const int32_t* __restrict__ obs_cam_s, const float* __restrict__ tpool, const float* __restrict__ dp,
             float* __restrict__ dl, const BatchLm* __restrict__ blm, const int32_t* __restrict__ lm_prob) {
    const int lane = threadIdx.x & 31, rank = lane & (BS_TEAM - 1);
    const int pos = (blockIdx.x * (32 * BS_WARPS) + threadIdx.x) / BS_TEAM;
    bool has = pos < n_pt;
    const int j = has ? lm_by_k[pos] : 0;
    if (has && blm && !batch_active(blm, lm_prob[j])) has = false;  // a stopped problem of a batch
    const int s0 = has ? pt_off[j] : 0, k = has ? pt_off[j + 1] - s0 : 0, ncol = 9 * k;
    const float* top = tpool + top_offset(s0, j);
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    for (int t = rank; t < k; t += BS_TEAM) {
        const float* d = dp + 9 * __ldg(obs_cam_s + s0 + t);
        const float* r0 = top + 9 * t;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float dc = __ldg(d + c);
            t0 += __ldg(r0 + c) * dc;
            t1 += __ldg(r0 + (ncol + 4) + c) * dc;
            t2 += __ldg(r0 + 2 * (ncol + 4) + c) * dc;
        }
    }
#pragma unroll
    for (int o = BS_TEAM / 2; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    }
    if (!has || rank != 0) return;
    const float* R0 = top + ncol;
    const float* R1 = top + (ncol + 4) + ncol;
    const float* R2 = top + 2 * (ncol + 4) + ncol;
    t0 += R0[3];
    t1 += R1[3];
    t2 += R2[3];
    const float r00 = R0[0], r01 = R0[1], r02 = R0[2], r11 = R1[1], r12 = R1[2], r22 = R2[2];
    const float l2 = -t2 / r22;
    const float l1 = (-t1 - r12 * l2) / r11;
    const float l0 = (-t0 - r01 * l1 - r02 * l2) / r00;
    dl[3 * j] = l0;
    dl[3 * j + 1] = l1;
    dl[3 * j + 2] = l2;
}

// The same in the implicit storage, which keeps no top rows: with
// u_s = V_s^T (J_s dx_p) (the observation's two Householder rows against its
// two linearised residual rows) the undamped top rows give
//   Q1^T J_p dx_p = sum_s D_s dx_p - P sum_s u_s
// (D_s dx_p is (J_s dx_p, 0) for slot 0 and (0, 0, first row) for slot 1),
// and the damped right-hand side is G_tt t + G_tt sum D_s dx_p - (G_tt P)
// sum u_s.  Lane t of a team reads observation t's record (6 float4, in
// storage order: coalesced over the team).
__global__ void __launch_bounds__(32 * BS_WARPS)
k_backsub_dl_implicit(int n_pt, const int32_t* __restrict__ lm_by_k, const int32_t* __restrict__ pt_off,
                      const int32_t* __restrict__ c_off, const int32_t* __restrict__ obs_cam_s,
                      const float4* __restrict__ ipool, int64_t n_obs, const float* __restrict__ dp,
                      float* __restrict__ dl, const float* __restrict__ lmrec, const BatchLm* __restrict__ blm,
                      const int32_t* __restrict__ lm_prob) {
    const int lane = threadIdx.x & 31, rank = lane & (BS_TEAM - 1);
    const int pos = (blockIdx.x * (32 * BS_WARPS) + threadIdx.x) / BS_TEAM;
    bool has = pos < n_pt;
    const int j = has ? lm_by_k[pos] : 0;
    if (has && blm && !batch_active(blm, lm_prob[j])) has = false;  // a stopped problem of a batch
    const int s0 = has ? pt_off[j] : 0, k = has ? pt_off[j + 1] - s0 : 0;
    const int64_t so0 = has ? (c_off[j] >> 1) : 0;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    for (int t = rank; t < k; t += BS_TEAM) {
        float f[24];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float4 c = __ldg(ipool + m * n_obs + so0 + t);
            f[4 * m] = c.x;
            f[4 * m + 1] = c.y;
            f[4 * m + 2] = c.z;
            f[4 * m + 3] = c.w;
        }
        const float* d = dp + 9 * __ldg(obs_cam_s + s0 + t);
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float dc = __ldg(d + c);
            e0 += f[c] * dc;
            e1 += f[9 + c] * dc;
        }
        u0 += f[18] * e0 + f[21] * e1;
        u1 += f[19] * e0 + f[22] * e1;
        u2 += f[20] * e0 + f[23] * e1;
        if (t == 0) {
            d0 = e0;
            d1 = e1;
        } else if (t == 1) {
            d2 = e0;
        }
    }
#pragma unroll
    for (int o = BS_TEAM / 2; o > 0; o >>= 1) {
        u0 += __shfl_xor_sync(0xffffffffu, u0, o);
        u1 += __shfl_xor_sync(0xffffffffu, u1, o);
        u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    }
    if (!has || rank != 0) return;
    const float* L = lmrec + (int64_t)LM_REC * pos;
    const float* GP = L + LR_GP;
    const float* Gt = L + LR_GT;
    const float* G = L + LR_G;
    const float* R = L + LR_RD;
    float a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        a[i] = Gt[i] + G[3 * i] * d0 + G[3 * i + 1] * d1 + G[3 * i + 2] * d2 -
               (GP[3 * i] * u0 + GP[3 * i + 1] * u1 + GP[3 * i + 2] * u2);
    const float l2 = -a[2] / R[5];
    const float l1 = (-a[1] - R[4] * l2) / R[3];
    const float l0 = (-a[0] - R[1] * l1 - R[2] * l2) / R[0];
    dl[3 * j] = l0;
    dl[3 * j + 1] = l1;
    dl[3 * j + 2] = l2;
}

// One observation: the Gauss-Newton model term ||r + J_p dp + J_l dl||^2 at
// the current state and, optionally, the energy term ||r||^2 at the candidate.
__device__ __forceinline__ void model_cost_obs(int64_t s, const float* __restrict__ frames, const float* __restrict__ pts,
                                               const int32_t* __restrict__ obs_cam_s,
                                               const int32_t* __restrict__ obs_pt_s,
                                               const float2* __restrict__ obs_xy_s, const float* __restrict__ dp,
                                               const float* __restrict__ dl, const float* __restrict__ cand_frames,
                                               const float* __restrict__ cand_pts, float huber, double& m,
                                               double& c) {
    const int j = obs_pt_s[s], cam = obs_cam_s[s];
    const float2 z = obs_xy_s[s];
    float r[2], Jp[18], Jl[6];
    frame_jacobians(frames + FRAME * cam, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r, Jp, Jl);
    const float* d = dp + 9 * cam;
    const float l0 = dl[3 * j], l1 = dl[3 * j + 1], l2 = dl[3 * j + 2];
    // robust norm: rho(s) - w s + w ||r + J dx||^2 (w = 1, rho(s) = s without
    // it); the observation's terms in FP32, their sums in FP64 (energy_term)
    const float w = huber_weight(huber, r[0], r[1]);
    float e[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        e[i] = r[i] + Jl[3 * i] * l0 + Jl[3 * i + 1] * l1 + Jl[3 * i + 2] * l2;
#pragma unroll
        for (int q = 0; q < 9; ++q) e[i] += Jp[9 * i + q] * d[q];
    }
    const float mo = e[0] * e[0] + e[1] * e[1];
    if (w == 1.f) {
        m += (double)mo;
    } else {
        const double s = (double)(r[0] * r[0] + r[1] * r[1]);
        m += huber_rho(huber, s) - (double)w * s + (double)w * (double)mo;
    }
    if (cand_frames) {
        float r0, r1;
        frame_residual(cand_frames + FRAME * cam, cand_pts[3 * j], cand_pts[3 * j + 1], cand_pts[3 * j + 2], z.x, z.y,
                       r0, r1);
        c += energy_term(huber, r0, r1);
    }
}

// K6 model cost (and with the candidate state, K7's energy) per observation,
// FP64 partial sums per CTA
__global__ void __launch_bounds__(256)
k_model_cost(int64_t n_obs, const float* __restrict__ frames, const float* __restrict__ pts,
             const int32_t* __restrict__ obs_cam_s, const int32_t* __restrict__ obs_pt_s,
             const float2* __restrict__ obs_xy_s, const float* __restrict__ dp, const float* __restrict__ dl,
             const float* __restrict__ cand_frames, const float* __restrict__ cand_pts, double* __restrict__ part_m,
             double* __restrict__ part_c, float huber) {
    __shared__ double red[32];
    double m = 0.0, c = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_obs; s += (int64_t)gridDim.x * blockDim.x)
        model_cost_obs(s, frames, pts, obs_cam_s, obs_pt_s, obs_xy_s, dp, dl, cand_frames, cand_pts, huber, m, c);
    m = block_sum_d(m, red);
    if (cand_frames) c = block_sum_d(c, red);
    if (threadIdx.x == 0) {
        part_m[blockIdx.x] = m;
        if (cand_frames) part_c[blockIdx.x] = c;
    }
}

// batch: the same per problem (one CTA per problem, its observation range)
__global__ void __launch_bounds__(256)
k_model_cost_seg(const int64_t* __restrict__ prob_obs_off, const float* __restrict__ frames,
                 const float* __restrict__ pts, const int32_t* __restrict__ obs_cam_s,
                 const int32_t* __restrict__ obs_pt_s, const float2* __restrict__ obs_xy_s,
                 const float* __restrict__ dp, const float* __restrict__ dl, const float* __restrict__ cand_frames,
                 const float* __restrict__ cand_pts, double* __restrict__ model, double* __restrict__ cost,
                 float huber, const BatchLm* __restrict__ blm) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    if (blm && !blm[b].active) {  // a stopped problem: its sums are not read
        if (threadIdx.x == 0) model[b] = cost[b] = 0.0;
        return;
    }
    double m = 0.0, c = 0.0;
    for (int64_t s = prob_obs_off[b] + threadIdx.x; s < prob_obs_off[b + 1]; s += blockDim.x)
        model_cost_obs(s, frames, pts, obs_cam_s, obs_pt_s, obs_xy_s, dp, dl, cand_frames, cand_pts, huber, m, c);
    m = block_sum_d(m, red);
    c = block_sum_d(c, red);
    if (threadIdx.x == 0) {
        model[b] = m;
        cost[b] = c;
    }
}

__global__ void __launch_bounds__(256)
k_cost(int64_t n_obs, const float* __restrict__ frames, const float* __restrict__ pts,
       const int32_t* __restrict__ obs_cam_s, const int32_t* __restrict__ obs_pt_s,
       const float2* __restrict__ obs_xy_s, double* __restrict__ partials, float huber) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_obs;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int j = obs_pt_s[s];
        const float2 z = obs_xy_s[s];
        float r0, r1;
        frame_residual(frames + FRAME * obs_cam_s[s], pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r0, r1);
        acc += energy_term(huber, r0, r1);
    }
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Fixed-order FP64 sums of the per-CTA partials by one warp: lane l adds
// partials l, l + 32, ... in order, then a fixed butterfly (deterministic; one
// warp keeps the FP64 instruction count and the latency chain short).
__global__ void __launch_bounds__(32)
k_sum_partials(const double* __restrict__ partials, int n, double* out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) acc += partials[i];
    acc = warp_sum_d(acc);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void __launch_bounds__(32)
k_sum_partials2(const double* __restrict__ a, const double* __restrict__ b, int n, double* out_a, double* out_b) {
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) {
        sa += a[i];
        sb += b[i];
    }
    sa = warp_sum_d(sa);
    sb = warp_sum_d(sb);
    if (threadIdx.x == 0) {
        *out_a = sa;
        *out_b = sb;
    }
}

__global__ void k_candidate(int n_cam, const float* __restrict__ cams, const float* __restrict__ dp,
                            float* __restrict__ cand_cams, float* __restrict__ cand_frames, int n_pt,
                            const float* __restrict__ pts, const float* __restrict__ dl, float* __restrict__ cand_pts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cam) {
        const float* c = cams + 9 * i;
        const float* d = dp + 9 * i;
        float w[3];
        compose_rotation(d, c, w);
        float* o = cand_cams + 9 * i;
        o[0] = w[0];
        o[1] = w[1];
        o[2] = w[2];
#pragma unroll
        for (int m = 3; m < 9; ++m) o[m] = c[m] + d[m];
        make_frame(o, cand_frames + FRAME * i);
    }
    if (i < 3 * n_pt) cand_pts[i] = pts[i] + dl[i];
}

}  // namespace

// K6: dl per landmark (the stored top rows, or the implicit storage's records)
static void launch_backsub_dl(Problem& p) {
    const int grid = (int)ceil_div((int64_t)p.n_pt * BS_TEAM, 32 * BS_WARPS);
    const BatchLm* blm = p.batch.n_prob > 0 ? p.batch.lm : nullptr;
    if (p.implicit)
        k_backsub_dl_implicit<<<grid, 32 * BS_WARPS, 0, p.stream>>>(
            p.n_pt, p.lm_by_k, p.pt_off, p.c_off, p.obs_cam_s, reinterpret_cast<const float4*>(p.ipool), p.n_obs,
            p.x, p.dl, p.lmrec, blm, p.batch.lm_prob);
    else
        k_backsub_dl<<<grid, 32 * BS_WARPS, 0, p.stream>>>(p.n_pt, p.lm_by_k, p.pt_off, p.obs_cam_s, p.tpool, p.x,
                                                          p.dl, blm, p.batch.lm_prob);
}

// K6: dl per landmark, then the model cost L(dx) per observation (FP64)
void launch_backsub(Problem& p) {
    count_launches(p, 3);
    if (p.schur)
        launch_schur_backsub(p);
    else
        launch_backsub_dl(p);
    k_model_cost<<<p.red_grid, 256, 0, p.stream>>>(p.n_obs, p.frames, p.pts, p.obs_cam_s, p.obs_pt_s, p.obs_xy_s, p.x,
                                                   p.dl, nullptr, nullptr, p.partials, nullptr, (float)p.opt.huber_delta);
    k_sum_partials<<<1, 32, 0, p.stream>>>(p.partials, p.red_grid, p.dsum + 1);
    BA_LAUNCH_CHECK();
}

// K6 + K7 of one LM iteration fused: dl, the candidate state, then one pass
// over the observations for the model cost (dsum[1]) and the candidate's
// energy (dsum[0]); a batch gets both per problem (cost_a, cost_b)
void launch_backsub_candidate_cost(Problem& p) {
    count_launches(p, p.batch.n_prob > 0 ? 2 : 3);
    if (p.schur)
        launch_schur_backsub(p);
    else
        launch_backsub_dl(p);
    launch_candidate(p);
    if (p.batch.n_prob > 0) {
        BatchState& B = p.batch;
        k_model_cost_seg<<<B.n_prob, 256, 0, p.stream>>>(B.prob_obs_off, p.frames, p.pts, p.obs_cam_s, p.obs_pt_s,
                                                         p.obs_xy_s, p.x, p.dl, p.cand_frames, p.cand_pts, B.cost_b,
                                                         B.cost_a, (float)p.opt.huber_delta, B.lm);
    } else {
        k_model_cost<<<p.red_grid, 256, 0, p.stream>>>(p.n_obs, p.frames, p.pts, p.obs_cam_s, p.obs_pt_s, p.obs_xy_s,
                                                       p.x, p.dl, p.cand_frames, p.cand_pts, p.partials,
                                                       p.partials + p.red_grid, (float)p.opt.huber_delta);
        k_sum_partials2<<<1, 32, 0, p.stream>>>(p.partials, p.partials + p.red_grid, p.red_grid, p.dsum + 1,
                                                  p.dsum + 0);
    }
    BA_LAUNCH_CHECK();
}

void launch_candidate(Problem& p) {
    count_launches(p, 1);
    const int n = std::max(p.n_cam, 3 * p.n_pt);
    k_candidate<<<ceil_div(n, 256), 256, 0, p.stream>>>(p.n_cam, p.cams, p.x, p.cand_cams, p.cand_frames, p.n_pt,
                                                       p.pts, p.dl, p.cand_pts);
    BA_LAUNCH_CHECK();
}

// E at the current state (its frames are recomputed first) or at the
// candidate (frames written by k_candidate)
void launch_cost(Problem& p, bool candidate, int slot) {
    if (!candidate) launch_frames(p);
    launch_cost_on(p, candidate ? p.cand_frames : p.frames, candidate ? p.cand_pts : p.pts, slot, p.stream);
}

// E from the given frames and points into dsum[slot] on stream st (the
// per-CTA partials, then their fixed-order sum)
void launch_cost_on(Problem& p, const float* frames, const float* pts, int slot, cudaStream_t st) {
    count_launches(p, 2);
    k_cost<<<p.red_grid, 256, 0, st>>>(p.n_obs, frames, pts, p.obs_cam_s, p.obs_pt_s, p.obs_xy_s, p.partials,
                                       (float)p.opt.huber_delta);
    k_sum_partials<<<1, 32, 0, st>>>(p.partials, p.red_grid, p.dsum + slot);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
