// The explicit Schur complement in FP32 (Sec. 4.2, Eq. red_normal_eq): the
// comparison solver of Sec. 6.4 ("explicit-32"), kept to test the paper's
// numerical claim that forming H~ = H_pp - H_pl H_ll^-1 H_lp in single
// precision loses positive definiteness where the square-root form does not.
// Enabled by ba_options.schur_explicit; every other step of the LM (damping
// diagonals, PCG recursion, model cost, candidate, decisions) is shared.
//
//   assembly (per lambda): one warp per landmark, lanes over its
//     observations: r, J_p, J_l from the camera model (robust rows if set),
//     H_ll + lambda D_l^2 and b_l (warp sums), its inverse (FP32 Cholesky),
//     W_s = J_s^T J_l,s; then H~_ss += J_s^T J_s - W_s H_ll^-1 W_s^T,
//     H~_st += -W_s H_ll^-1 W_t^T (s < t, both (a, b) and (b, a) blocks) and
//     b~_s += J_s^T r_s - W_s H_ll^-1 b_l with FP32 atomics into a block-sparse
//     matrix (both triangles) whose pattern the host builds at create;
//   matvec: one thread per row of H~ (9 per camera) over its row's blocks;
//   preconditioner: the diagonal blocks (plus lambda D_p^2) inverted as in K3;
//   back substitution (Eq. backsub_sc): dl_j = -(H_ll + lambda D_l^2)^-1
//     (b_l + sum_s W_s^T dp_s), recomputed per landmark.
#include <algorithm>
#include <vector>

#include "camera.cuh"
#include "precond.cuh"
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int SC_WARPS = 4;
constexpr int SC_KMAX = 64;  // observations per landmark staged in shared memory at once

// 3x3 symmetric positive definite inverse by Cholesky; false if not PD in FP32
__device__ __forceinline__ bool inv3_spd(const float H[6], float I[9]) {
    // H = [h00 h01 h02; . h11 h12; . . h22] (upper, row-major order 00 01 02 11 12 22)
    const float l00s = H[0];
    if (!(l00s > 0.f)) return false;
    const float l00 = sqrtf(l00s), l10 = H[1] / l00, l20 = H[2] / l00;
    const float l11s = H[3] - l10 * l10;
    if (!(l11s > 0.f)) return false;
    const float l11 = sqrtf(l11s), l21 = (H[4] - l20 * l10) / l11;
    const float l22s = H[5] - l20 * l20 - l21 * l21;
    if (!(l22s > 0.f)) return false;
    const float l22 = sqrtf(l22s);
    // L^-1 (lower)
    const float a00 = 1.f / l00, a11 = 1.f / l11, a22 = 1.f / l22;
    const float a10 = -l10 * a00 * a11;
    const float a21 = -l21 * a11 * a22;
    const float a20 = -(l20 * a00 + l21 * a10) * a22;
    // H^-1 = L^-T L^-1
    I[0] = a00 * a00 + a10 * a10 + a20 * a20;
    I[1] = a10 * a11 + a20 * a21;
    I[2] = a20 * a22;
    I[4] = a11 * a11 + a21 * a21;
    I[5] = a21 * a22;
    I[8] = a22 * a22;
    I[3] = I[1];
    I[6] = I[2];
    I[7] = I[5];
    return true;
}

struct ScArgs {
    const float* frames;
    const float* pts;
    const int32_t* obs_cam_s;
    const float2* obs_xy_s;
    const int32_t* pt_off;
    const float* dl2;
    float lambda;
    const float* lam_prob;  // batch: damping per problem
    const int32_t* lm_prob;
    float huber;
    const int64_t* pair_off;   // per landmark: first pair index (pairs s < t in slot order)
    const int32_t* pair_blk;   // per pair: block (a, b) and block (b, a)
    const int32_t* diag_blk;   // per camera: its diagonal block
    float* blk;                // nblk x 81
    float* bt;                 // 9 n_cam (b~)
    uint32_t* err;
};

__device__ __forceinline__ void sc_obs(const ScArgs& a, int64_t s, int j, float r[2], float Jp[18], float Jl[6]) {
    const float2 z = a.obs_xy_s[s];
    frame_jacobians(a.frames + FRAME * a.obs_cam_s[s], a.pts[3 * j], a.pts[3 * j + 1], a.pts[3 * j + 2], z.x, z.y, r,
                    Jp, Jl);
    huber_scale_rows(a.huber, r, Jp, Jl);
}

// The landmark's H_ll + lambda D_l^2 (upper) and b_l, and W_s, bp_s of this lane's observations into shared memory
__global__ void __launch_bounds__(32 * SC_WARPS) k_sc_assemble(ScArgs a, int n_pt) {
    __shared__ float sW[SC_WARPS][SC_KMAX][27];
    __shared__ float sHi[SC_WARPS][9], sYb[SC_WARPS][3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * SC_WARPS + w;
    if (j >= n_pt) return;
    const int64_t s0 = a.pt_off[j];
    const int k = a.pt_off[j + 1] - (int)s0;
    // pass 1: H_ll and b_l
    float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, bl[3] = {0.f, 0.f, 0.f};
    for (int t = lane; t < k; t += 32) {
        float r[2], Jp[18], Jl[6];
        sc_obs(a, s0 + t, j, r, Jp, Jl);
        int q = 0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            bl[u] += Jl[u] * r[0] + Jl[3 + u] * r[1];
#pragma unroll
            for (int v = u; v < 3; ++v) h[q++] += Jl[u] * Jl[v] + Jl[3 + u] * Jl[3 + v];
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) h[q] = warp_sum(h[q]);
#pragma unroll
    for (int u = 0; u < 3; ++u) bl[u] = warp_sum(bl[u]);
    const float lam = a.lam_prob ? a.lam_prob[a.lm_prob[j]] : a.lambda;
    h[0] += lam * a.dl2[3 * j];
    h[3] += lam * a.dl2[3 * j + 1];
    h[5] += lam * a.dl2[3 * j + 2];
    float Hi[9];
    if (!inv3_spd(h, Hi)) {
        if (lane == 0) atomicOr(a.err, ERRBIT_PRECOND);
        return;  // the landmark's terms are left out (flagged)
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) sHi[w][q] = Hi[q];
#pragma unroll
        for (int u = 0; u < 3; ++u) sYb[w][u] = Hi[3 * u] * bl[0] + Hi[3 * u + 1] * bl[1] + Hi[3 * u + 2] * bl[2];
    }
    __syncwarp();
    const float yb0 = sYb[w][0], yb1 = sYb[w][1], yb2 = sYb[w][2];
    // chunks of SC_KMAX observations: W_s staged, then the pairs of the chunk with every t >= s
    for (int c0 = 0; c0 < k; c0 += SC_KMAX) {
        // diagonal blocks, b~ and this chunk's W_s (recomputed)
        for (int t = c0 + lane; t < min(k, c0 + SC_KMAX); t += 32) {
            float r[2], Jp[18], Jl[6];
            sc_obs(a, s0 + t, j, r, Jp, Jl);
            float W[27], Y[27];  // W_s (9 x 3) and W_s H^-1
#pragma unroll
            for (int u = 0; u < 9; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) W[3 * u + v] = Jp[u] * Jl[v] + Jp[9 + u] * Jl[3 + v];
#pragma unroll
            for (int u = 0; u < 9; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v)
                    Y[3 * u + v] = W[3 * u] * Hi[v] + W[3 * u + 1] * Hi[3 + v] + W[3 * u + 2] * Hi[6 + v];
#pragma unroll
            for (int q = 0; q < 27; ++q) sW[w][t - c0][q] = W[q];
            const int cam = a.obs_cam_s[s0 + t];
            float* B = a.blk + 81LL * a.diag_blk[cam];
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                const float bp = Jp[u] * r[0] + Jp[9 + u] * r[1];
                atomicAdd(a.bt + 9 * cam + u, bp - (W[3 * u] * yb0 + W[3 * u + 1] * yb1 + W[3 * u + 2] * yb2));
#pragma unroll
                for (int v = 0; v < 9; ++v) {
                    const float jj = Jp[u] * Jp[v] + Jp[9 + u] * Jp[9 + v];
                    atomicAdd(B + 9 * u + v, jj - (Y[3 * u] * W[3 * v] + Y[3 * u + 1] * W[3 * v + 1] +
                                                   Y[3 * u + 2] * W[3 * v + 2]));
                }
            }
        }
        __syncwarp();
        // off-diagonal pairs (s, t), s in this chunk, s < t < k: t recomputed when outside the chunk
        for (int sl = c0; sl < min(k, c0 + SC_KMAX); ++sl) {
            float Y[27];
            {
                const float* W = sW[w][sl - c0];
#pragma unroll
                for (int u = 0; u < 9; ++u)
#pragma unroll
                    for (int v = 0; v < 3; ++v)
                        Y[3 * u + v] = W[3 * u] * Hi[v] + W[3 * u + 1] * Hi[3 + v] + W[3 * u + 2] * Hi[6 + v];
            }
            for (int t = sl + 1 + lane; t < k; t += 32) {
                float Wt[27];
                if (t < c0 + SC_KMAX) {
#pragma unroll
                    for (int q = 0; q < 27; ++q) Wt[q] = sW[w][t - c0][q];
                } else {
                    float r[2], Jp[18], Jl[6];
                    sc_obs(a, s0 + t, j, r, Jp, Jl);
#pragma unroll
                    for (int u = 0; u < 9; ++u)
#pragma unroll
                        for (int v = 0; v < 3; ++v) Wt[3 * u + v] = Jp[u] * Jl[v] + Jp[9 + u] * Jl[3 + v];
                }
                // pair index of (sl, t) within the landmark: pairs ordered by s, then t
                const int64_t pi = a.pair_off[j] + (int64_t)sl * k - (int64_t)sl * (sl + 1) / 2 + (t - sl - 1);
                float* Bab = a.blk + 81LL * a.pair_blk[2 * pi];
                float* Bba = a.blk + 81LL * a.pair_blk[2 * pi + 1];
#pragma unroll
                for (int u = 0; u < 9; ++u)
#pragma unroll
                    for (int v = 0; v < 9; ++v) {
                        const float val = -(Y[3 * u] * Wt[3 * v] + Y[3 * u + 1] * Wt[3 * v + 1] +
                                            Y[3 * u + 2] * Wt[3 * v + 2]);
                        atomicAdd(Bab + 9 * u + v, val);
                        atomicAdd(Bba + 9 * v + u, val);
                    }
            }
        }
        __syncwarp();
    }
}

// y = H~ v (both triangles stored): one thread per row
__global__ void __launch_bounds__(256)
k_sc_matvec(int n_cam, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
            const float* __restrict__ blk, const float* __restrict__ v, float* __restrict__ y,
            const PcgScalars* S) {
    if (S != nullptr && S->done) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= 9 * n_cam) return;
    const int a = row / 9, u = row - 9 * a;
    float acc = 0.f;
    for (int bi = row_ptr[a]; bi < row_ptr[a + 1]; ++bi) {
        const float* B = blk + 81LL * bi + 9 * u;
        const float* x = v + 9 * col[bi];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc += B[q] * __ldg(x + q);
    }
    y[row] += acc;
}

// the diagonal blocks and b~ as the 54 sums of the K3 finish (upper triangle, then g = -b~)
__global__ void k_sc_precond(int n_cam, const int32_t* __restrict__ diag_blk, const float* __restrict__ blk,
                             const float* __restrict__ bt, const float* __restrict__ dp2, float lam,
                             const float* __restrict__ lam_prob, const int32_t* __restrict__ cam_prob,
                             float* __restrict__ mdiag, float* __restrict__ minv, float* __restrict__ g,
                             uint32_t* err) {
    __shared__ float tot[56], sM[81], sL[81];
    const int cam = blockIdx.x, lane = threadIdx.x;
    const float* B = blk + 81LL * diag_blk[cam];
    if (lane == 0) {
        int q = 0;
        for (int u = 0; u < 9; ++u)
            for (int v = u; v < 9; ++v) tot[q++] = 0.5f * (B[9 * u + v] + B[9 * v + u]);
        for (int u = 0; u < 9; ++u) tot[45 + u] = bt[9 * cam + u];
    }
    __syncwarp();
    if (lam_prob) lam = lam_prob[cam_prob[cam]];
    precond_finish_warp(cam, tot, dp2, lam, mdiag, minv, g, err, sM, sL, lane);
}

// dl_j = -(H_ll + lambda D_l^2)^-1 (b_l + sum_s J_l,s^T J_p,s dp_s), one warp per landmark
__global__ void __launch_bounds__(32 * SC_WARPS) k_sc_backsub(ScArgs a, int n_pt, const float* __restrict__ dp,
                                                              float* __restrict__ dl) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * SC_WARPS + w;
    if (j >= n_pt) return;
    const int64_t s0 = a.pt_off[j];
    const int k = a.pt_off[j + 1] - (int)s0;
    float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
    for (int t = lane; t < k; t += 32) {
        float r[2], Jp[18], Jl[6];
        sc_obs(a, s0 + t, j, r, Jp, Jl);
        const float* d = dp + 9 * a.obs_cam_s[s0 + t];
        float q0 = r[0], q1 = r[1];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            q0 += Jp[c] * d[c];
            q1 += Jp[9 + c] * d[c];
        }
        int q = 0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            e[u] += Jl[u] * q0 + Jl[3 + u] * q1;
#pragma unroll
            for (int v = u; v < 3; ++v) h[q++] += Jl[u] * Jl[v] + Jl[3 + u] * Jl[3 + v];
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) h[q] = warp_sum(h[q]);
#pragma unroll
    for (int u = 0; u < 3; ++u) e[u] = warp_sum(e[u]);
    if (lane != 0) return;
    const float lam = a.lam_prob ? a.lam_prob[a.lm_prob[j]] : a.lambda;
    h[0] += lam * a.dl2[3 * j];
    h[3] += lam * a.dl2[3 * j + 1];
    h[5] += lam * a.dl2[3 * j + 2];
    float Hi[9];
    if (!inv3_spd(h, Hi)) {
        dl[3 * j] = dl[3 * j + 1] = dl[3 * j + 2] = 0.f;
        return;
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) dl[3 * j + u] = -(Hi[3 * u] * e[0] + Hi[3 * u + 1] * e[1] + Hi[3 * u + 2] * e[2]);
}

// D_l^2 = clamp(diag(J_l^T J_l)) per landmark (one warp each)
__global__ void __launch_bounds__(32 * SC_WARPS) k_sc_dl2(ScArgs a, int n_pt, float* __restrict__ dl2) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * SC_WARPS + w;
    if (j >= n_pt) return;
    const int64_t s0 = a.pt_off[j];
    const int k = a.pt_off[j + 1] - (int)s0;
    float d[3] = {0.f, 0.f, 0.f};
    for (int t = lane; t < k; t += 32) {
        float r[2], Jp[18], Jl[6];
        sc_obs(a, s0 + t, j, r, Jp, Jl);
#pragma unroll
        for (int u = 0; u < 3; ++u) d[u] += Jl[u] * Jl[u] + Jl[3 + u] * Jl[3 + u];
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) d[u] = warp_sum(d[u]);
    if (lane == 0)
        for (int u = 0; u < 3; ++u) dl2[3 * j + u] = fminf(fmaxf(d[u], 1e-6f), 1e32f);
}

ScArgs sc_args(Problem& p, float lambda) {
    return ScArgs{p.frames, p.pts, p.obs_cam_s, p.obs_xy_s, p.pt_off, p.dl2, lambda, p.batch.lam,
                  p.batch.lm_prob, (float)p.opt.huber_delta, p.sc_pair_off, p.sc_pair_blk, p.sc_diag_blk,
                  p.sc_blk, p.sc_bt, p.err};
}

}  // namespace

// Pattern of the explicit reduced camera system: a block (a, b) for every pair
// of cameras that share a landmark and every camera's diagonal; both
// triangles are stored (row-major block CSR), and every landmark pair (s < t)
// is mapped to its two blocks.  Host work, O(sum k^2).
void plan_schur(Problem& p, const std::vector<int32_t>& pt_off, const std::vector<int32_t>& obs_cam_s) {
    const int n_cam = p.n_cam;
    std::vector<std::vector<int32_t>> nb(n_cam);
    for (int a = 0; a < n_cam; ++a) nb[a].push_back(a);
    int64_t npair = 0;
    for (int j = 0; j < p.n_pt; ++j) {
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        npair += (int64_t)k * (k - 1) / 2;
        for (int s = 0; s < k; ++s)
            for (int t = 0; t < k; ++t)
                if (s != t) nb[obs_cam_s[s0 + s]].push_back(obs_cam_s[s0 + t]);
    }
    std::vector<int32_t> row_ptr(n_cam + 1, 0), col;
    for (int a = 0; a < n_cam; ++a) {
        std::sort(nb[a].begin(), nb[a].end());
        nb[a].erase(std::unique(nb[a].begin(), nb[a].end()), nb[a].end());
        row_ptr[a + 1] = row_ptr[a] + (int32_t)nb[a].size();
        col.insert(col.end(), nb[a].begin(), nb[a].end());
    }
    auto find = [&](int a, int b) {
        const auto it = std::lower_bound(col.begin() + row_ptr[a], col.begin() + row_ptr[a + 1], b);
        return (int32_t)(it - col.begin());
    };
    std::vector<int32_t> diag(n_cam), pair_blk(2 * std::max<int64_t>(npair, 1));
    std::vector<int64_t> pair_off(p.n_pt + 1, 0);
    for (int a = 0; a < n_cam; ++a) diag[a] = find(a, a);
    int64_t q = 0;
    for (int j = 0; j < p.n_pt; ++j) {
        pair_off[j] = q;
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        for (int s = 0; s < k; ++s)
            for (int t = s + 1; t < k; ++t) {
                const int a = obs_cam_s[s0 + s], b = obs_cam_s[s0 + t];
                pair_blk[2 * q] = find(a, b);
                pair_blk[2 * q + 1] = find(b, a);
                ++q;
            }
    }
    pair_off[p.n_pt] = q;
    p.sc_nblk = (int64_t)col.size();
    p.sc_row_ptr = dalloc<int32_t>(p, n_cam + 1);
    p.sc_col = dalloc<int32_t>(p, p.sc_nblk);
    p.sc_diag_blk = dalloc<int32_t>(p, n_cam);
    p.sc_pair_off = dalloc<int64_t>(p, p.n_pt + 1);
    p.sc_pair_blk = dalloc<int32_t>(p, 2 * std::max<int64_t>(npair, 1));
    p.sc_blk = dalloc<float>(p, 81 * p.sc_nblk);
    p.sc_bt = dalloc<float>(p, 9 * (int64_t)n_cam);
    BA_CUDA_TRY(cudaMemcpyAsync(p.sc_row_ptr, row_ptr.data(), sizeof(int32_t) * (n_cam + 1), cudaMemcpyHostToDevice,
                                p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(p.sc_col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice,
                                p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(p.sc_diag_blk, diag.data(), sizeof(int32_t) * n_cam, cudaMemcpyHostToDevice,
                                p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(p.sc_pair_off, pair_off.data(), sizeof(int64_t) * (p.n_pt + 1),
                                cudaMemcpyHostToDevice, p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(p.sc_pair_blk, pair_blk.data(), sizeof(int32_t) * pair_blk.size(),
                                cudaMemcpyHostToDevice, p.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
}

void launch_schur_dl2(Problem& p) {
    count_launches(p, 1);
    k_sc_dl2<<<ceil_div(p.n_pt, SC_WARPS), 32 * SC_WARPS, 0, p.stream>>>(sc_args(p, 0.f), p.n_pt, p.dl2);
    BA_LAUNCH_CHECK();
}

void launch_schur_assemble(Problem& p, float lambda) {
    count_launches(p, 3);
    BA_CUDA_TRY(cudaMemsetAsync(p.sc_blk, 0, sizeof(float) * 81 * p.sc_nblk, p.stream));
    BA_CUDA_TRY(cudaMemsetAsync(p.sc_bt, 0, sizeof(float) * 9 * p.n_cam, p.stream));
    k_sc_assemble<<<ceil_div(p.n_pt, SC_WARPS), 32 * SC_WARPS, 0, p.stream>>>(sc_args(p, lambda), p.n_pt);
    BA_LAUNCH_CHECK();
}

void launch_schur_precond(Problem& p) {
    count_launches(p, 1);
    k_sc_precond<<<p.n_cam, 32, 0, p.stream>>>(p.n_cam, p.sc_diag_blk, p.sc_blk, p.sc_bt, p.dp2,
                                               (float)p.lambda_damped, p.batch.lam, p.batch.cam_prob, p.mdiag,
                                               p.minv, p.g, p.err);
    BA_LAUNCH_CHECK();
}

void launch_schur_matvec(Problem& p, const float* v, float* y, const PcgScalars* S) {
    k_sc_matvec<<<ceil_div(9LL * p.n_cam, 256), 256, 0, p.stream>>>(p.n_cam, p.sc_row_ptr, p.sc_col, p.sc_blk, v, y,
                                                                    S);
    BA_LAUNCH_CHECK();
}

void launch_schur_backsub(Problem& p) {
    count_launches(p, 1);
    k_sc_backsub<<<ceil_div(p.n_pt, SC_WARPS), 32 * SC_WARPS, 0, p.stream>>>(sc_args(p, (float)p.lambda_damped),
                                                                             p.n_pt, p.x, p.dl);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
