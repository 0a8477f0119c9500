// Batches of independent problems solved together.  The problems are
// concatenated into one index space (cameras, landmarks and observations of
// problem b are contiguous), so every phase of the hot path is one launch
// over all problems: K1 and K2 run per landmark, K3 per observation and
// camera, and the K4 matvec is one persistent launch over the tiles of every
// problem's blocks (the reduced camera system of the batch is block
// diagonal).  What is per problem: the LM damping (K2, K3 and K5 read it per
// landmark / camera / problem), the CG scalars (one CTA per problem in K5),
// the FP64 energy and model-cost sums (one CTA per problem, fixed order) and
// the accept / reject decision with Nielsen's damping update (Sec. 6.1), here
// on the device, one thread per problem.
#include <algorithm>
#include <cmath>

#include "camera.cuh"
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int SEG_T = 256;

// E_b = sum ||r||^2 over the sorted observations of problem b (FP64)
__global__ void __launch_bounds__(SEG_T)
k_cost_seg(const int64_t* __restrict__ prob_obs_off, const float* __restrict__ frames, const float* __restrict__ pts,
           const int32_t* __restrict__ obs_cam_s, const int32_t* __restrict__ obs_pt_s,
           const float2* __restrict__ obs_xy_s, double* __restrict__ out, float huber) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    double acc = 0.0;
    for (int64_t s = prob_obs_off[b] + threadIdx.x; s < prob_obs_off[b + 1]; s += SEG_T) {
        const int j = obs_pt_s[s];
        const float2 z = obs_xy_s[s];
        float r0, r1;
        frame_residual(frames + FRAME * obs_cam_s[s], pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r0, r1);
        acc += energy_term(huber, r0, r1);
    }
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) out[b] = acc;
}

__global__ void k_batch_start(int n_prob, BatchLm* __restrict__ lm, const double* __restrict__ cost,
                              float* __restrict__ lam, double lambda0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_prob) return;
    BatchLm s{};
    s.lambda = lambda0;
    s.nu = 2.0;
    s.cost = cost[b];
    s.cost0 = cost[b];
    s.new_cost = cost[b];
    s.model_cost = cost[b];
    s.active = 1;
    s.finish = -1;
    lm[b] = s;
    lam[b] = (float)lambda0;
}

// Gain ratio rho = (E - E_new) / (E - L) in FP64; a step is accepted iff the
// model predicts a decrease (E - L > 0), E_new is finite and rho > 1e-3.
// Accept: lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2, stop when
// |E - E_new| / E < func_tol.  Reject: lambda *= nu, nu *= 2, stop at 1e32.
// Every linear solve counts as one LM iteration.
__global__ void k_batch_decide(int n_prob, BatchLm* __restrict__ lm, const double* __restrict__ cand_cost,
                               const double* __restrict__ model, const PcgScalars* __restrict__ pcg,
                               float* __restrict__ lam, int max_lm_iters, double func_tol, int iteration,
                               int32_t* __restrict__ n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_prob) return;
    BatchLm s = lm[b];
    s.last_acc = 0;
    if (s.active) {
        const double E = s.cost, L = model[b], En = cand_cost[b];
        const double rho = (E - En) / (E - L);
        const bool acc = isfinite(En) && isfinite(rho) && (E - L) > 0.0 && rho > 1e-3;
        s.new_cost = En;
        s.model_cost = L;
        s.cg_total += pcg[b].it;
        s.iter += 1;
        int stop = 0;
        if (acc) {
            s.accepted += 1;
            s.cost = En;
            const double t = 2.0 * rho - 1.0;
            s.lambda *= fmax(1.0 / 3.0, 1.0 - t * t * t);
            s.lambda = fmax(s.lambda, 1e-16);
            s.nu = 2.0;
            if (fabs(E - En) / E < func_tol) stop = 1;
        } else {
            s.lambda *= s.nu;
            s.nu *= 2.0;
            if (s.lambda >= 1e32) {
                s.lambda = 1e32;
                stop = 3;
            }
        }
        if (stop == 0 && s.iter >= max_lm_iters) stop = 2;
        s.last_acc = acc ? 1 : 0;
        if (stop) {
            s.stop = stop;
            s.active = 0;
            s.finish = iteration;
        }
        lam[b] = (float)s.lambda;
    }
    lm[b] = s;
    if (s.active) atomicAdd(n_active, 1);
}

// accepted problems take their candidate state
__global__ void k_batch_commit(int n_cam, int n_pt, const int32_t* __restrict__ cam_prob,
                               const int32_t* __restrict__ lm_prob, const BatchLm* __restrict__ lm,
                               float* __restrict__ cams, const float* __restrict__ cand_cams, float* __restrict__ pts,
                               const float* __restrict__ cand_pts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cam && lm[cam_prob[i]].last_acc)
        for (int m = 0; m < 9; ++m) cams[9 * i + m] = cand_cams[9 * i + m];
    if (i < n_pt && lm[lm_prob[i]].last_acc)
        for (int m = 0; m < 3; ++m) pts[3 * i + m] = cand_pts[3 * i + m];
}

}  // namespace

void launch_batch_cost(Problem& p, bool candidate, double* out) {
    BatchState& B = p.batch;
    count_launches(p, 1);
    if (!candidate) launch_frames(p);
    k_cost_seg<<<B.n_prob, SEG_T, 0, p.stream>>>(B.prob_obs_off, candidate ? p.cand_frames : p.frames,
                                                 candidate ? p.cand_pts : p.pts, p.obs_cam_s, p.obs_pt_s,
                                                 p.obs_xy_s, out, (float)p.opt.huber_delta);
    BA_LAUNCH_CHECK();
}

void launch_batch_start(Problem& p) {
    BatchState& B = p.batch;
    count_launches(p, 1);
    k_batch_start<<<ceil_div(B.n_prob, 128), 128, 0, p.stream>>>(B.n_prob, B.lm, B.cost_a, B.lam, p.opt.lambda0);
    BA_LAUNCH_CHECK();
}

void launch_batch_decide(Problem& p, int iteration) {
    BatchState& B = p.batch;
    count_launches(p, 1);
    BA_CUDA_TRY(cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), p.stream));
    k_batch_decide<<<ceil_div(B.n_prob, 128), 128, 0, p.stream>>>(B.n_prob, B.lm, B.cost_a, B.cost_b, B.pcg, B.lam,
                                                                 p.opt.max_lm_iters, p.opt.func_tol, iteration,
                                                                 B.n_active);
    BA_LAUNCH_CHECK();
}

void launch_batch_commit(Problem& p) {
    BatchState& B = p.batch;
    count_launches(p, 1);
    const int n = std::max(p.n_cam, p.n_pt);
    k_batch_commit<<<ceil_div(n, 256), 256, 0, p.stream>>>(p.n_cam, p.n_pt, B.cam_prob, B.lm_prob, B.lm, p.cams,
                                                          p.cand_cams, p.pts, p.cand_pts);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
