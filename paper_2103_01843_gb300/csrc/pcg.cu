// K3-K5: block-Jacobi preconditioned CG on the reduced camera system
// (Sec. 5.4, Eq. cg_mult, Sec. 6.1), working only on the stored landmark
// blocks A_j = Q2^T J_p (2k x 9k, the last three rows being the rotated
// landmark-damping rows) and c_j = Q2^T r.
//
//   K3  M_i = sum_j A_ji^T A_ji + lambda D_p,i^2,  g_i = -sum_j A_ji^T c_j,
//       Cholesky-inverted per camera (the block diagonal of H~, Sec. 6.1):
//       per-observation records from the tile pipeline (matvec.cu), summed
//       here per camera in a fixed order
//   K4  y = sum_j P_j^T A_j^T (A_j P_j v) (matvec.cu) + lambda D_p^2 v, the pose
//       damping added only in the product (Sec. 5.3), inside K5
//   K5  the CG recursion with the Nash-Sofer stop
//       i (Q_i - Q_{i-1}) / Q_i < eta, Q(x) = 1/2 x^T H~ x - g^T x = -1/2 x^T (g + r).
#include <algorithm>

#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int PC_WARPS = 8;

// ---------------------------------------------------------------------------
// K3: per-camera preconditioner block and right-hand side
// ---------------------------------------------------------------------------
__device__ int cholesky_inverse9(const float* M, float* Minv) {
    float L[81];
    for (int i = 0; i < 81; ++i) L[i] = 0.f;
    for (int jj = 0; jj < 9; ++jj) {
        float s = M[jj * 9 + jj];
        for (int m = 0; m < jj; ++m) s -= L[jj * 9 + m] * L[jj * 9 + m];
        if (!(s > 0.f)) return -1;
        const float l = sqrtf(s);
        L[jj * 9 + jj] = l;
        for (int i = jj + 1; i < 9; ++i) {
            float t = M[i * 9 + jj];
            for (int m = 0; m < jj; ++m) t -= L[i * 9 + m] * L[jj * 9 + m];
            L[i * 9 + jj] = t / l;
        }
    }
    // columns of M^-1: solve L L^T x = e_c
    for (int c = 0; c < 9; ++c) {
        float y[9];
        for (int i = 0; i < 9; ++i) {
            float s = i == c ? 1.f : 0.f;
            for (int m = 0; m < i; ++m) s -= L[i * 9 + m] * y[m];
            y[i] = s / L[i * 9 + i];
        }
        for (int i = 8; i >= 0; --i) {
            float s = y[i];
            for (int m = i + 1; m < 9; ++m) s -= L[m * 9 + i] * y[m];
            y[i] = s / L[i * 9 + i];
        }
        for (int i = 0; i < 9; ++i) Minv[i * 9 + c] = y[i];
    }
    return 0;
}

// Second half of K3: per camera, the 54 sums (upper triangle of
// sum_j A_ji^T A_ji and sum_j A_ji^T c_j) are formed in a fixed order, lambda
// D_p^2 is added and the 9x9 block inverted by Cholesky.
__device__ void finish_block(int cam, const float* tot, const float* __restrict__ dp2, float lam,
                             float* __restrict__ mdiag, float* __restrict__ minv, float* __restrict__ g,
                             uint32_t* err) {
    float M[81], Mi[81];
    int t = 0;
    for (int u = 0; u < 9; ++u)
        for (int v = u; v < 9; ++v) {
            M[u * 9 + v] = tot[t];
            M[v * 9 + u] = tot[t];
            ++t;
        }
    for (int u = 0; u < 9; ++u) M[u * 9 + u] += lam * dp2[9 * cam + u];
    for (int i = 0; i < 81; ++i) mdiag[81 * (int64_t)cam + i] = M[i];
    if (cholesky_inverse9(M, Mi) != 0) {
        // not positive definite in FP32: fall back to the diagonal (Jacobi)
        atomicOr(err, ERRBIT_PRECOND);
        for (int i = 0; i < 81; ++i) Mi[i] = 0.f;
        for (int u = 0; u < 9; ++u) Mi[u * 9 + u] = M[u * 9 + u] > 0.f ? 1.f / M[u * 9 + u] : 0.f;
    }
    for (int i = 0; i < 81; ++i) minv[81 * (int64_t)cam + i] = Mi[i];
    for (int u = 0; u < 9; ++u) g[9 * cam + u] = -tot[45 + u];
}

// from per-observation records: one warp reads one record (27 float2 lanes)
__global__ void __launch_bounds__(32 * PC_WARPS)
k_precond_reduce(int n_cam, const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list_st,
                 const float* __restrict__ rec, const float* __restrict__ dp2, const float lam,
                 float* __restrict__ mdiag, float* __restrict__ minv, float* __restrict__ g, uint32_t* err) {
    __shared__ float2 part[PC_WARPS][27];
    __shared__ float tot[54];
    const int cam = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 acc = make_float2(0.f, 0.f);
    if (lane < 27) {
        for (int e = cam_off[cam] + w; e < cam_off[cam + 1]; e += PC_WARPS) {
            const float2 r = __ldg(reinterpret_cast<const float2*>(rec + (int64_t)cam_list_st[e] * 54) + lane);
            acc.x += r.x;
            acc.y += r.y;
        }
        part[w][lane] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 27) {
        float2 s2 = make_float2(0.f, 0.f);
        for (int m = 0; m < PC_WARPS; ++m) {
            s2.x += part[m][threadIdx.x].x;
            s2.y += part[m][threadIdx.x].y;
        }
        tot[2 * threadIdx.x] = s2.x;
        tot[2 * threadIdx.x + 1] = s2.y;
    }
    __syncthreads();
    if (threadIdx.x == 0) finish_block(cam, tot, dp2, lam, mdiag, minv, g, err);
}

// from per-CTA partial blocks (grid x 54 n_cam), summed in CTA order
__global__ void __launch_bounds__(64)
k_precond_reduce_partials(int n_cam, int grid, const float* __restrict__ mpart, const float* __restrict__ dp2,
                          const float lam, float* __restrict__ mdiag, float* __restrict__ minv,
                          float* __restrict__ g, uint32_t* err) {
    __shared__ float tot[54];
    const int cam = blockIdx.x;
    if (threadIdx.x < 54) {
        float acc = 0.f;
        const float* src = mpart + (int64_t)cam * 54 + threadIdx.x;
        for (int b = 0; b < grid; ++b) acc += __ldg(src + (int64_t)b * 54 * n_cam);
        tot[threadIdx.x] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) finish_block(cam, tot, dp2, lam, mdiag, minv, g, err);
}

// ---------------------------------------------------------------------------
// K5: the CG recursion, one CTA (the vectors hold 9 n_cam floats)
// ---------------------------------------------------------------------------
constexpr int PCG_T = 1024;

__device__ __forceinline__ void precond_apply(int n_cam, const float* __restrict__ minv,
                                              const float* __restrict__ r, float* __restrict__ z,
                                              float& rz) {
    for (int i = threadIdx.x; i < 9 * n_cam; i += PCG_T) {
        const int cam = i / 9, row = i - 9 * cam;
        const float* Mi = minv + 81 * (int64_t)cam + 9 * row;
        const float* rc = r + 9 * cam;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) s += Mi[c] * rc[c];
        z[i] = s;
        rz += r[i] * s;
    }
}

__global__ void __launch_bounds__(PCG_T)
k_pcg_init(int n_cam, const float* __restrict__ g, const float* __restrict__ minv, float* x, float* r,
           float* z, float* p, float* q, PcgScalars* S, float lambda, float eta, int max_it) {
    __shared__ float red[32];
    const int n = 9 * n_cam;
    float gg = 0.f;
    for (int i = threadIdx.x; i < n; i += PCG_T) {
        const float gi = g[i];
        x[i] = 0.f;
        r[i] = gi;
        q[i] = 0.f;
        gg += gi * gi;
    }
    __syncthreads();
    float rz = 0.f;
    precond_apply(n_cam, minv, r, z, rz);
    gg = block_sum(gg, red);
    rz = block_sum(rz, red);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += PCG_T) p[i] = z[i];
    if (threadIdx.x == 0) {
        S->rho = rz;
        S->q_prev = 0.f;
        S->gnorm = sqrtf(gg);
        S->rnorm = sqrtf(gg);
        S->lambda = lambda;
        S->eta = eta;
        S->it = 0;
        S->max_it = max_it;
        S->done = (gg > 0.f && rz > 0.f) ? 0 : 1;
        S->stop = (gg > 0.f && rz > 0.f) ? -1 : 4;
    }
}

__global__ void __launch_bounds__(PCG_T)
k_pcg_update(int n_cam, const float* __restrict__ g, const float* __restrict__ dp2,
             const float* __restrict__ minv, float* x, float* r, float* z, float* p, float* q,
             PcgScalars* S) {
    __shared__ float red[32];
    if (S->done) return;
    const int n = 9 * n_cam;
    const float lam = S->lambda;
    const float rho = S->rho;
    float pq = 0.f;
    for (int i = threadIdx.x; i < n; i += PCG_T) {
        const float qi = q[i] + lam * dp2[i] * p[i];
        q[i] = qi;
        pq += p[i] * qi;
    }
    pq = block_sum(pq, red);
    if (!(pq > 0.f)) {
        if (threadIdx.x == 0) {
            S->done = 1;
            S->stop = 3;
        }
        return;
    }
    const float alpha = rho / pq;
    float rr = 0.f, xgr = 0.f;
    for (int i = threadIdx.x; i < n; i += PCG_T) {
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
    if (stop >= 0) return;
    float rz = 0.f;
    precond_apply(n_cam, minv, r, z, rz);
    rz = block_sum(rz, red);
    const float beta = rz / rho;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += PCG_T) {
        p[i] = z[i] + beta * p[i];
        q[i] = 0.f;
    }
    if (threadIdx.x == 0) S->rho = rz;
}

}  // namespace

void launch_precond_rhs(Problem& p) {
    if (launch_precond_records(p)) {
        count_launches(p, 2);
        k_precond_reduce_partials<<<p.n_cam, 64, 0, p.stream>>>(p.n_cam, p.mv_grid, p.mpart, p.dp2,
                                                                (float)p.lambda_damped, p.mdiag, p.minv, p.g, p.err);
    } else {
        count_launches(p, 2 + (p.n_obs_direct_big > 0 ? 1 : 0));
        k_precond_reduce<<<p.n_cam, 32 * PC_WARPS, 0, p.stream>>>(p.n_cam, p.cam_off, p.cam_list_st, p.prec, p.dp2,
                                                                 (float)p.lambda_damped, p.mdiag, p.minv, p.g, p.err);
    }
    BA_LAUNCH_CHECK();
}

void launch_pcg_init(Problem& p) {
    count_launches(p, 1);
    k_pcg_init<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, p.minv, p.x, p.r, p.z, p.p, p.q, p.pcg,
                                          (float)p.lambda_damped, (float)p.opt.cg_eta, p.opt.max_cg_iters);
    BA_LAUNCH_CHECK();
}

void launch_pcg_iteration(Problem& p, cudaEvent_t mv_begin, cudaEvent_t mv_end) {
    count_launches(p, 2);
    auto record = [&](cudaEvent_t ev) {
        if (!ev) return;
        if (p.capturing) BA_CUDA_TRY(cudaEventRecordWithFlags(ev, p.stream, cudaEventRecordExternal));
        else BA_CUDA_TRY(cudaEventRecord(ev, p.stream));
    };
    record(mv_begin);
    launch_matvec_raw(p, p.p, p.q, p.pcg);
    record(mv_end);
    k_pcg_update<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, p.dp2, p.minv, p.x, p.r, p.z, p.p, p.q, p.pcg);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
