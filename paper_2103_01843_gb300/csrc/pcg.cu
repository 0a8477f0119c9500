// K3-K5: block-Jacobi preconditioned CG on the reduced camera system
// (Sec. 5.4, Eq. cg_mult, Sec. 6.1), working only on the stored landmark
// blocks A_j = Q2^T J_p (2k x 9k, the last three rows being the rotated
// landmark-damping rows) and c_j = Q2^T r.
//
//   K3  M_i = sum_j A_ji^T A_ji + lambda D_p,i^2,  g_i = -sum_j A_ji^T c_j,
//       Cholesky-inverted per camera (the block diagonal of H~, Sec. 6.1)
//   K4  y = sum_j P_j^T A_j^T (A_j P_j v) + lambda D_p^2 v  (Eq. cg_mult; pose
//       damping added only in the product, Sec. 5.3)
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

__global__ void __launch_bounds__(32 * PC_WARPS)
k_precond_rhs(int n_cam, const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list,
              const int32_t* __restrict__ obs_pt_s, const int32_t* __restrict__ pt_off,
              const int64_t* __restrict__ a_off, const float* __restrict__ apool,
              const float* __restrict__ cpool, const float* __restrict__ dp2,
              const float lam, float* __restrict__ mdiag, float* __restrict__ minv,
              float* __restrict__ g, uint32_t* err) {
    __shared__ float part[PC_WARPS][54];
    __shared__ float tot[54];
    const int cam = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[45], accg[9];
#pragma unroll
    for (int i = 0; i < 45; ++i) acc[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) accg[i] = 0.f;
    for (int e = cam_off[cam] + w; e < cam_off[cam + 1]; e += PC_WARPS) {
        const int s = cam_list[e];
        const int j = obs_pt_s[s];
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        const int ncol = 9 * k;
        const float* Ab = apool + a_off[j] + 9 * (s - s0);
        const float* cj = cpool + 2 * (int64_t)s0;
        for (int row = lane; row < 2 * k; row += 32) {
            float a[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) a[c] = __ldg(Ab + (int64_t)row * ncol + c);
            const float cv = __ldg(cj + row);
            int t = 0;
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                accg[u] += a[u] * cv;
#pragma unroll
                for (int v = u; v < 9; ++v) acc[t++] += a[u] * a[v];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 45; ++i) {
        const float v = warp_sum(acc[i]);
        if (lane == 0) part[w][i] = v;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float v = warp_sum(accg[i]);
        if (lane == 0) part[w][45 + i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 54) {
        float s = 0.f;
        for (int m = 0; m < PC_WARPS; ++m) s += part[m][threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
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
}

// ---------------------------------------------------------------------------
// K4: y += sum_j A_j^T (A_j v_j)   (v_j = the landmark's camera sub-vector)
// One warp per landmark.  Row-wise single pass over A_j: u_r = A_j[r,:] v_j
// (warp reduction), then y_j += u_r A_j[r,:]; the 9k-entry y_j stays in
// registers (k <= MV_KREG) and is added into a per-CTA copy of y in shared
// memory, which is flushed to global memory once per CTA.  Larger k use two
// passes with u_j in shared memory.
// ---------------------------------------------------------------------------
constexpr int MV_WARPS = 8;
constexpr int MV_KREG = 64;              // 9k <= 576 -> 18 columns per lane
constexpr int MV_NM = (9 * MV_KREG + 31) / 32;
constexpr int MV_UCAP = 2 * 1024;        // shared u_j capacity per warp (k <= 1024)

template <bool SMEM_Y>
__global__ void __launch_bounds__(32 * MV_WARPS)
k_matvec(int n_cam, const int32_t* __restrict__ begin, const int32_t* __restrict__ pt_off,
         const int32_t* __restrict__ obs_cam_s, const int64_t* __restrict__ a_off,
         const float* __restrict__ apool, const float* __restrict__ v, float* __restrict__ y,
         const PcgScalars* __restrict__ S) {
    extern __shared__ float smem[];
    if (S != nullptr && S->done) return;
    float* ys = smem;                                    // 9 n_cam (SMEM_Y)
    float* ubuf = smem + (SMEM_Y ? 9 * n_cam : 0);       // per-warp u for big k
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (SMEM_Y) {
        for (int i = threadIdx.x; i < 9 * n_cam; i += blockDim.x) ys[i] = 0.f;
        __syncthreads();
    }
    const int jb = begin[blockIdx.x], je = begin[blockIdx.x + 1];
    for (int j = jb + w; j < je; j += MV_WARPS) {
        const int s0 = pt_off[j], k = pt_off[j + 1] - s0;
        const int ncol = 9 * k, nr = 2 * k;
        const float* __restrict__ Aj = apool + a_off[j];
        if (k <= MV_KREG) {
            float vr[MV_NM], yr[MV_NM];
            int yi[MV_NM];
#pragma unroll
            for (int m = 0; m < MV_NM; ++m) {
                const int col = lane + 32 * m;
                vr[m] = 0.f;
                yr[m] = 0.f;
                yi[m] = 0;
                if (col < ncol) {
                    const int s = col / 9;
                    yi[m] = 9 * obs_cam_s[s0 + s] + (col - 9 * s);
                    vr[m] = __ldg(v + yi[m]);
                }
            }
            for (int r = 0; r < nr; ++r) {
                const float* row = Aj + (int64_t)r * ncol;
                float a[MV_NM];
                float part = 0.f;
#pragma unroll
                for (int m = 0; m < MV_NM; ++m) {
                    const int col = lane + 32 * m;
                    a[m] = col < ncol ? __ldcs(row + col) : 0.f;
                    part += a[m] * vr[m];
                }
                const float u = warp_sum(part);
#pragma unroll
                for (int m = 0; m < MV_NM; ++m) yr[m] += u * a[m];
            }
#pragma unroll
            for (int m = 0; m < MV_NM; ++m) {
                const int col = lane + 32 * m;
                if (col < ncol) {
                    if (SMEM_Y) atomicAdd(ys + yi[m], yr[m]);
                    else atomicAdd(y + yi[m], yr[m]);
                }
            }
        } else {
            float* u = ubuf + w * MV_UCAP;
            for (int r = 0; r < nr; ++r) {
                const float* row = Aj + (int64_t)r * ncol;
                float part = 0.f;
                for (int col = lane; col < ncol; col += 32) {
                    const int s = col / 9;
                    part += row[col] * __ldg(v + 9 * obs_cam_s[s0 + s] + (col - 9 * s));
                }
                part = warp_sum(part);
                if (lane == 0) u[r] = part;
            }
            __syncwarp();
            for (int col = lane; col < ncol; col += 32) {
                float acc = 0.f;
                for (int r = 0; r < nr; ++r) acc += Aj[(int64_t)r * ncol + col] * u[r];
                const int s = col / 9;
                const int yi = 9 * obs_cam_s[s0 + s] + (col - 9 * s);
                if (SMEM_Y) atomicAdd(ys + yi, acc);
                else atomicAdd(y + yi, acc);
            }
            __syncwarp();
        }
    }
    if (SMEM_Y) {
        __syncthreads();
        for (int i = threadIdx.x; i < 9 * n_cam; i += blockDim.x) {
            const float val = ys[i];
            if (val != 0.f) atomicAdd(y + i, val);
        }
    }
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

__global__ void k_add_damping(int n, const float* __restrict__ dp2, float lam, const float* __restrict__ v,
                              float* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += lam * dp2[i] * v[i];
}

bool matvec_smem_y(const Problem& p) { return 9 * (int64_t)p.n_cam * 4 <= 96 * 1024; }

size_t matvec_smem(const Problem& p) {
    return (matvec_smem_y(p) ? 9 * (size_t)p.n_cam * 4 : 0) +
           (p.k_max > MV_KREG ? (size_t)MV_WARPS * MV_UCAP * 4 : 0);
}

void matvec_raw(Problem& p, const float* v, float* y, const PcgScalars* S) {
    const size_t sm = matvec_smem(p);
    if (matvec_smem_y(p)) {
        k_matvec<true><<<p.mv_grid, 32 * MV_WARPS, sm, p.stream>>>(p.n_cam, p.mv_begin, p.pt_off, p.obs_cam_s,
                                                                   p.a_off, p.apool, v, y, S);
    } else {
        k_matvec<false><<<p.mv_grid, 32 * MV_WARPS, sm, p.stream>>>(p.n_cam, p.mv_begin, p.pt_off,
                                                                    p.obs_cam_s, p.a_off, p.apool, v, y, S);
    }
    BA_LAUNCH_CHECK();
}

}  // namespace

int matvec_ctas_per_sm() { return 2; }

void configure_matvec(Problem& p) {
    const int sm = (int)matvec_smem(p);
    BA_CUDA_TRY(cudaFuncSetAttribute(k_matvec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_matvec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
}

void launch_precond_rhs(Problem& p) {
    count_launches(p, 1);
    k_precond_rhs<<<p.n_cam, 32 * PC_WARPS, 0, p.stream>>>(p.n_cam, p.cam_off, p.cam_list, p.obs_pt_s, p.pt_off,
                                                          p.a_off, p.apool, p.cpool, p.dp2, (float)p.lambda_damped, p.mdiag,
                                                          p.minv, p.g, p.err);
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
    matvec_raw(p, p.p, p.q, p.pcg);
    record(mv_end);
    k_pcg_update<<<1, PCG_T, 0, p.stream>>>(p.n_cam, p.g, p.dp2, p.minv, p.x, p.r, p.z, p.p, p.q, p.pcg);
    BA_LAUNCH_CHECK();
}

void launch_matvec(Problem& p, const float* v, float* y, bool add_damping) {
    count_launches(p, 1 + (add_damping ? 1 : 0));
    BA_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(float) * 9 * p.n_cam, p.stream));
    matvec_raw(p, v, y, nullptr);
    if (add_damping) {
        k_add_damping<<<ceil_div(9 * (int64_t)p.n_cam, 256), 256, 0, p.stream>>>(9 * p.n_cam, p.dp2,
                                                                                 (float)p.lambda_damped, v, y);
        BA_LAUNCH_CHECK();
    }
}

}  // namespace sqrtba
