// Implicit landmark blocks: the storage variant of Sec. 5.1 / Table
// tab:complexities that keeps the factorisation of each landmark block
// instead of Q2^T J_p.  Per observation (storage order, 24 floats): its two
// pose Jacobian rows J_s (2 x 9) and its two rows of the Householder vectors
// V (2 x 3); per landmark (storage position, LM_REC floats): the compact-WY
// factor Tm (Q^T = I - V Tm^T V^T, upper triangular) and, after the landmark
// damping, S = G_dt^T G_dt, G_tt and the damped R (the 6 Givens rotations G of
// Sec. 5.3 act on the 3 top rows and the 3 damping rows; G_tt / G_dt are the
// blocks of G that map the undamped top rows to the new top / damping rows).
// The matvec reads Tm and S (48 bytes) of the record.
//
// Products with A_j = the rows of Q^ T [J_p; 0] below the top rows:
//     A_j^T A_j v = J_p^T Q diag(S, I) Q^T J_p v
// because the damping rows [0 | sqrt(lambda) D_l | 0] carry no pose entries:
// after the rotations the top rows are dropped (Eq. reduced), the damping rows
// keep G_dt times the top entries, so the top three entries of Q^T u enter
// through S and all others unchanged.  Per landmark: u = J_p v (2k), two
// reductions over its rows (V^T u, V^T z), no block is formed.  Reads 100 bytes
// per observation and 48 per landmark instead of 72 k bytes per observation.
//
// Work: warps over tasks of landmarks of equal k in storage order (decreasing
// k); k <= 32: teams of W = 2, 4, 8, 16 or 32 lanes (W >= k), one landmark per
// team and one observation per lane; k > 32: one warp per landmark, lanes over
// its observations in chunks of 32 (three passes over the records).  y is
// accumulated in shared memory when it fits (9 n_cam floats), flushed once per
// CTA, else in global memory; v is staged in shared memory beside it when both
// fit (see implicit_mode).
#include <algorithm>
#include <vector>

#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int IM_WARPS = 16;
constexpr int IM_THREADS = 32 * IM_WARPS;
constexpr int IM_SMEM_Y_MAX = 200 * 1024;  // bytes of shared y (9 n_cam floats) at most

struct ImTask {
    int32_t so0;   // storage index of the first observation of the first landmark
    int32_t pos0;  // storage position of the first landmark
    int16_t k;     // observations per landmark
    int16_t n;     // landmarks in the task
    int32_t pad;
};
static_assert(sizeof(ImTask) == 16, "task record");

struct ImArgs {
    const ImTask* tasks;
    int n_tasks;
    int n_big;             // tasks [0, n_big) have k > 32 (one landmark each), taken dynamically
    unsigned* ctr;         // [0] next big task, [32] CTAs done (both zero between launches)
    float* pq_part;        // non-null: per-CTA sums of ||A_j v||^2 (the CG's p^T A^T A p as a sum of squares)
    const float4* ipool;   // 6 float4 chunks per observation, chunk m at m * n_obs
    int64_t n_obs;
    const float* lmrec;    // LM_REC floats per storage position (Tm and S read here)
    const int32_t* mv_cam;
    const float* v;
    float* y;
    int n_cam;
    const PcgScalars* S;
    const BatchLm* blm;      // batch: per-problem LM state (null for a single problem)
    const int32_t* lm_prob;  // batch: problem of every landmark
    const int32_t* lm_by_k;  // landmark at every storage position
};

__host__ __device__ constexpr int team_width(int k) { return k <= 2 ? 2 : (k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32))); }

// one observation record: J rows (18) and V rows (6)
struct ObsRec {
    float J[18];
    float V[6];
};

__device__ __forceinline__ void load_rec(const ImArgs& a, int64_t so, ObsRec& r) {
    float f[24];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const float4 c = __ldg(a.ipool + m * a.n_obs + so);
        f[4 * m] = c.x;
        f[4 * m + 1] = c.y;
        f[4 * m + 2] = c.z;
        f[4 * m + 3] = c.w;
    }
#pragma unroll
    for (int i = 0; i < 18; ++i) r.J[i] = f[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) r.V[i] = f[18 + i];
}

template <int W>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct LmFactors {
    float T00, T01, T02, T11, T12, T22;  // Tm, upper
    float S00, S01, S02, S11, S12, S22;  // S, symmetric
};

__device__ __forceinline__ LmFactors load_factors(const float* lmrec, int pos) {
    const float4* p = reinterpret_cast<const float4*>(lmrec + (int64_t)LM_REC * pos);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    return LmFactors{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

__device__ __forceinline__ void accumulate_y(float* yt, int cam, const ObsRec& r, float w0, float w1) {
    float* y = yt + 9 * cam;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float val = r.J[c] * w0 + r.J[9 + c] * w1;
        atomicAdd(y + c, val);
    }
}

// v element i: shared memory (SV) or the read-only global path
template <bool SV>
__device__ __forceinline__ float load_v(const float* vt, int i) {
    if constexpr (SV) return vt[i];
    else return __ldg(vt + i);
}

// k <= 32: teams of W lanes, lane t of a team holds observation t (rows 2t, 2t+1)
template <int W, bool SV>
__device__ void small_task(const ImArgs& a, const ImTask& tk, const float* vt, float* yt, int lane, float& pqa) {
    const int team = lane / W, t = lane - team * W, base = team * W;
    const int k = tk.k;
    const bool has = team < tk.n;
    // a stopped problem of a batch contributes nothing (its CG has stopped)
    const bool act = has && t < k && (!a.blm || batch_active(a.blm, a.lm_prob[a.lm_by_k[tk.pos0 + team]]));
    ObsRec r;
    float vv[9];
    int cam = 0;
    const int64_t so = (int64_t)tk.so0 + (int64_t)team * k + t;
    if (act) {
        load_rec(a, so, r);
        cam = __ldg(a.mv_cam + so);
#pragma unroll
        for (int c = 0; c < 9; ++c) vv[c] = load_v<SV>(vt, 9 * cam + c);
    } else {
#pragma unroll
        for (int i = 0; i < 18; ++i) r.J[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) r.V[i] = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) vv[c] = 0.f;
    }
    const LmFactors F = load_factors(a.lmrec, has ? tk.pos0 + team : tk.pos0);
    // u = J_p v (this lane's two rows)
    float u0 = 0.f, u1 = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        u0 += r.J[c] * vv[c];
        u1 += r.J[9 + c] * vv[c];
    }
    // z = Q^T u = u - V Tm^T (V^T u)
    float p0 = r.V[0] * u0 + r.V[3] * u1, p1 = r.V[1] * u0 + r.V[4] * u1, p2 = r.V[2] * u0 + r.V[5] * u1;
    p0 = team_sum<W>(p0);
    p1 = team_sum<W>(p1);
    p2 = team_sum<W>(p2);
    const float h0 = F.T00 * p0, h1 = F.T01 * p0 + F.T11 * p1, h2 = F.T02 * p0 + F.T12 * p1 + F.T22 * p2;
    float z0 = u0 - (r.V[0] * h0 + r.V[1] * h1 + r.V[2] * h2);
    float z1 = u1 - (r.V[3] * h0 + r.V[4] * h1 + r.V[5] * h2);
    // ||A_j v||^2: the rows below the top three, squared, ...
    if (act) pqa += t >= 2 ? z0 * z0 + z1 * z1 : (t == 1 ? z1 * z1 : 0.f);
    // top rows 0, 1 (lane t = 0) and 2 (lane t = 1) enter through S
    const float zt0 = __shfl_sync(0xffffffffu, z0, base), zt1 = __shfl_sync(0xffffffffu, z1, base);
    const float zt2 = __shfl_sync(0xffffffffu, z0, base + 1);
    if (t == 0) {
        z0 = F.S00 * zt0 + F.S01 * zt1 + F.S02 * zt2;
        z1 = F.S01 * zt0 + F.S11 * zt1 + F.S12 * zt2;
        // ... and the top entries through S
        if (act) pqa += zt0 * z0 + zt1 * z1 + zt2 * (F.S02 * zt0 + F.S12 * zt1 + F.S22 * zt2);
    } else if (t == 1) {
        z0 = F.S02 * zt0 + F.S12 * zt1 + F.S22 * zt2;
    }
    // w = Q z = z - V Tm (V^T z)
    float q0 = r.V[0] * z0 + r.V[3] * z1, q1 = r.V[1] * z0 + r.V[4] * z1, q2 = r.V[2] * z0 + r.V[5] * z1;
    q0 = team_sum<W>(q0);
    q1 = team_sum<W>(q1);
    q2 = team_sum<W>(q2);
    const float g0 = F.T00 * q0 + F.T01 * q1 + F.T02 * q2, g1 = F.T11 * q1 + F.T12 * q2, g2 = F.T22 * q2;
    const float w0 = z0 - (r.V[0] * g0 + r.V[1] * g1 + r.V[2] * g2);
    const float w1 = z1 - (r.V[3] * g0 + r.V[4] * g1 + r.V[5] * g2);
    if (act) accumulate_y(yt, cam, r, w0, w1);
}

// k > 32: one warp, lanes over the observations in chunks of 32
template <bool SV>
__device__ void big_task(const ImArgs& a, const ImTask& tk, const float* vt, float* yt, int lane, float& pqa) {
    const int k = tk.k;
    if (a.blm && !batch_active(a.blm, a.lm_prob[a.lm_by_k[tk.pos0]])) return;  // whole warp
    const LmFactors F = load_factors(a.lmrec, tk.pos0);
    auto load = [&](int t, ObsRec& r, float (&vv)[9], int& cam) {
        const int64_t so = (int64_t)tk.so0 + t;
        load_rec(a, so, r);
        cam = __ldg(a.mv_cam + so);
#pragma unroll
        for (int c = 0; c < 9; ++c) vv[c] = load_v<SV>(vt, 9 * cam + c);
    };
    // pass 1: V^T u
    float p0 = 0.f, p1 = 0.f, p2 = 0.f;
    for (int t = lane; t < k; t += 32) {
        ObsRec r;
        float vv[9];
        int cam;
        load(t, r, vv, cam);
        float u0 = 0.f, u1 = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            u0 += r.J[c] * vv[c];
            u1 += r.J[9 + c] * vv[c];
        }
        p0 += r.V[0] * u0 + r.V[3] * u1;
        p1 += r.V[1] * u0 + r.V[4] * u1;
        p2 += r.V[2] * u0 + r.V[5] * u1;
    }
    p0 = warp_sum(p0);
    p1 = warp_sum(p1);
    p2 = warp_sum(p2);
    const float h0 = F.T00 * p0, h1 = F.T01 * p0 + F.T11 * p1, h2 = F.T02 * p0 + F.T12 * p1 + F.T22 * p2;
    auto zrows = [&](const ObsRec& r, const float (&vv)[9], float& z0, float& z1) {
        float u0 = 0.f, u1 = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            u0 += r.J[c] * vv[c];
            u1 += r.J[9 + c] * vv[c];
        }
        z0 = u0 - (r.V[0] * h0 + r.V[1] * h1 + r.V[2] * h2);
        z1 = u1 - (r.V[3] * h0 + r.V[4] * h1 + r.V[5] * h2);
    };
    // the top entries (rows 0, 1 of observation 0, row 0 of observation 1)
    float zt0, zt1, zt2;
    {
        float z0 = 0.f, z1 = 0.f;
        if (lane < 2) {
            ObsRec r;
            float vv[9];
            int cam;
            load(lane, r, vv, cam);
            zrows(r, vv, z0, z1);
        }
        zt0 = __shfl_sync(0xffffffffu, z0, 0);
        zt1 = __shfl_sync(0xffffffffu, z1, 0);
        zt2 = __shfl_sync(0xffffffffu, z0, 1);
    }
    const float s0 = F.S00 * zt0 + F.S01 * zt1 + F.S02 * zt2;
    const float s1 = F.S01 * zt0 + F.S11 * zt1 + F.S12 * zt2;
    const float s2 = F.S02 * zt0 + F.S12 * zt1 + F.S22 * zt2;
    if (lane == 0) pqa += zt0 * s0 + zt1 * s1 + zt2 * s2;  // ||A_j v||^2: the top entries through S
    // pass 2: V^T z with the top entries replaced
    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
    for (int t = lane; t < k; t += 32) {
        ObsRec r;
        float vv[9];
        int cam;
        load(t, r, vv, cam);
        float z0, z1;
        zrows(r, vv, z0, z1);
        pqa += t >= 2 ? z0 * z0 + z1 * z1 : (t == 1 ? z1 * z1 : 0.f);  // and the rows below them
        if (t == 0) {
            z0 = s0;
            z1 = s1;
        } else if (t == 1) {
            z0 = s2;
        }
        q0 += r.V[0] * z0 + r.V[3] * z1;
        q1 += r.V[1] * z0 + r.V[4] * z1;
        q2 += r.V[2] * z0 + r.V[5] * z1;
    }
    q0 = warp_sum(q0);
    q1 = warp_sum(q1);
    q2 = warp_sum(q2);
    const float g0 = F.T00 * q0 + F.T01 * q1 + F.T02 * q2, g1 = F.T11 * q1 + F.T12 * q2, g2 = F.T22 * q2;
    // pass 3: w = Q z, y += J^T w
    for (int t = lane; t < k; t += 32) {
        ObsRec r;
        float vv[9];
        int cam;
        load(t, r, vv, cam);
        float z0, z1;
        zrows(r, vv, z0, z1);
        if (t == 0) {
            z0 = s0;
            z1 = s1;
        } else if (t == 1) {
            z0 = s2;
        }
        const float w0 = z0 - (r.V[0] * g0 + r.V[1] * g1 + r.V[2] * g2);
        const float w1 = z1 - (r.V[3] * g0 + r.V[4] * g1 + r.V[5] * g2);
        accumulate_y(yt, cam, r, w0, w1);
    }
}

// SMEM_Y: y accumulated in shared memory (flushed once per CTA); SMEM_V: v
// staged in shared memory too (one coalesced copy per CTA: the nine gathers of
// an observation's camera then hit shared memory, not 32-sector L1 requests).
// NT threads per CTA: 512 (two CTAs per SM) or 1024 (one, when y and v do
// not fit twice).
template <bool SMEM_Y, bool SMEM_V, int NT>
__device__ __forceinline__ void matvec_body(const ImArgs& a, float* ys) {
    const int acc_n = 9 * a.n_cam;
    float* vs = ys + (SMEM_Y ? acc_n : 0);
    if (SMEM_Y)
        for (int i = threadIdx.x; i < acc_n; i += NT) ys[i] = 0.f;
    if (SMEM_V)
        for (int i = threadIdx.x; i < acc_n; i += NT) vs[i] = __ldg(a.v + i);
    if (SMEM_Y || SMEM_V) __syncthreads();
    float* yt = SMEM_Y ? ys : a.y;
    const float* vt = SMEM_V ? vs : a.v;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (NT / 32) + (threadIdx.x >> 5), nw = gridDim.x * (NT / 32);
    float pqa = 0.f;
    // the k <= 32 tasks statically, round robin over the warps ...
    for (int ti = a.n_big + gw; ti < a.n_tasks; ti += nw) {
        const ImTask tk = a.tasks[ti];
        switch (team_width(tk.k)) {
            case 2: small_task<2, SMEM_V>(a, tk, vt, yt, lane, pqa); break;
            case 4: small_task<4, SMEM_V>(a, tk, vt, yt, lane, pqa); break;
            case 8: small_task<8, SMEM_V>(a, tk, vt, yt, lane, pqa); break;
            case 16: small_task<16, SMEM_V>(a, tk, vt, yt, lane, pqa); break;
            default: small_task<32, SMEM_V>(a, tk, vt, yt, lane, pqa); break;
        }
    }
    // ... then the k > 32 ones (three passes each, up to k = 900) one at a time
    // to whichever warp asks next, so that they do not set the kernel's tail
    // (a plain read first: once they are gone no warp queues on the atomic)
    if (a.n_big > 0) {
        for (;;) {
            unsigned ti = (unsigned)a.n_big;
            if (lane == 0 && *(volatile unsigned*)a.ctr < (unsigned)a.n_big) ti = atomicAdd(a.ctr, 1u);
            ti = __shfl_sync(0xffffffffu, ti, 0);
            if (ti >= (unsigned)a.n_big) break;
            big_task<SMEM_V>(a, a.tasks[ti], vt, yt, lane, pqa);
        }
        // the last CTA to finish resets the counters for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(a.ctr + 32, 1u) == gridDim.x - 1) {
                atomicExch(a.ctr, 0u);
                atomicExch(a.ctr + 32, 0u);
            }
        }
    }
    if (a.pq_part) {  // this CTA's share of p^T A^T A p (summed by the CG update in CTA order)
        __shared__ float red[32];
        pqa = block_sum(pqa, red);
        if (threadIdx.x == 0) a.pq_part[blockIdx.x] = pqa;
    }
    if (SMEM_Y) {
        __syncthreads();
        const int i0 = (int)(((int64_t)blockIdx.x * acc_n) / gridDim.x);
        for (int q = threadIdx.x; q < acc_n; q += NT) {
            const int i = q + i0 < acc_n ? q + i0 : q + i0 - acc_n;
            const float val = ys[i];
            if (val != 0.f) atomicAdd(a.y + i, val);
        }
    }
}

// SMEM_Y: y accumulated in shared memory (flushed once per CTA); SMEM_V: v
// staged in shared memory too (one coalesced copy per CTA: the nine gathers of
// an observation's camera then hit shared memory, not 32-sector L1 requests).
// NT threads per CTA: 512 (two CTAs per SM) or 1024 (one, when y and v do
// not fit twice).
template <bool SMEM_Y, bool SMEM_V, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_matvec_implicit(ImArgs a) {
    extern __shared__ float ys[];
    if (a.S != nullptr && a.S->done) return;
    matvec_body<SMEM_Y, SMEM_V, NT>(a, ys);
}

// shared-memory plan of the matvec: y and v in shared memory at two CTAs of
// 512 threads per SM when both fit twice, else at one CTA of 1024 threads;
// then y alone (v from global memory); else neither
enum ImMode { IM_YV2, IM_YV1, IM_Y2, IM_NONE };
constexpr int64_t IM_SMEM_SM = 220 * 1024;  // shared memory used per SM at most

ImMode implicit_mode(const Problem& p) {
    const int64_t b = 36LL * p.n_cam;
    if (2 * b <= IM_SMEM_SM / 2) return IM_YV2;
    if (2 * b <= IM_SMEM_SM) return IM_YV1;
    if (b <= IM_SMEM_Y_MAX) return IM_Y2;
    return IM_NONE;
}


// The undamped top rows [Q1^T J_p | R1 | Q1^T r] of landmark j (3 rows of
// 9 k + 4, the stored form's layout) rebuilt from the records, one thread per
// element: camera s's column c of row i is D_s[i][c] - sum_b P[i][b] u_s[b][c],
// u_s = V_s^T J_s (export only; the solver's readers fold this into their sums).
__global__ void k_implicit_top_rows(int j, const int32_t* __restrict__ pt_off, const int32_t* __restrict__ c_off,
                                    const int32_t* __restrict__ lm_pos, const float4* __restrict__ ipool,
                                    int64_t n_obs, const float* __restrict__ lmrec, float* __restrict__ top) {
    const int s0 = pt_off[j], k = pt_off[j + 1] - s0, ncol = 9 * k;
    const int64_t so0 = c_off[j] >> 1;
    const float* L = lmrec + (int64_t)LM_REC * lm_pos[j];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * (ncol + 4); e += gridDim.x * blockDim.x) {
        const int i = e / (ncol + 4), col = e - i * (ncol + 4);
        float out;
        if (col < ncol) {
            const int q = col / 9, c = col - 9 * q;
            float f[24];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const float4 v = ipool[m * n_obs + so0 + q];
                f[4 * m] = v.x;
                f[4 * m + 1] = v.y;
                f[4 * m + 2] = v.z;
                f[4 * m + 3] = v.w;
            }
            out = 0.f;
            if (q == 0 && i < 2) out = f[9 * i + c];
            if (q == 1 && i == 2) out = f[c];
#pragma unroll
            for (int b = 0; b < 3; ++b) out -= L[LR_P + 3 * i + b] * (f[18 + b] * f[c] + f[21 + b] * f[9 + c]);
        } else if (col < ncol + 3) {
            const int c = col - ncol;  // R1, upper (00 01 02 11 12 22)
            const int idx[3][3] = {{0, 1, 2}, {-1, 3, 4}, {-1, -1, 5}};
            out = idx[i][c] < 0 ? 0.f : L[LR_R1 + idx[i][c]];
        } else {
            out = L[LR_T + i];
        }
        top[e] = out;
    }
}

}  // namespace

void launch_implicit_top_rows(Problem& p, int j, int k, float* top) {
    k_implicit_top_rows<<<ceil_div(3 * (9 * (int64_t)k + 4), 256), 256, 0, p.stream>>>(
        j, p.pt_off, p.c_off, p.lm_pos, reinterpret_cast<const float4*>(p.ipool), p.n_obs, p.lmrec, top);
    BA_LAUNCH_CHECK();
}

// Tasks in storage order (decreasing k): k <= 32, the landmarks of one warp
// (32 / W teams); k > 32, one landmark each.
void plan_implicit(Problem& p) {
    std::vector<ImTask> tasks;
    const int kmax = p.k_max;
    int64_t pos = 0;
    for (int b = 0; b <= kmax; ++b) {
        const int k = kmax - b;
        const int64_t cnt = p.k_run_count[b];
        if (cnt == 0) continue;
        const int64_t so_run = p.run_co[b];
        const int per = k <= 32 ? 32 / team_width(k) : 1;
        for (int64_t l = 0; l < cnt; l += per) {
            ImTask t{};
            t.so0 = (int32_t)(so_run + l * k);
            t.pos0 = (int32_t)(pos + l);
            t.k = (int16_t)k;
            t.n = (int16_t)std::min<int64_t>(per, cnt - l);
            tasks.push_back(t);
        }
        pos += cnt;
    }
    p.im_ntasks = (int)tasks.size();
    p.im_nbig = 0;
    while (p.im_nbig < p.im_ntasks && tasks[p.im_nbig].k > 32) ++p.im_nbig;
    p.im_ctr = dalloc<uint32_t>(p, 64);
    BA_CUDA_TRY(cudaMemsetAsync(p.im_ctr, 0, 64 * sizeof(uint32_t), p.stream));
    p.im_tasks = dalloc<ImTask>(p, std::max<int64_t>(1, (int64_t)tasks.size()));
    if (!tasks.empty())
        BA_CUDA_TRY(cudaMemcpyAsync(p.im_tasks, tasks.data(), sizeof(ImTask) * tasks.size(), cudaMemcpyHostToDevice,
                                    p.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
}

void configure_implicit(Problem&) {
    BA_CUDA_TRY(cudaFuncSetAttribute(k_matvec_implicit<true, true, IM_THREADS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(IM_SMEM_SM / 2)));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_matvec_implicit<true, true, 2 * IM_THREADS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IM_SMEM_SM));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_matvec_implicit<true, false, IM_THREADS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, IM_SMEM_Y_MAX));
}

int implicit_matvec_grid(const Problem& p) { return implicit_mode(p) == IM_YV1 ? p.sm_count : 2 * p.sm_count; }

void launch_matvec_implicit(Problem& p, const float* v, float* y, const PcgScalars* S, float* pq_part) {
    const ImArgs a{static_cast<const ImTask*>(p.im_tasks), p.im_ntasks, p.im_nbig, p.im_ctr, pq_part,
                   reinterpret_cast<const float4*>(p.ipool),
                   p.n_obs, p.lmrec, p.mv_cam, v, y, p.n_cam, S,
                   p.batch.n_prob > 0 ? p.batch.lm : nullptr, p.batch.lm_prob, p.lm_by_k};
    const size_t b = 36 * (size_t)p.n_cam;
    switch (implicit_mode(p)) {
        case IM_YV2:
            k_matvec_implicit<true, true, IM_THREADS><<<p.sm_count * 2, IM_THREADS, 2 * b, p.stream>>>(a);
            break;
        case IM_YV1:
            k_matvec_implicit<true, true, 2 * IM_THREADS><<<p.sm_count, 2 * IM_THREADS, 2 * b, p.stream>>>(a);
            break;
        case IM_Y2:
            k_matvec_implicit<true, false, IM_THREADS><<<p.sm_count * 2, IM_THREADS, b, p.stream>>>(a);
            break;
        default:
            k_matvec_implicit<false, false, IM_THREADS><<<p.sm_count * 2, IM_THREADS, 0, p.stream>>>(a);
            break;
    }
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
