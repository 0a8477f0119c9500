// K1: per-landmark linearisation and in-place nullspace marginalisation.
//
// For landmark j with k observations the dense landmark block of Sec. 5.1
// (Fig. 2b) is [J_p | J_l | r] with 2k rows.  Three Householder reflections
// H_a = I - tau_a v_a v_a^T (Sec. 5.2: "three Householder reflections per
// landmark block") reduce J_l to R1; Q^T = H_3 H_2 H_1 is applied to the pose
// columns and the residual in compact WY form, Q^T = I - V T^T V^T, so that
// each output element costs three FMAs plus the one non-zero of the sparse
// J_p column:   out[i][col] = M[i][col] - sum_a V[i][a] W[a][col],
// W = T^T (V^T M) with M = [J_p | r].  Rows 0..2 are the R1 rows
// (Q1^T J_p, R1, Q1^T r, used by back substitution, Eq. backsub_nm); rows
// 3..2k-1 are Q2^T J_p and Q2^T r (Eq. reduced).  Q is never stored.
// The implicit storage writes no rows at all: per observation J_s and the
// two Householder rows, per landmark Tm, P = V[0:3, :] Tm^T, R1, Q1^T r and
// D_l^2; its readers rebuild camera s's top slice as D_s - P (V_s^T J_s).
//
// One warp handles a landmark with k <= 32 (2k rows fit one row per lane for
// the reductions); a 256-thread CTA handles larger k.  Work is taken from
// the landmark list ordered by decreasing k, so long blocks start first.
#include <algorithm>

#include "camera.cuh"
#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int K_WARP = 32;     // largest k handled by one warp
constexpr int LIN_WARPS = 4;   // warps per CTA in the warp kernel
constexpr int BIG_TEAM = 256;  // threads per CTA for k > K_WARP

__host__ __device__ constexpr int lin_smem_floats(int k) { return 59 * k + 24; }

// A team of TEAM threads factors one landmark block.  TEAM = 8 or 16: a
// sub-warp team (segmented shuffles), several landmarks per warp; 32: a warp;
// BIG_TEAM: a CTA.  Teams: 8 lanes for k <= 4, 16 for k <= 8, a warp for
// k <= 32, a CTA above.  Every team of a warp runs the same sequence of shuffles
// and syncs whatever its k, so teams of one warp may hold different k.
template <int TEAM>
struct Team {
    static_assert(TEAM == 8 || TEAM == 16, "sub-warp team width");
    __device__ static int rank() { return threadIdx.x & (TEAM - 1); }
    __device__ static void sync() { __syncwarp(); }
    __device__ static float tsum(float v) {
#pragma unroll
        for (int o = TEAM / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    __device__ static void sum3(float& a, float& b, float& c, float*) {
        a = tsum(a);
        b = tsum(b);
        c = tsum(c);
    }
};

template <>
struct Team<32> {
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static void sync() { __syncwarp(); }
    __device__ static void sum3(float& a, float& b, float& c, float*) {
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
    }
};

template <>
struct Team<BIG_TEAM> {
    __device__ static int rank() { return threadIdx.x; }
    __device__ static void sync() { __syncthreads(); }
    // red: >= 3 * (BIG_TEAM / 32) floats of shared memory
    __device__ static void sum3(float& a, float& b, float& c, float* red) {
        constexpr int NW = BIG_TEAM / 32;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) {
            red[3 * w] = a;
            red[3 * w + 1] = b;
            red[3 * w + 2] = c;
        }
        __syncthreads();
        a = b = c = 0.0f;
#pragma unroll
        for (int m = 0; m < NW; ++m) {
            a += red[3 * m];
            b += red[3 * m + 1];
            c += red[3 * m + 2];
        }
        __syncthreads();
    }
};

struct LinArgs {
    const float* frames;   // camera frames (FRAME floats per camera)
    const float* pts;
    const int32_t* obs_cam_s;
    const float2* obs_xy_s;
    const int32_t* pt_off;
    const int64_t* a_off;
    float* apool;
    float* tpool;
    float* cpool;
    const int32_t* c_off;
    float* dl2;
    // implicit storage (null in the explicit form): per observation record
    // chunks (6 float4 at m n_obs + so), residuals, per storage position Tm
    float* ipool;
    float* rpool;
    float* lmrec;
    int64_t n_obs;
    float huber;  // Huber parameter (<= 0: squared norm)
    const BatchLm* blm;      // batch: per-problem LM state (null for a single problem)
    const int32_t* lm_prob;  // batch: problem of every landmark
};

// Q^T J_p rows of a landmark with K observations, lanes over the columns
// col = rank + TEAM m (W of those columns in registers):
//   out[i][col] = J_p[i][col] - (V[i][0] W0 + V[i][1] W1 + V[i][2] W2),
// rows 0..2 to the top block, rows 3.. to A_j.  Specialised per K so that the
// column count, the row strides and the valid columns are compile-time; row
// i's J_p entries sit in columns 9 (i / 2) .. + 8, this lane's first such
// column is m0 (and, for teams narrower than 9, m0 + 1).
template <int TEAM, int K, int MC>
__device__ __forceinline__ void write_rows(const float* __restrict__ V, const float* __restrict__ JP,
                                           const float (&w0)[MC], const float (&w1)[MC], const float (&w2)[MC],
                                           float* __restrict__ top, float* __restrict__ Aj, int rank) {
    constexpr int NC = 9 * K, NR = 2 * K;
    constexpr int MK = (NC + TEAM - 1) / TEAM;
    static_assert(MK <= MC, "columns per lane");
    const int mfull = (NC - rank + TEAM - 1) / TEAM;  // this lane's valid columns
#pragma unroll 2
    for (int i = 0; i < NR; ++i) {
        const float v0 = V[3 * i], v1 = V[3 * i + 1], v2 = V[3 * i + 2];
        float* __restrict__ dst = i < 3 ? top + i * (NC + 4) : Aj + (i - 3) * NC;
        const int base = 9 * (i >> 1);
        const int m0 = base > rank ? (base - rank + TEAM - 1) / TEAM : 0;
        const int c0 = rank + TEAM * m0 - base, c1 = c0 + TEAM;
        const float j0 = c0 < 9 ? JP[i * 9 + c0] : 0.f;
        const float j1 = (TEAM < 9 && c1 < 9) ? JP[i * 9 + c1] : 0.f;
#pragma unroll
        for (int m = 0; m < MK; ++m) {
            float out = -(v0 * w0[m] + v1 * w1[m] + v2 * w2[m]);
            if (m == m0) out += j0;
            if (TEAM < 9 && m == m0 + 1) out += j1;
            if (m < MK - 1 || m < mfull) dst[rank + TEAM * m] = out;
        }
    }
}

template <int TEAM, int MC>
__device__ __forceinline__ void write_rows_dispatch(int k, const float* V, const float* JP, const float (&w0)[MC],
                                                    const float (&w1)[MC], const float (&w2)[MC], float* top,
                                                    float* Aj, int rank) {
    if constexpr (TEAM == 32) {
        switch (k) {
#define WR_CASE(KK) \
    case KK: write_rows<TEAM, KK, MC>(V, JP, w0, w1, w2, top, Aj, rank); break;
            WR_CASE(9) WR_CASE(10) WR_CASE(11) WR_CASE(12) WR_CASE(13) WR_CASE(14) WR_CASE(15) WR_CASE(16)
            WR_CASE(17) WR_CASE(18) WR_CASE(19) WR_CASE(20) WR_CASE(21) WR_CASE(22) WR_CASE(23) WR_CASE(24)
            WR_CASE(25) WR_CASE(26) WR_CASE(27) WR_CASE(28) WR_CASE(29) WR_CASE(30) WR_CASE(31) WR_CASE(32)
            default: break;
        }
    } else if constexpr (TEAM == 16) {
        switch (k) {
            WR_CASE(5) WR_CASE(6) WR_CASE(7) WR_CASE(8)
            default: break;
        }
    } else {
        switch (k) {
            WR_CASE(2) WR_CASE(3) WR_CASE(4)
            default: break;
        }
#undef WR_CASE
    }
}

// Linearise and marginalise landmark j; sm holds lin_smem_floats(k) floats.
// write = false runs the same steps without storing (an idle team of a warp).
// MC: columns per lane for TEAM <= 32 (ceil(9 k_max / TEAM)); the team's
// lanes own the pose columns col = rank + TEAM m, keep their W = Tm^T V^T J_p
// entries in registers and write Q^T J_p row by row (coalesced), three FMAs
// per element.  The CTA-wide team (k > 32) goes through shared memory.
template <int TEAM, int MC = 1>
__device__ void marginalize_landmark(const LinArgs& A, int j, int pos, float* sm, float* red, bool write = true) {
    using T = Team<TEAM>;
    const int rank = T::rank();
    const int s0 = A.pt_off[j];
    const int k = A.pt_off[j + 1] - s0;
    const int nr = 2 * k;        // rows
    const int ncol = 9 * k;      // pose columns
    float* L = sm;               // nr x 3   (J_l -> R1 and reflector tails)
    float* JP = L + 3 * nr;      // nr x 9   (pose Jacobian rows, block-sparse)
    float* RV = JP + 9 * nr;     // nr       (residuals)
    float* V = RV + nr;          // nr x 3   (Householder vectors, v_a[a] = 1)
    float* W = V + 3 * nr;       // 3 x (ncol + 1)
    float* misc = W + 3 * (ncol + 1);  // tau[3], beta, v0, Tm[9], vr[3]

    // 1. residuals and Jacobians of every observation (Sec. 6.1: analytic)
    const float X0 = A.pts[3 * j], X1 = A.pts[3 * j + 1], X2 = A.pts[3 * j + 2];
    for (int s = rank; s < k; s += TEAM) {
        const float2 z = A.obs_xy_s[s0 + s];
        float r[2], Jp[18], Jl[6];
        frame_jacobians(A.frames + FRAME * A.obs_cam_s[s0 + s], X0, X1, X2, z.x, z.y, r, Jp, Jl);
        huber_scale_rows(A.huber, r, Jp, Jl);  // IRLS rows of the robust norm
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            RV[2 * s + i] = r[i];
#pragma unroll
            for (int c = 0; c < 9; ++c) JP[(2 * s + i) * 9 + c] = Jp[9 * i + c];
#pragma unroll
            for (int c = 0; c < 3; ++c) L[(2 * s + i) * 3 + c] = Jl[3 * i + c];
        }
    }
    T::sync();

    // D_l^2 = clamp(diag(J_l^T J_l), 1e-6, 1e32)
    {
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        for (int i = rank; i < nr; i += TEAM) {
            d0 += L[3 * i] * L[3 * i];
            d1 += L[3 * i + 1] * L[3 * i + 1];
            d2 += L[3 * i + 2] * L[3 * i + 2];
        }
        T::sum3(d0, d1, d2, red);
        if (rank == 0 && write) {
            const float c0 = fminf(fmaxf(d0, 1e-6f), 1e32f), c1 = fminf(fmaxf(d1, 1e-6f), 1e32f),
                        c2 = fminf(fmaxf(d2, 1e-6f), 1e32f);
            A.dl2[3 * j] = c0;
            A.dl2[3 * j + 1] = c1;
            A.dl2[3 * j + 2] = c2;
            if (A.lmrec) {  // implicit storage: K2 reads D_l^2 with R1 from the landmark record
                float* Lr = A.lmrec + (int64_t)LM_REC * pos + LR_DL2;
                Lr[0] = c0;
                Lr[1] = c1;
                Lr[2] = c2;
            }
        }
    }

    // 2. Householder QR of J_l (2k x 3), reflector a acts on rows a..2k-1
    for (int a = 0; a < 3; ++a) {
        float sg = 0.f, u1 = 0.f, u2 = 0.f;
        for (int i = a + 1 + rank; i < nr; i += TEAM) sg += L[3 * i + a] * L[3 * i + a];
        T::sum3(sg, u1, u2, red);
        if (rank == 0) {
            const float alpha = L[3 * a + a];
            float tau = 0.f, beta = alpha, v0 = 1.f;
            if (sg > 0.f) {
                const float mu = sqrtf(alpha * alpha + sg);
                beta = alpha > 0.f ? -mu : mu;
                v0 = alpha - beta;
                tau = (beta - alpha) / beta;
            }
            misc[a] = tau;
            misc[3] = beta;
            misc[4] = v0;
        }
        T::sync();
        const float tau = misc[a], inv_v0 = 1.0f / misc[4];
        for (int i = rank; i < nr; i += TEAM)
            V[3 * i + a] = i < a ? 0.f : (i == a ? 1.f : (tau == 0.f ? 0.f : L[3 * i + a] * inv_v0));
        T::sync();
        // apply H_a to the remaining landmark columns
        float w1 = 0.f, w2 = 0.f, w0 = 0.f;
        for (int i = a + rank; i < nr; i += TEAM) {
            if (a + 1 < 3) w1 += V[3 * i + a] * L[3 * i + a + 1];
            if (a + 2 < 3) w2 += V[3 * i + a] * L[3 * i + a + 2];
        }
        T::sum3(w1, w2, w0, red);
        for (int i = a + rank; i < nr; i += TEAM) {
            const float va = V[3 * i + a];
            if (a + 1 < 3) L[3 * i + a + 1] -= tau * w1 * va;
            if (a + 2 < 3) L[3 * i + a + 2] -= tau * w2 * va;
        }
        T::sync();
        if (rank == 0) L[3 * a + a] = misc[3];
        T::sync();
    }

    // 3. compact WY: H_1 H_2 H_3 = I - V Tm V^T, Tm upper triangular
    {
        float d01 = 0.f, d02 = 0.f, d12 = 0.f;
        for (int i = rank; i < nr; i += TEAM) {
            d01 += V[3 * i] * V[3 * i + 1];
            d02 += V[3 * i] * V[3 * i + 2];
            d12 += V[3 * i + 1] * V[3 * i + 2];
        }
        T::sum3(d01, d02, d12, red);
        float r0 = 0.f, r1 = 0.f, r2 = 0.f;  // V^T r
        for (int i = rank; i < nr; i += TEAM) {
            r0 += V[3 * i] * RV[i];
            r1 += V[3 * i + 1] * RV[i];
            r2 += V[3 * i + 2] * RV[i];
        }
        T::sum3(r0, r1, r2, red);
        if (rank == 0) {
            const float t0 = misc[0], t1 = misc[1], t2 = misc[2];
            float* Tm = misc + 5;
            Tm[0] = t0;
            Tm[4] = t1;
            Tm[8] = t2;
            Tm[3] = Tm[6] = Tm[7] = 0.f;
            Tm[1] = -t0 * t1 * d01;
            Tm[5] = -t2 * (t1 * d12);
            Tm[2] = -t2 * (t0 * d02 + Tm[1] * d12);
            // W column of the residual: Tm^T (V^T r)
            float* vr = misc + 14;
            vr[0] = Tm[0] * r0;
            vr[1] = Tm[1] * r0 + Tm[4] * r1;
            vr[2] = Tm[2] * r0 + Tm[5] * r1 + Tm[8] * r2;
        }
        T::sync();
    }

    const bool implicit = A.ipool != nullptr;
    float* __restrict__ top = implicit ? nullptr : A.tpool + top_offset(s0, j);
    float* __restrict__ Aj = implicit ? nullptr : A.apool + A.a_off[j];
    if (implicit && write) {
        // per observation: J_s rows and Householder rows (6 float4 chunks,
        // coalesced over the team's observations), residuals; per landmark Tm
        const int64_t so0 = A.c_off[j] >> 1;
        float4* ip = reinterpret_cast<float4*>(A.ipool);
        for (int s = rank; s < k; s += TEAM) {
            float f[24];
#pragma unroll
            for (int c = 0; c < 18; ++c) f[c] = JP[18 * s + c];
#pragma unroll
            for (int c = 0; c < 6; ++c) f[18 + c] = V[6 * s + c];
#pragma unroll
            for (int m = 0; m < 6; ++m)
                ip[m * A.n_obs + so0 + s] = make_float4(f[4 * m], f[4 * m + 1], f[4 * m + 2], f[4 * m + 3]);
            A.rpool[2 * (so0 + s)] = RV[2 * s];
            A.rpool[2 * (so0 + s) + 1] = RV[2 * s + 1];
        }
        if (rank == 0) {
            // Tm and P = V[0:3, :] Tm^T (the top rows are rebuilt from P by
            // their readers: rows 0..2 of Q^T M are M[0:3] - P (V^T M))
            const float* Tm = misc + 5;
            float* L = A.lmrec + (int64_t)LM_REC * pos;
            L[LR_TM] = Tm[0];
            L[LR_TM + 1] = Tm[1];
            L[LR_TM + 2] = Tm[2];
            L[LR_TM + 3] = Tm[4];
            L[LR_TM + 4] = Tm[5];
            L[LR_TM + 5] = Tm[8];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    L[LR_P + 3 * i + b] = V[3 * i] * Tm[3 * b] + V[3 * i + 1] * Tm[3 * b + 1] + V[3 * i + 2] * Tm[3 * b + 2];
        }
    }
    if (implicit) {
        // nothing more per column: the readers rebuild the top rows
    } else if constexpr (TEAM <= 32) {
        // 4+5. W for this lane's columns (registers), then Q^T J_p row by row
        const float* Tm = misc + 5;
        const float T00 = Tm[0], T01 = Tm[1], T02 = Tm[2], T11 = Tm[4], T12 = Tm[5], T22 = Tm[8];
        float w0[MC], w1[MC], w2[MC];
#pragma unroll
        for (int m = 0; m < MC; ++m) {
            const int col = rank + TEAM * m;
            const bool ok = col < ncol;
            const int sb = ok ? col / 9 : 0, c = ok ? col - 9 * sb : 0;
            const float ja = ok ? JP[(2 * sb) * 9 + c] : 0.f, jb = ok ? JP[(2 * sb + 1) * 9 + c] : 0.f;
            const float m0 = V[3 * (2 * sb)] * ja + V[3 * (2 * sb + 1)] * jb;
            const float m1 = V[3 * (2 * sb) + 1] * ja + V[3 * (2 * sb + 1) + 1] * jb;
            const float m2 = V[3 * (2 * sb) + 2] * ja + V[3 * (2 * sb + 1) + 2] * jb;
            w0[m] = T00 * m0;
            w1[m] = T01 * m0 + T11 * m1;
            w2[m] = T02 * m0 + T12 * m1 + T22 * m2;
        }
        if (write) write_rows_dispatch<TEAM, MC>(k, V, JP, w0, w1, w2, top, Aj, rank);
    } else {
        // 4. W = Tm^T (V^T J_p) for the pose columns (two non-zero rows each)
        {
            const float* Tm = misc + 5;
            const float T00 = Tm[0], T01 = Tm[1], T02 = Tm[2], T11 = Tm[4], T12 = Tm[5], T22 = Tm[8];
            for (int col = rank; col < ncol; col += TEAM) {
                const int s = col / 9, c = col - 9 * s;
                const float ja = JP[(2 * s) * 9 + c], jb = JP[(2 * s + 1) * 9 + c];
                const float m0 = V[3 * (2 * s)] * ja + V[3 * (2 * s + 1)] * jb;
                const float m1 = V[3 * (2 * s) + 1] * ja + V[3 * (2 * s + 1) + 1] * jb;
                const float m2 = V[3 * (2 * s) + 2] * ja + V[3 * (2 * s + 1) + 2] * jb;
                W[col] = T00 * m0;
                W[(ncol + 1) + col] = T01 * m0 + T11 * m1;
                W[2 * (ncol + 1) + col] = T02 * m0 + T12 * m1 + T22 * m2;
            }
            T::sync();
        }
        // 5. write Q^T J_p: rows 0..2 to the top block, rows 3.. to A_j
        const int64_t total = (int64_t)nr * ncol;
        int e = rank;
        int i = e / ncol, col = e - i * ncol;
        for (; write && e < total; e += TEAM) {
            const int s = col / 9;
            const float mval = (s == (i >> 1)) ? JP[i * 9 + (col - 9 * s)] : 0.f;
            const float out = mval - (V[3 * i] * W[col] + V[3 * i + 1] * W[(ncol + 1) + col] +
                                      V[3 * i + 2] * W[2 * (ncol + 1) + col]);
            if (i < 3) top[i * (ncol + 4) + col] = out;
            else if (i < nr) Aj[e - 3 * ncol] = out;
            col += TEAM;
            while (col >= ncol) {
                col -= ncol;
                ++i;
            }
        }
    }
    // the residual column's W (misc[14..16], computed above)
    const float wr0 = misc[14], wr1 = misc[15], wr2 = misc[16];
    // residual column and R1
    for (int ii = rank; write && ii < nr; ii += TEAM) {
        const float out = RV[ii] - (V[3 * ii] * wr0 + V[3 * ii + 1] * wr1 + V[3 * ii + 2] * wr2);
        if (ii < 3 && implicit) {
            // R1 (upper: 00 01 02 11 12 22) and t = Q1^T r into the landmark record
            float* Lr = A.lmrec + (int64_t)LM_REC * pos;
            Lr[LR_T + ii] = out;
            if (ii == 0) {
                Lr[LR_R1] = L[0];
                Lr[LR_R1 + 1] = L[1];
                Lr[LR_R1 + 2] = L[2];
            } else if (ii == 1) {
                Lr[LR_R1 + 3] = L[4];
                Lr[LR_R1 + 4] = L[5];
            } else {
                Lr[LR_R1 + 5] = L[8];
            }
        } else if (ii < 3) {
            float* row = top + ii * (ncol + 4) + ncol;
            row[0] = ii <= 0 ? L[3 * ii] : 0.f;
            row[1] = ii <= 1 ? L[3 * ii + 1] : 0.f;
            row[2] = L[3 * ii + 2];
            row[3] = out;
        } else if (!implicit) {
            A.cpool[A.c_off[j] + (ii - 3)] = out;
        }
    }
}

// landmarks order[first .. first + count) with k <= KMAX, one team of W lanes each
template <int W, int KMAX>
__global__ void __launch_bounds__(32 * LIN_WARPS)
k_linearize_team(LinArgs A, const int32_t* __restrict__ order, int first, int count) {
    extern __shared__ float smem[];
    constexpr int TPW = 32 / W;
    const int w = threadIdx.x >> 5, tm = (threadIdx.x & 31) / W;
    const int idx0 = (blockIdx.x * LIN_WARPS + w) * TPW;
    if (idx0 >= count) return;  // whole warp
    const int idx = idx0 + tm;
    // a batch re-linearises only the problems whose last step was accepted
    const bool active = idx < count && (!A.blm || batch_relin(A.blm, A.lm_prob[order[first + idx]]));
    if (!__any_sync(0xffffffffu, active)) return;  // whole warp
    float* sm = smem + (w * TPW + tm) * lin_smem_floats(KMAX);
    const int pos = first + (active ? idx : idx0);
    marginalize_landmark<W, (9 * KMAX + W - 1) / W>(A, order[pos], pos, sm, nullptr, active);
}

// The implicit storage for k <= 32: register-resident teams of T lanes per
// landmark (T = 1, 2, 4, 8 for k <= 4, 8, 16, 32), lane r holding the rows of
// observations s = r, r + T, ... (at most four), so that the whole 2k x 4
// block [J_l | r] stays in registers.  The record's J_s part is written as each
// observation is linearised; Householder QR in place (R1 on and above the
// diagonal, v_a below it with v_a[a] = 1 implied), the reflectors applied to r
// directly (Q^T r = H_3 H_2 H_1 r); the team sums take log2 T shuffles, the
// pivot rows come from their owner lane.  A warp's teams all use the k of its
// first landmark (the largest: landmarks are in decreasing-k order); a shorter
// landmark's missing observations are zero rows, which leave R1, V's real
// rows and Q^T r unchanged and write nothing.  Then Tm, P, R1, Q1^T r and D_l^2
// as 16-byte stores and the records' Householder part.
template <int T>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// MO: observations per lane (ceil(k / T) for the warp's largest k); the code
// depends on k only through MO (fewer rows are zero), so one instantiation
// serves every k with the same MO
template <int T, int MO>
__device__ __forceinline__ void linearize_regteam(const LinArgs& A, int j, int pos, bool act) {
    constexpr int MR = 2 * MO;           // rows per lane: local row 2m + e is global row 2 (r + T m) + e
    const int lane = threadIdx.x & 31, r = lane & (T - 1), base = lane & ~(T - 1);
    int s0 = 0, k = 0;
    int64_t so0 = 0;
    float X0 = 0.f, X1 = 0.f, X2 = 0.f;
    if (act) {
        s0 = A.pt_off[j];
        k = A.pt_off[j + 1] - s0;
        so0 = A.c_off[j] >> 1;
        X0 = __ldg(A.pts + 3 * j);
        X1 = __ldg(A.pts + 3 * j + 1);
        X2 = __ldg(A.pts + 3 * j + 2);
    }
    const int64_t n = A.n_obs;
    float4* __restrict__ ip = reinterpret_cast<float4*>(A.ipool);
    float B[MR][4];  // [J_l | r] -> [R1 and v_1..v_3 | Q^T r], this lane's rows
    float jt[MO][2];  // J_s entries 16 and 17 (record chunk 4, with the Householder rows)
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int m = 0; m < MO; ++m) {
        const int s = r + T * m;
        if (s < k) {
            const float2 z = A.obs_xy_s[s0 + s];
            float rr[2], Jp[18], Jl[6];
            frame_jacobians(A.frames + FRAME * A.obs_cam_s[s0 + s], X0, X1, X2, z.x, z.y, rr, Jp, Jl);
            huber_scale_rows(A.huber, rr, Jp, Jl);
            const int64_t so = so0 + s;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ip[q * n + so] = make_float4(Jp[4 * q], Jp[4 * q + 1], Jp[4 * q + 2], Jp[4 * q + 3]);
            reinterpret_cast<float2*>(A.rpool)[so] = make_float2(rr[0], rr[1]);
            jt[m][0] = Jp[16];
            jt[m][1] = Jp[17];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                B[2 * m + e][0] = Jl[3 * e];
                B[2 * m + e][1] = Jl[3 * e + 1];
                B[2 * m + e][2] = Jl[3 * e + 2];
                B[2 * m + e][3] = rr[e];
                d0 += Jl[3 * e] * Jl[3 * e];
                d1 += Jl[3 * e + 1] * Jl[3 * e + 1];
                d2 += Jl[3 * e + 2] * Jl[3 * e + 2];
            }
        } else {
            jt[m][0] = jt[m][1] = 0.f;
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int c = 0; c < 4; ++c) B[2 * m + e][c] = 0.f;
        }
    }
    d0 = team_sum<T>(d0);
    d1 = team_sum<T>(d1);
    d2 = team_sum<T>(d2);
    const float c0 = fminf(fmaxf(d0, 1e-6f), 1e32f), c1 = fminf(fmaxf(d1, 1e-6f), 1e32f),
                c2 = fminf(fmaxf(d2, 1e-6f), 1e32f);
    if (act && r == 0) {
        A.dl2[3 * j] = c0;
        A.dl2[3 * j + 1] = c1;
        A.dl2[3 * j + 2] = c2;
    }
    auto grow = [&](int lr) { return 2 * (r + T * (lr >> 1)) + (lr & 1); };  // global row of local row lr
    // Householder QR: reflector a acts on global rows a..2k-1; pivot row a is
    // local row pl of lane (a / 2) % T
    float tau[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int own = (a >> 1) % T, pl = 2 * ((a >> 1) / T) + (a & 1);
        float sg = 0.f;
#pragma unroll
        for (int lr = 0; lr < MR; ++lr)
            if (grow(lr) > a) sg += B[lr][a] * B[lr][a];
        sg = team_sum<T>(sg);
        const float alpha = __shfl_sync(0xffffffffu, B[pl][a], base + own);
        float t = 0.f, beta = alpha, v0 = 1.f;
        if (sg > 0.f) {
            const float mu = sqrtf(alpha * alpha + sg);
            beta = alpha > 0.f ? -mu : mu;
            v0 = alpha - beta;
            t = (beta - alpha) / beta;
        }
        tau[a] = t;
        const float iv = 1.0f / v0;
#pragma unroll
        for (int lr = 0; lr < MR; ++lr)
            if (grow(lr) > a) B[lr][a] = t == 0.f ? 0.f : B[lr][a] * iv;
        if (r == own) B[pl][a] = beta;
        // w_c = B[a][c] + sum_{i > a} v_i B[i][c] for the columns c > a (and r)
        float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = a + 1; c < 4; ++c) {
#pragma unroll
            for (int lr = 0; lr < MR; ++lr)
                if (grow(lr) > a) w[c - a - 1] += B[lr][a] * B[lr][c];
            w[c - a - 1] = team_sum<T>(w[c - a - 1]);
            w[c - a - 1] = t * (w[c - a - 1] + __shfl_sync(0xffffffffu, B[pl][c], base + own));
        }
#pragma unroll
        for (int c = a + 1; c < 4; ++c) {
            const float wc = w[c - a - 1];
#pragma unroll
            for (int lr = 0; lr < MR; ++lr)
                if (grow(lr) > a) B[lr][c] -= wc * B[lr][a];
            if (r == own) B[pl][c] -= wc;
        }
    }
    // compact WY: H_1 H_2 H_3 = I - V Tm V^T (V(i, a) = 1 at i = a, 0 above)
    auto V = [&](int lr, int a) {
        const int i = grow(lr);
        return i == a ? 1.f : (i > a ? B[lr][a] : 0.f);
    };
    float d01 = 0.f, d02 = 0.f, d12 = 0.f;
#pragma unroll
    for (int lr = 0; lr < MR; ++lr) {
        d01 += V(lr, 0) * V(lr, 1);
        d02 += V(lr, 0) * V(lr, 2);
        d12 += V(lr, 1) * V(lr, 2);
    }
    d01 = team_sum<T>(d01);
    d02 = team_sum<T>(d02);
    d12 = team_sum<T>(d12);
    float Tm[3][3];
    Tm[0][0] = tau[0];
    Tm[1][1] = tau[1];
    Tm[2][2] = tau[2];
    Tm[1][0] = Tm[2][0] = Tm[2][1] = 0.f;
    Tm[0][1] = -tau[0] * tau[1] * d01;
    Tm[1][2] = -tau[2] * (tau[1] * d12);
    Tm[0][2] = -tau[2] * (tau[0] * d02 + Tm[0][1] * d12);
    // rows 0 and 1 live on lane 0 (local rows 0, 1), row 2 on lane 1 % T (local row 2 (1 / T))
    constexpr int own2 = 1 % T, pl2 = 2 * (1 / T);
    const float b20 = __shfl_sync(0xffffffffu, B[pl2][0], base + own2);
    const float b21 = __shfl_sync(0xffffffffu, B[pl2][1], base + own2);
    const float b22 = __shfl_sync(0xffffffffu, B[pl2][2], base + own2);
    const float b23 = __shfl_sync(0xffffffffu, B[pl2][3], base + own2);
    if (act && r == 0) {
        const float Vt[3][3] = {{1.f, 0.f, 0.f}, {B[1][0], 1.f, 0.f}, {b20, b21, 1.f}};
        float P[3][3];  // P = V[0:3, :] Tm^T
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int b = 0; b < 3; ++b) P[i][b] = Vt[i][0] * Tm[b][0] + Vt[i][1] * Tm[b][1] + Vt[i][2] * Tm[b][2];
        static_assert(LR_TM == 0 && LR_R1 == 40 && LR_DL2 == 46 && LR_T == 49 && LR_P == 52, "record");
        float4* L4 = reinterpret_cast<float4*>(A.lmrec + (int64_t)LM_REC * pos);
        L4[0] = make_float4(Tm[0][0], Tm[0][1], Tm[0][2], Tm[1][1]);
        *reinterpret_cast<float2*>(L4 + 1) = make_float2(Tm[1][2], Tm[2][2]);
        L4[10] = make_float4(B[0][0], B[0][1], B[0][2], B[1][1]);
        L4[11] = make_float4(B[1][2], b22, c0, c1);
        L4[12] = make_float4(c2, B[0][3], B[1][3], b23);
        L4[13] = make_float4(P[0][0], P[0][1], P[0][2], P[1][0]);
        L4[14] = make_float4(P[1][1], P[1][2], P[2][0], P[2][1]);
        L4[15] = make_float4(P[2][2], 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int m = 0; m < MO; ++m) {
        const int s = r + T * m;
        if (s < k) {
            const int lr = 2 * m;
            ip[4 * n + so0 + s] = make_float4(jt[m][0], jt[m][1], V(lr, 0), V(lr, 1));
            ip[5 * n + so0 + s] = make_float4(V(lr, 2), V(lr + 1, 0), V(lr + 1, 1), V(lr + 1, 2));
        }
    }
}

template <int T, int MLO, int MHI>
__device__ __forceinline__ void linearize_regteam_m(int mo, const LinArgs& A, int j, int pos, bool act) {
    if constexpr (MLO <= MHI) {
        if (mo == MLO) linearize_regteam<T, MLO>(A, j, pos, act);
        else linearize_regteam_m<T, MLO + 1, MHI>(mo, A, j, pos, act);
    }
}

// landmarks order[first .. first + count) with KLO <= k <= KHI, teams of T
// lanes; `cta` is the CTA's index within its segment
template <int T, int KLO, int KHI>
__device__ __forceinline__ void linearize_reg_segment(const LinArgs& A, const int32_t* __restrict__ order, int first,
                                                      int count, int cta) {
    constexpr int TPW = 32 / T;
    const int lane = threadIdx.x & 31;
    const int idx0 = ((cta * blockDim.x + threadIdx.x) >> 5) * TPW;
    if (idx0 >= count) return;  // whole warp
    const int idx = idx0 + lane / T;
    bool act = idx < count;
    const int pos = first + (act ? idx : idx0);
    const int j = order[pos];
    // a batch re-linearises only the problems whose last step was accepted
    if (act && A.blm && !batch_relin(A.blm, A.lm_prob[j])) act = false;
    const int j0 = order[first + idx0];  // the warp's largest k (uniform over the warp)
    const int kw = A.pt_off[j0 + 1] - A.pt_off[j0];
    if (kw >= KLO && kw <= KHI)
        linearize_regteam_m<T, (KLO + T - 1) / T, (KHI + T - 1) / T>((kw + T - 1) / T, A, j, pos, act);
}

// The four segments k 17..32, 9..16, 5..8, 2..4 (teams of 8, 4, 2, 1 lanes) in
// one grid, longest k first, so that their per-warp latencies overlap: a
// CTA's segment is fixed by its index (uniform over the CTA).
struct RegSegments {
    int first[4], count[4], cta_end[4];
};

__global__ void __launch_bounds__(128)
k_linearize_reg(LinArgs A, const int32_t* __restrict__ order, RegSegments g) {
    const int b = blockIdx.x;
    if (b < g.cta_end[0]) linearize_reg_segment<8, 17, 32>(A, order, g.first[0], g.count[0], b);
    else if (b < g.cta_end[1]) linearize_reg_segment<4, 9, 16>(A, order, g.first[1], g.count[1], b - g.cta_end[0]);
    else if (b < g.cta_end[2]) linearize_reg_segment<2, 5, 8>(A, order, g.first[2], g.count[2], b - g.cta_end[1]);
    else linearize_reg_segment<1, 2, 4>(A, order, g.first[3], g.count[3], b - g.cta_end[2]);
}

__global__ void __launch_bounds__(BIG_TEAM)
k_linearize_block(LinArgs A, const int32_t* __restrict__ order, int count) {
    extern __shared__ float smem[];
    __shared__ float red[3 * (BIG_TEAM / 32)];
    if ((int)blockIdx.x >= count) return;
    if (A.blm && !batch_relin(A.blm, A.lm_prob[order[blockIdx.x]])) return;
    marginalize_landmark<BIG_TEAM>(A, order[blockIdx.x], blockIdx.x, smem, red);
}

// D_p^2 = clamp(diag(J_p^T J_p), 1e-6, 1e32) per camera: one CTA per camera,
// threads strided over its observations, then a fixed-order block reduction
// (deterministic).
constexpr int CD_THREADS = 256;
__global__ void __launch_bounds__(CD_THREADS)
k_camera_diag(int n_cam, const float* __restrict__ frames, const float* __restrict__ pts,
              const int32_t* __restrict__ obs_pt_s, const float2* __restrict__ obs_xy_s,
              const int32_t* __restrict__ cam_off, const int32_t* __restrict__ cam_list,
              float* __restrict__ dp2, float huber, const BatchLm* __restrict__ blm,
              const int32_t* __restrict__ cam_prob) {
    __shared__ float part[CD_THREADS / 32][9];
    const int cam = blockIdx.x;
    if (blm && !batch_relin(blm, cam_prob[cam])) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.f;
    for (int e = cam_off[cam] + threadIdx.x; e < cam_off[cam + 1]; e += CD_THREADS) {
        const int s = cam_list[e];
        const int j = obs_pt_s[s];
        const float2 z = obs_xy_s[s];
        float r[2], Jp[18], Jl[6];
        frame_jacobians(frames + FRAME * cam, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r, Jp, Jl);
        huber_scale_rows(huber, r, Jp, Jl);
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] += Jp[c] * Jp[c] + Jp[9 + c] * Jp[9 + c];
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float v = warp_sum(acc[c]);
        if (lane == 0) part[w][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        float v = 0.f;
        for (int q = 0; q < CD_THREADS / 32; ++q) v += part[q][threadIdx.x];
        dp2[9 * cam + threadIdx.x] = fminf(fmaxf(v, 1e-6f), 1e32f);
    }
}

__global__ void k_export_jacobians(int64_t n_obs, const float* __restrict__ frames, const float* __restrict__ pts,
                                   const int32_t* __restrict__ obs_cam_s, const int32_t* __restrict__ obs_pt_s,
                                   const float2* __restrict__ obs_xy_s, float* r_out, float* jp_out,
                                   float* jl_out, float huber) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_obs;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int j = obs_pt_s[s];
        const float2 z = obs_xy_s[s];
        float r[2], Jp[18], Jl[6];
        frame_jacobians(frames + FRAME * obs_cam_s[s], pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], z.x, z.y, r,
                        Jp, Jl);
        huber_scale_rows(huber, r, Jp, Jl);
        for (int i = 0; i < 2; ++i) r_out[2 * s + i] = r[i];
        for (int i = 0; i < 18; ++i) jp_out[18 * s + i] = Jp[i];
        for (int i = 0; i < 6; ++i) jl_out[6 * s + i] = Jl[i];
    }
}

__global__ void k_frames(int n_cam, const float* __restrict__ cams, float* __restrict__ frames) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cam) make_frame(cams + 9 * i, frames + FRAME * i);
}

}  // namespace

void launch_frames(Problem& p) {
    count_launches(p, 1);
    k_frames<<<ceil_div(p.n_cam, 128), 128, 0, p.stream>>>(p.n_cam, p.cams, p.frames);
    BA_LAUNCH_CHECK();
}

int linearize_k_limit() { return 900; }

// landmark counts with k in (lo, hi] (lm_by_k is ordered by decreasing k)
int count_k(const Problem& p, int lo, int hi) {
    int n = 0;
    for (int b = 0; b <= p.k_max; ++b) {
        const int k = p.k_max - b;
        if (k > lo && k <= hi) n += p.k_run_count[b];
    }
    return n;
}

template <int W, int KMAX>
constexpr int team_smem_bytes() { return (int)sizeof(float) * lin_smem_floats(KMAX) * LIN_WARPS * (32 / W); }

void configure_linearize(Problem& p) {
    const int sb = (int)(sizeof(float) * lin_smem_floats(std::max(p.k_max, K_WARP)));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_linearize_block, cudaFuncAttributeMaxDynamicSharedMemorySize, sb));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_linearize_team<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     team_smem_bytes<32, 32>()));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_linearize_team<16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     team_smem_bytes<16, 8>()));
    BA_CUDA_TRY(cudaFuncSetAttribute(k_linearize_team<8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     team_smem_bytes<8, 4>()));
}

// The K1 kernels work on disjoint landmarks and D_p^2 only reads: D_p^2 and
// the few long k > 32 factorisations run on a side stream (forked from and
// joined back into the problem's stream) beside the team kernels, which run
// one after the other (run side by side they only contend).  The energy at
// the linearisation point, which only reads too, follows them on the side
// stream: K1's kernels are latency-bound at low occupancy and leave room.
void launch_linearize(Problem& p, int cost_slot) {
    if (p.schur) {  // no factorisation: D_p^2 and D_l^2 only (the Schur complement is formed per damping)
        launch_camera_diag(p);
        launch_schur_dl2(p);
        if (cost_slot >= 0) launch_cost_on(p, p.frames, p.pts, cost_slot, p.stream);
        return;
    }
    LinArgs A{p.frames, p.pts, p.obs_cam_s, p.obs_xy_s, p.pt_off, p.a_off, p.apool, p.tpool, p.cpool, p.c_off,
              p.dl2, p.implicit ? p.ipool : nullptr, p.rpool, p.lmrec, p.n_obs, (float)p.opt.huber_delta,
              p.batch.n_prob > 0 ? p.batch.lm : nullptr, p.batch.lm_prob};
    // segments of lm_by_k: k > 32 | 9..32 | 5..8 | 2..4
    const int n_big = p.n_big, n32 = count_k(p, 8, 32), n16 = count_k(p, 4, 8), n8 = count_k(p, 1, 4);
    BA_CUDA_TRY(cudaEventRecord(p.ev_fork, p.stream));
    BA_CUDA_TRY(cudaStreamWaitEvent(p.side, p.ev_fork, 0));
    // side: D_p^2, then the landmarks with k > 32 (one CTA each)
    k_camera_diag<<<p.n_cam, CD_THREADS, 0, p.side>>>(p.n_cam, p.frames, p.pts, p.obs_pt_s, p.obs_xy_s, p.cam_off,
                                                      p.cam_list, p.dp2, (float)p.opt.huber_delta,
                                                      p.batch.n_prob > 0 ? p.batch.lm : nullptr, p.batch.cam_prob);
    count_launches(p, 1);
    if (n_big > 0) {
        const size_t sm = sizeof(float) * lin_smem_floats(p.k_max);
        k_linearize_block<<<n_big, BIG_TEAM, sm, p.side>>>(A, p.lm_by_k, n_big);
        count_launches(p, 1);
    }
    if (cost_slot >= 0) launch_cost_on(p, p.frames, p.pts, cost_slot, p.side);
    if (p.implicit) {
        // register-resident teams of 8, 4, 2 and 1 lanes: k 17..32, 9..16, 5..8, 2..4, one grid
        RegSegments g{};
        const int cnt[4] = {count_k(p, 16, 32), count_k(p, 8, 16), count_k(p, 4, 8), count_k(p, 1, 4)};
        const int lanes[4] = {8, 4, 2, 1};
        int f = n_big, ctas = 0;
        for (int q = 0; q < 4; ++q) {
            g.first[q] = f;
            g.count[q] = cnt[q];
            f += cnt[q];
            ctas += ceil_div((int64_t)cnt[q] * lanes[q], 128);
            g.cta_end[q] = ctas;
        }
        if (ctas > 0) {
            k_linearize_reg<<<ctas, 128, 0, p.stream>>>(A, p.lm_by_k, g);
            count_launches(p, 1);
        }
    } else {
        int first = n_big;
        if (n32 > 0) {
            k_linearize_team<32, 32><<<ceil_div(n32, LIN_WARPS), 32 * LIN_WARPS, team_smem_bytes<32, 32>(),
                                       p.stream>>>(A, p.lm_by_k, first, n32);
            count_launches(p, 1);
        }
        first += n32;
        if (n16 > 0) {
            k_linearize_team<16, 8><<<ceil_div(n16, 2 * LIN_WARPS), 32 * LIN_WARPS, team_smem_bytes<16, 8>(),
                                      p.stream>>>(A, p.lm_by_k, first, n16);
            count_launches(p, 1);
        }
        first += n16;
        if (n8 > 0) {
            k_linearize_team<8, 4><<<ceil_div(n8, 4 * LIN_WARPS), 32 * LIN_WARPS, team_smem_bytes<8, 4>(),
                                     p.stream>>>(A, p.lm_by_k, first, n8);
            count_launches(p, 1);
        }
    }
    BA_LAUNCH_CHECK();
    BA_CUDA_TRY(cudaEventRecord(p.ev_join, p.side));
    BA_CUDA_TRY(cudaStreamWaitEvent(p.stream, p.ev_join, 0));
}

void launch_camera_diag(Problem& p) {
    count_launches(p, 1);
    k_camera_diag<<<p.n_cam, CD_THREADS, 0, p.stream>>>(p.n_cam, p.frames, p.pts, p.obs_pt_s, p.obs_xy_s, p.cam_off,
                                                        p.cam_list, p.dp2, (float)p.opt.huber_delta,
                                                        p.batch.n_prob > 0 ? p.batch.lm : nullptr,
                                                        p.batch.cam_prob);
    BA_LAUNCH_CHECK();
}

void launch_export_jacobians(Problem& p, float* r, float* jp, float* jl) {
    launch_frames(p);
    k_export_jacobians<<<p.sm_count * 4, 256, 0, p.stream>>>(p.n_obs, p.frames, p.pts, p.obs_cam_s, p.obs_pt_s,
                                                             p.obs_xy_s, r, jp, jl, (float)p.opt.huber_delta);
    BA_LAUNCH_CHECK();
}

}  // namespace sqrtba
