// K8 / K9: the per-camera MLP of the learned warm start and
// block-preconditioner correction (no counterpart in the paper; the solver
// it plugs into is the block-Jacobi PCG of Sec. 5.4).
//
// Forward (inference and training), one CTA of 128 threads per 128 rows:
// the four layers are dense BF16 GEMMs on the 5th-generation tensor cores.
// One thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// N = 256 or 64, K = 16 per instruction) with both operands in shared
// memory (K-major, 128-byte swizzle) and the accumulator in tensor memory
// (two halves of the 512 columns used alternately by successive layers).
// The epilogue (bias, GELU, BF16 rounding) reads the accumulator with
// tcgen05.ld, one row per thread, and writes the next layer's A operand in
// the swizzled layout.  Weights are stored in global memory already in that
// operand layout and staged with bulk asynchronous copies.
//
// Training: FP32 head loss and output gradient, FP32 backward on the CUDA
// cores (the same BF16-rounded weights and activations the forward used;
// rounding is passed straight through), Adam on FP32 master weights.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "learned.cuh"
#include "problem.cuh"
#include "ptx.cuh"

namespace sqrtba {

namespace {

constexpr int ML_OUTP = 64, ML_INP = 64;  // padded N of the last layer, K of the first
constexpr int ML_THREADS = 128;
// layer shapes: outputs NR, inputs KR, padded to the MMA shapes NP (N) and
// KP (multiple of 64); flat parameter offsets; operand image offsets
__host__ __device__ constexpr int NR(int l) { return l == 3 ? 54 : 256; }
__host__ __device__ constexpr int KR(int l) { return l == 0 ? 19 : 256; }
__host__ __device__ constexpr int NP(int l) { return l == 3 ? 64 : 256; }
__host__ __device__ constexpr int KP(int l) { return l == 0 ? 64 : 256; }
__host__ __device__ constexpr int64_t W_OFF(int l) {
    return l == 0 ? 0 : (l == 1 ? 5120 : (l == 2 ? 70912 : 136704));
}
__host__ __device__ constexpr int64_t b_off(int l) { return W_OFF(l) + (int64_t)NR(l) * KR(l); }
__host__ __device__ constexpr uint32_t IMG_OFF(int l) {
    return l == 0 ? 0u : (l == 1 ? 32768u : (l == 2 ? 163840u : (l == 3 ? 294912u : 327680u)));
}
static_assert(W_OFF(1) == b_off(0) + 256 && W_OFF(2) == b_off(1) + 256 && W_OFF(3) == b_off(2) + 256 &&
                  b_off(3) + 54 == ML_P,
              "parameter layout");
static_assert(IMG_OFF(1) == 2 * NP(0) * KP(0) && IMG_OFF(2) == IMG_OFF(1) + 2 * NP(1) * KP(1) &&
                  IMG_OFF(3) == IMG_OFF(2) + 2 * NP(2) * KP(2) && IMG_OFF(4) == IMG_OFF(3) + 2 * NP(3) * KP(3),
              "operand image layout");

// shared-memory plan of the forward kernel (from a 1024-byte aligned base)
constexpr int FW_A = 0;                  // A operand: 128 rows x 256 BF16 (64 KB)
constexpr int FW_W = 65536;              // B operand: up to 256 x 256 BF16 (128 KB)
constexpr int FW_BAR = 65536 + 131072;   // two mbarriers, TMEM slot, abort flag
constexpr int FW_SMEM = FW_BAR + 64 + 1024;
constexpr uint32_t TMEM_COLS = 512;

// byte offset of element (row, col) in a K-major operand image with 128-byte
// swizzle: 64-column (128-byte) blocks of `rows` rows, the 16-byte chunk index
// XOR-ed with row % 8
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int col, int rows) {
    const int kb = col >> 6, c = col & 63;
    return (uint32_t)kb * rows * 128u + (uint32_t)row * 128u + (uint32_t)((((c >> 3) ^ (row & 7)) << 4) + (c & 7) * 2);
}

// --- tcgen05 wrappers -------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// 32 consecutive FP32 columns of this thread's row (lane = row within the
// warp's 32-lane quarter), waited for inside the same asm block
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&f)[32]) {
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16(x)); }

// --- the fused forward --------------------------------------------------------------
struct FwdArgs {
    const uint8_t* ximg;   // feature tiles (16 KB each)
    const uint8_t* wimg;   // weight images
    const float* master;   // biases (FP32)
    int n;                 // valid rows
    int ld_z;              // rows of each z plane (padded)
    float* y;              // [rows][64]
    float* z;              // training: [3][ld_z][256]; nullptr for inference
    uint32_t* err;
};

__global__ void __launch_bounds__(ML_THREADS, 1) k_mlp_forward(FwdArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sA = smem_u32(sm + FW_A), sW = smem_u32(sm + FW_W);
    const uint32_t tma_bar = smem_u32(sm + FW_BAR), mma_bar = smem_u32(sm + FW_BAR + 8);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + FW_BAR + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + FW_BAR + 20);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = warp * 32 + lane;
    const int64_t grow = (int64_t)blockIdx.x * ML_ROWS + row;

    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(tma_bar, 1);
        mbar_init(mma_bar, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    if (threadIdx.x == 0) {
        mbar_expect_tx(tma_bar, 16384u + (IMG_OFF(1) - IMG_OFF(0)));
        bulk_g2s(sA, a.ximg + (int64_t)blockIdx.x * 16384, 16384u, tma_bar);
        bulk_g2s(sW, a.wimg + IMG_OFF(0), IMG_OFF(1) - IMG_OFF(0), tma_bar);
    }
    for (int l = 0; l < 4; ++l) {
        const int N = NP(l), K = KP(l);
        const uint32_t dcol = (l & 1) ? 256u : 0u;
        if (threadIdx.x == 0 && !*abort_flag) {
            if (mbar_wait(tma_bar, l & 1, abort_flag, a.err)) {
                tc_fence_after();
                const uint32_t idesc = mma_idesc(N);
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint32_t kb = kk >> 2, ks = kk & 3;
                    tc_mma(tbase + dcol, sw128_desc(sA + kb * (ML_ROWS * 128u) + ks * 32u),
                           sw128_desc(sW + kb * (uint32_t)(N * 128) + ks * 32u), idesc, kk > 0 ? 1u : 0u);
                }
                tc_commit(mma_bar);
            }
        }
        if (!mbar_wait(mma_bar, l & 1, abort_flag, a.err)) break;
        tc_fence_after();
        if (threadIdx.x == 0 && l < 3) {
            // the layer's MMAs are done with the B buffer: stage the next weights
            const uint32_t bytes = IMG_OFF(l + 2) - IMG_OFF(l + 1);
            mbar_expect_tx(tma_bar, bytes);
            bulk_g2s(sW, a.wimg + IMG_OFF(l + 1), bytes, tma_bar);
        }
        const float* bias = a.master + b_off(l);
        const uint32_t taddr = tbase + dcol + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc_ld32(taddr + c0, v);
            if (l < 3) {
                uint32_t packed[16];
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    const float z0 = v[j] + __ldg(bias + c0 + j), z1 = v[j + 1] + __ldg(bias + c0 + j + 1);
                    if (a.z && grow < a.n) {
                        float* zr = a.z + ((int64_t)l * a.ld_z + grow) * 256 + c0 + j;
                        zr[0] = z0;
                        zr[1] = z1;
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(gelu(z0), gelu(z1));
                    packed[j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t off = sw128_off(row, c0 + 8 * q, ML_ROWS);
                    *reinterpret_cast<uint4*>(sm + FW_A + off) =
                        make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                }
            } else if (grow < a.n) {
#pragma unroll
                for (int j = 0; j < 32; ++j) a.y[grow * ML_OUTP + c0 + j] = v[j] + (c0 + j < ML_OUT ? __ldg(bias + c0 + j) : 0.f);
            }
        }
        // the next layer's A operand is complete and visible to the tensor cores
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
}

// --- operand images -------------------------------------------------------------------
__global__ void k_pack_weights(const float* __restrict__ master, uint8_t* __restrict__ wimg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int l = 0; l < 4; ++l) {
        const int64_t cnt = (int64_t)NP(l) * KP(l);
        if (i < cnt) {
            const int nrow = (int)(i / KP(l)), k = (int)(i - (int64_t)nrow * KP(l));
            const float v = (nrow < NR(l) && k < KR(l)) ? master[W_OFF(l) + (int64_t)nrow * KR(l) + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(wimg + IMG_OFF(l) + sw128_off(nrow, k, NP(l))) = __float2bfloat16(v);
            return;
        }
        i -= cnt;
    }
}

// features (n x 19 FP32) -> BF16 tile images (rows >= n zero) and an FP32 copy
__global__ void k_pack_x(const float* __restrict__ feats, int n, int rows, uint8_t* __restrict__ ximg,
                         float* __restrict__ xf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * ML_INP) return;
    const int r = (int)(i / ML_INP), c = (int)(i - (int64_t)r * ML_INP);
    const float v = (r < n && c < ML_IN) ? feats[(int64_t)r * ML_IN + c] : 0.f;
    const int tile = r / ML_ROWS, tr = r - tile * ML_ROWS;
    *reinterpret_cast<__nv_bfloat16*>(ximg + (int64_t)tile * 16384 + sw128_off(tr, c, ML_ROWS)) = __float2bfloat16(v);
    if (c < ML_IN) xf[(int64_t)r * ML_IN + c] = v;
}

// --- per-sample preparation and heads --------------------------------------------
// Cholesky M = L L^T of one 9x9 block (row-major); false if not positive definite
__device__ bool chol9(const float* M, float* L) {
    for (int i = 0; i < 81; ++i) L[i] = 0.f;
    for (int j = 0; j < 9; ++j) {
        float s = M[j * 9 + j];
        for (int k = 0; k < j; ++k) s -= L[j * 9 + k] * L[j * 9 + k];
        if (!(s > 0.f)) return false;
        const float d = sqrtf(s);
        L[j * 9 + j] = d;
        for (int i = j + 1; i < 9; ++i) {
            float t = M[i * 9 + j];
            for (int k = 0; k < j; ++k) t -= L[i * 9 + k] * L[j * 9 + k];
            L[i * 9 + j] = t / d;
        }
    }
    return true;
}

// features [log diag M, w / |w|, log count] and head inputs [L, w, s, z*]
__device__ void prepare_one(const float* M, const float* g, const float* xs, int count, float* f, float* aux) {
    float L[81];
    if (!chol9(M, L)) {
        for (int c = 0; c < ML_IN; ++c) f[c] = 0.f;
        for (int c = 0; c < ML_AUX; ++c) aux[c] = 0.f;
        return;
    }
    float w[9], s[9];
    for (int i = 0; i < 9; ++i) {
        float t = g[i];
        for (int k = 0; k < i; ++k) t -= L[i * 9 + k] * w[k];
        w[i] = t / L[i * 9 + i];
    }
    for (int i = 8; i >= 0; --i) {
        float t = w[i];
        for (int k = i + 1; k < 9; ++k) t -= L[k * 9 + i] * s[k];
        s[i] = t / L[i * 9 + i];
    }
    float nw = 0.f;
    for (int i = 0; i < 9; ++i) nw += w[i] * w[i];
    nw = sqrtf(nw);
    for (int i = 0; i < 9; ++i) {
        f[i] = logf(M[i * 9 + i]);
        f[9 + i] = nw > 0.f ? w[i] / nw : 0.f;
    }
    f[18] = logf((float)max(count, 1));
    int t = 0;
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j <= i; ++j) aux[t++] = L[i * 9 + j];
    for (int i = 0; i < 9; ++i) {
        aux[45 + i] = w[i];
        aux[54 + i] = s[i];
        float zi = 0.f;
        if (xs)
            for (int k = i; k < 9; ++k) zi += L[k * 9 + i] * xs[k];  // (L^T x*)_i
        aux[63 + i] = zi;
    }
}

__global__ void k_prepare(const float* __restrict__ M, const float* __restrict__ g, const float* __restrict__ xs,
                          const int32_t* __restrict__ count, int n, float* __restrict__ feats,
                          float* __restrict__ aux) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    prepare_one(M + 81LL * i, g + 9LL * i, xs ? xs + 9LL * i : nullptr, count[i], feats + (int64_t)ML_IN * i,
                aux + (int64_t)ML_AUX * i);
}

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// F = I + E from the 45 outputs (diagonal 1 + 0.9 tanh(e_ii))
__device__ __forceinline__ void build_F(const float* e, float* F) {
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            float v = 0.f;
            if (j < i) v = e[tri(i, j)];
            else if (j == i) v = 1.f + 0.9f * tanhf(e[tri(i, i)]);
            F[i * 9 + j] = v;
        }
}

// per-sample normalised loss and dY (scaled by 1 / n); the batch loss sum is
// accumulated in FP64
__global__ void __launch_bounds__(256)
k_head_loss(const float* __restrict__ y, const float* __restrict__ aux, int n, int rows, float* __restrict__ dy,
            double* __restrict__ loss) {
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double li = 0.0;
    if (i < rows) {
        float* d = dy + (int64_t)i * ML_OUTP;
        for (int c = 0; c < ML_OUTP; ++c) d[c] = 0.f;
        if (i < n) {
            const float* Y = y + (int64_t)i * ML_OUTP;
            const float* A = aux + (int64_t)ML_AUX * i;
            float L[81], F[81];
            for (int r = 0; r < 9; ++r)
                for (int c = 0; c < 9; ++c) L[r * 9 + c] = c <= r ? A[tri(r, c)] : 0.f;
            const float* w = A + 45;
            const float* s = A + 54;
            const float* zs = A + 63;
            build_F(Y + 9, F);
            float den = 1e-30f, x0[9], th[9];
            for (int k = 0; k < 9; ++k) {
                den += zs[k] * zs[k];
                th[k] = tanhf(Y[k]);
                x0[k] = s[k] * (1.f + th[k]);
            }
            float R1[9], u[9], R2[9], q[9];
            for (int k = 0; k < 9; ++k) {
                float a = 0.f, b = 0.f;
                for (int m = 0; m < 9; ++m) {
                    a += L[m * 9 + k] * x0[m];  // (L^T x0)_k
                    b += F[m * 9 + k] * w[m];   // (F^T w)_k
                }
                R1[k] = a - zs[k];
                u[k] = b;
            }
            for (int k = 0; k < 9; ++k) {
                float v = 0.f;
                for (int m = 0; m < 9; ++m) v += F[k * 9 + m] * u[m];
                R2[k] = v - zs[k];
            }
            for (int k = 0; k < 9; ++k) {
                float v = 0.f;
                for (int m = 0; m < 9; ++m) v += F[m * 9 + k] * R2[m];
                q[k] = v;
            }
            float l1 = 0.f, l2 = 0.f;
            for (int k = 0; k < 9; ++k) {
                l1 += R1[k] * R1[k];
                l2 += R2[k] * R2[k];
            }
            li = (double)((l1 + l2) / den);
            const float sc = 2.f / (den * (float)n);
            for (int k = 0; k < 9; ++k) {
                float gx = 0.f;
                for (int m = 0; m < 9; ++m) gx += L[k * 9 + m] * R1[m];
                d[k] = sc * gx * s[k] * (1.f - th[k] * th[k]);
            }
            for (int r = 0; r < 9; ++r)
                for (int c = 0; c <= r; ++c) {
                    const float gF = sc * (R2[r] * u[c] + w[r] * q[c]);
                    if (r == c) {
                        const float te = tanhf(Y[9 + tri(r, r)]);
                        d[9 + tri(r, r)] = gF * 0.9f * (1.f - te * te);
                    } else {
                        d[9 + tri(r, c)] = gF;
                    }
                }
        }
    }
    li = block_sum_d(li, red);
    if (threadIdx.x == 0) atomicAdd(loss, li);
}

// --- backward (FP32, CUDA cores) ----------------------------------------------------
constexpr int BT = 64;   // output tile (rows x cols) of the backward GEMMs
constexpr int BK = 16;   // reduction chunk

// dZp[r][k] = (sum_n dZ[r][n] bf16(W[n][k])) * gelu'(Zp[r][k]) for k < 256
__global__ void __launch_bounds__(256)
k_dgrad(const float* __restrict__ dz, int ldz, int nr, const float* __restrict__ W, const float* __restrict__ zp,
        float* __restrict__ dzp, int rows) {
    __shared__ float sA[BK][BT + 1];
    __shared__ float sB[BK][BT + 1];
    const int r0 = blockIdx.x * BT, k0 = blockIdx.y * BT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int n0 = 0; n0 < nr; n0 += BK) {
        for (int e = threadIdx.x; e < BK * BT; e += 256) {
            const int a = e / BT, b = e - a * BT;  // a: n within chunk, b: row / col within tile
            const int nn = n0 + a;
            sA[a][b] = (nn < nr && r0 + b < rows) ? dz[(int64_t)(r0 + b) * ldz + nn] : 0.f;
            sB[a][b] = nn < nr ? bf16r(W[(int64_t)nn * 256 + k0 + b]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < BK; ++a) {
            float ra[4], rb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ra[q] = sA[a][ty * 4 + q];
                rb[q] = sB[a][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += ra[p] * rb[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int r = r0 + ty * 4 + p;
        if (r >= rows) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + tx * 4 + q;
            dzp[(int64_t)r * 256 + k] = acc[p][q] * gelu_grad(zp[(int64_t)r * 256 + k]);
        }
    }
}

// dW[n][k] += sum_r dZ[r][n] H[r][k] over a chunk of rows, db[n] += sum_r dZ[r][n];
// H = bf16(gelu(Zp)) (hidden layers) or the BF16-rounded features (layer 0)
__global__ void __launch_bounds__(256)
k_wgrad(const float* __restrict__ dz, int ldz, int nr, const float* __restrict__ zp, const float* __restrict__ xf,
        int kr, int rows, int rows_per_block, float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float sA[BK][BT + 1];
    __shared__ float sB[BK][BT + 1];
    const int n0 = blockIdx.x * BT, k0 = blockIdx.y * BT;
    const int rb = blockIdx.z * rows_per_block, re = min(rows, rb + rows_per_block);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    float bacc = 0.f;
    for (int c0 = rb; c0 < re; c0 += BK) {
        for (int e = threadIdx.x; e < BK * BT; e += 256) {
            const int a = e / BT, b = e - a * BT;
            const int r = c0 + a;
            const bool rok = r < re;
            sA[a][b] = (rok && n0 + b < nr) ? dz[(int64_t)r * ldz + n0 + b] : 0.f;
            float h = 0.f;
            if (rok && k0 + b < kr)
                h = xf ? bf16r(xf[(int64_t)r * ML_IN + k0 + b]) : bf16r(gelu(zp[(int64_t)r * 256 + k0 + b]));
            sB[a][b] = h;
        }
        __syncthreads();
        if (blockIdx.y == 0 && threadIdx.x < BT)
            for (int a = 0; a < BK; ++a) bacc += sA[a][threadIdx.x];
#pragma unroll
        for (int a = 0; a < BK; ++a) {
            float ra[4], rb2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ra[q] = sA[a][ty * 4 + q];
                rb2[q] = sB[a][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += ra[p] * rb2[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int nn = n0 + ty * 4 + p;
        if (nn >= nr) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + tx * 4 + q;
            if (k < kr) atomicAdd(dW + (int64_t)nn * kr + k, acc[p][q]);
        }
    }
    if (blockIdx.y == 0 && threadIdx.x < BT && n0 + threadIdx.x < nr) atomicAdd(db + n0 + threadIdx.x, bacc);
}

__global__ void k_adam(int64_t n, float* __restrict__ w, float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
}

// --- solver side ----------------------------------------------------------------------
// per camera: M_i (damped block), g_i and the observation count -> features
__global__ void k_camera_prepare(int n_cam, const float* __restrict__ mdiag, const float* __restrict__ g,
                                 const int32_t* __restrict__ cam_off, float* __restrict__ feats,
                                 float* __restrict__ aux) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cam) return;
    prepare_one(mdiag + 81LL * i, g + 9LL * i, nullptr, cam_off[i + 1] - cam_off[i],
                feats + (int64_t)ML_IN * i, aux + (int64_t)ML_AUX * i);
}

// warm start x0 = s (1 + tanh o) and B = L^-T F F^T L^-1; cameras whose block
// was not positive definite keep the plain block-Jacobi inverse and x0 = 0
__global__ void k_learned_head(int n_cam, const float* __restrict__ y, const float* __restrict__ aux,
                               const float* __restrict__ minv, float* __restrict__ minv_l, float* __restrict__ x0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cam) return;
    const float* A = aux + (int64_t)ML_AUX * i;
    float* B = minv_l + 81LL * i;
    if (!(A[0] > 0.f)) {
        for (int k = 0; k < 81; ++k) B[k] = minv[81LL * i + k];
        for (int k = 0; k < 9; ++k) x0[9LL * i + k] = 0.f;
        return;
    }
    const float* Y = y + (int64_t)i * ML_OUTP;
    float Li[81], F[81], T[81];
    // L^-1 (lower triangular) column by column
    for (int c = 0; c < 9; ++c)
        for (int r = 0; r < 9; ++r) {
            float t = r == c ? 1.f : 0.f;
            if (r < c) {
                Li[r * 9 + c] = 0.f;
                continue;
            }
            for (int k = c; k < r; ++k) t -= A[tri(r, k)] * Li[k * 9 + c];
            Li[r * 9 + c] = t / A[tri(r, r)];
        }
    build_F(Y + 9, F);
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            float t = 0.f;
            for (int k = 0; k < 9; ++k) t += F[r * 9 + k] * F[c * 9 + k];
            T[r * 9 + c] = t;
        }
    // B = Li^T T Li
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            float t = 0.f;
            for (int k = 0; k < 9; ++k) {
                float u = 0.f;
                for (int m = 0; m < 9; ++m) u += T[k * 9 + m] * Li[m * 9 + c];
                t += Li[k * 9 + r] * u;
            }
            B[r * 9 + c] = t;
        }
    for (int k = 0; k < 9; ++k) x0[9LL * i + k] = A[54 + k] * (1.f + tanhf(Y[k]));
}

template <typename T>
T* malloc_tracked(Mlp& m, int64_t n) {
    void* p = nullptr;
    BA_CUDA_TRY(cudaMalloc(&p, sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
    m.allocations.push_back(p);
    return static_cast<T*>(p);
}

void pack_weights(Mlp& m) {
    const int64_t total = (int64_t)IMG_OFF(4) / 2;
    k_pack_weights<<<ceil_div(total, 256), 256, 0, m.stream>>>(m.master, m.wimg);
    BA_LAUNCH_CHECK();
}

void run_forward(Mlp& m, int n, bool training) {
    const int tiles = (n + ML_ROWS - 1) / ML_ROWS;
    FwdArgs a{m.ximg, m.wimg, m.master, n, tiles * ML_ROWS, m.y, training ? m.z : nullptr, m.err};
    k_mlp_forward<<<tiles, ML_THREADS, FW_SMEM, m.stream>>>(a);
    BA_LAUNCH_CHECK();
}

void pack_x(Mlp& m, const float* feats, int n) {
    const int rows = ((n + ML_ROWS - 1) / ML_ROWS) * ML_ROWS;
    k_pack_x<<<ceil_div((int64_t)rows * ML_INP, 256), 256, 0, m.stream>>>(feats, n, rows, m.ximg, m.xf);
    BA_LAUNCH_CHECK();
}

}  // namespace

void mlp_init(Mlp& m, const float* host_params, cudaStream_t stream) {
    if (stream) {
        m.stream = stream;
    } else {
        BA_CUDA_TRY(cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking));
        m.own_stream = true;
    }
    BA_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    m.master = malloc_tracked<float>(m, ML_P);
    m.grad = malloc_tracked<float>(m, ML_P);
    m.adam_m = malloc_tracked<float>(m, ML_P);
    m.adam_v = malloc_tracked<float>(m, ML_P);
    m.wimg = malloc_tracked<uint8_t>(m, IMG_OFF(4));
    m.loss = malloc_tracked<double>(m, 1);
    m.err = malloc_tracked<uint32_t>(m, 1);
    BA_CUDA_TRY(cudaMallocHost(&m.loss_host, sizeof(double)));
    BA_CUDA_TRY(cudaMemcpyAsync(m.master, host_params, sizeof(float) * ML_P, cudaMemcpyHostToDevice, m.stream));
    BA_CUDA_TRY(cudaMemsetAsync(m.grad, 0, sizeof(float) * ML_P, m.stream));
    BA_CUDA_TRY(cudaMemsetAsync(m.adam_m, 0, sizeof(float) * ML_P, m.stream));
    BA_CUDA_TRY(cudaMemsetAsync(m.adam_v, 0, sizeof(float) * ML_P, m.stream));
    BA_CUDA_TRY(cudaMemsetAsync(m.err, 0, sizeof(uint32_t), m.stream));
    pack_weights(m);
    BA_CUDA_TRY(cudaStreamSynchronize(m.stream));
}

void mlp_free(Mlp& m) {
    if (m.stream) cudaStreamSynchronize(m.stream);
    for (void* p : m.allocations) cudaFree(p);
    m.allocations.clear();
    if (m.loss_host) cudaFreeHost(m.loss_host);
    m.loss_host = nullptr;
    if (m.own_stream && m.stream) cudaStreamDestroy(m.stream);
    m.stream = nullptr;
}

void mlp_reserve(Mlp& m, int n) {
    const int rows = ((std::max(n, 1) + ML_ROWS - 1) / ML_ROWS) * ML_ROWS;
    if (rows <= m.cap) return;
    m.cap = rows;
    m.ximg = malloc_tracked<uint8_t>(m, (int64_t)rows / ML_ROWS * 16384);
    m.xf = malloc_tracked<float>(m, (int64_t)rows * ML_IN);
    m.z = malloc_tracked<float>(m, 3LL * rows * 256);
    m.y = malloc_tracked<float>(m, (int64_t)rows * ML_OUTP);
    m.dy = malloc_tracked<float>(m, (int64_t)rows * ML_OUTP);
    m.dza = malloc_tracked<float>(m, (int64_t)rows * 256);
    m.dzb = malloc_tracked<float>(m, (int64_t)rows * 256);
}

void mlp_forward(Mlp& m, const float* feats, int n, float* out) {
    mlp_reserve(m, n);
    pack_x(m, feats, n);
    run_forward(m, n, false);
    BA_CUDA_TRY(cudaMemcpy2DAsync(out, sizeof(float) * ML_OUT, m.y, sizeof(float) * ML_OUTP, sizeof(float) * ML_OUT,
                                  n, cudaMemcpyDeviceToDevice, m.stream));
}

double mlp_loss_grad(Mlp& m, const float* feats, const float* aux, int n) {
    mlp_reserve(m, n);
    const int rows = ((n + ML_ROWS - 1) / ML_ROWS) * ML_ROWS;
    pack_x(m, feats, n);
    run_forward(m, n, true);
    BA_CUDA_TRY(cudaMemsetAsync(m.loss, 0, sizeof(double), m.stream));
    BA_CUDA_TRY(cudaMemsetAsync(m.grad, 0, sizeof(float) * ML_P, m.stream));
    k_head_loss<<<ceil_div(rows, 256), 256, 0, m.stream>>>(m.y, aux, n, rows, m.dy, m.loss);
    BA_LAUNCH_CHECK();
    // backward: layer 3 (dZ = dY, 54 outputs) down to layer 0
    const float* dz = m.dy;
    int ldz = ML_OUTP;
    float* bufs[2] = {m.dza, m.dzb};
    const int rpb = 1024;
    for (int l = 3; l >= 0; --l) {
        const float* zp = l > 0 ? m.z + (int64_t)(l - 1) * rows * 256 : nullptr;
        dim3 gw(ceil_div(NR(l), BT), ceil_div(KR(l), BT), ceil_div(n, rpb));
        k_wgrad<<<gw, 256, 0, m.stream>>>(dz, ldz, NR(l), zp, l == 0 ? m.xf : nullptr, KR(l), n, rpb,
                                          m.grad + W_OFF(l), m.grad + b_off(l));
        BA_LAUNCH_CHECK();
        if (l > 0) {
            float* dzp = bufs[l & 1];
            dim3 gd(ceil_div(n, BT), 256 / BT);
            k_dgrad<<<gd, 256, 0, m.stream>>>(dz, ldz, NR(l), m.master + W_OFF(l), zp, dzp, n);
            BA_LAUNCH_CHECK();
            dz = dzp;
            ldz = 256;
        }
    }
    BA_CUDA_TRY(cudaMemcpyAsync(m.loss_host, m.loss, sizeof(double), cudaMemcpyDeviceToHost, m.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(m.stream));
    return *m.loss_host / std::max(n, 1);
}

void mlp_adam(Mlp& m, float lr, float beta1, float beta2, float eps) {
    m.adam_t += 1;
    const float c1 = 1.f - std::pow(beta1, (float)m.adam_t), c2 = 1.f - std::pow(beta2, (float)m.adam_t);
    k_adam<<<ceil_div(ML_P, 256), 256, 0, m.stream>>>(ML_P, m.master, m.grad, m.adam_m, m.adam_v, lr, beta1, beta2,
                                                      eps, c1, c2);
    BA_LAUNCH_CHECK();
    pack_weights(m);
}

void mlp_prepare(cudaStream_t st, const float* M, const float* g, const float* xstar, const int32_t* count, int n,
                 float* feats, float* aux) {
    k_prepare<<<ceil_div(n, 128), 128, 0, st>>>(M, g, xstar, count, n, feats, aux);
    BA_LAUNCH_CHECK();
}

void learned_apply(Problem& p, Mlp& m) {
    // the MLP's work runs on the problem's stream
    cudaStream_t saved = m.stream;
    m.stream = p.stream;
    try {
        mlp_reserve(m, p.n_cam);
        count_launches(p, 5);
        k_camera_prepare<<<ceil_div(p.n_cam, 128), 128, 0, p.stream>>>(p.n_cam, p.mdiag, p.g, p.cam_off, p.lfeat,
                                                                      p.laux);
        BA_LAUNCH_CHECK();
        pack_x(m, p.lfeat, p.n_cam);
        run_forward(m, p.n_cam, false);
        k_learned_head<<<ceil_div(p.n_cam, 128), 128, 0, p.stream>>>(p.n_cam, m.y, p.laux, p.minv, p.minv_l, p.x);
        BA_LAUNCH_CHECK();
    } catch (...) {
        m.stream = saved;
        throw;
    }
    m.stream = saved;
}

}  // namespace sqrtba
