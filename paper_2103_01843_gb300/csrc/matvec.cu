// K4: the PCG matvec of Eq. cg_mult without forming H~:
//     y += sum_j P_j^T A_j^T (A_j P_j v)
// where A_j = Q^T J_p below R1 (2k x 9k, FP32, stored in the landmark block,
// Sec. 5.1-5.3) and P_j gathers the landmark's k camera sub-vectors.
//
// HBM-bound: every block is read once per launch (72 k^2 bytes per landmark).
// Blocks are stored by decreasing k, so equal-k blocks are adjacent.  The
// host plans tiles of the block pool (runs of equal-k blocks up to 32 KB, or
// 4-row-aligned row ranges of one block when a block is larger); each CTA
// (one per SM) streams its range of tiles through a ring of 4 to 6 stages in
// shared memory with bulk asynchronous copies (cp.async.bulk + mbarrier),
// one producer thread and 15 consumer warps.  A tile rarely needs every
// consumer warp, so successive tiles are handed to successive groups of
// warps, and a stage is released once the warps of its tile are done.
//   small tiles (k <= 21): teams of 8/16/32 lanes, one block per team, code
//     specialised per k; per row u_r = A_j[r,:] v_j (team shuffle reduction)
//     and y_j += u_r A_j[r,:] (single pass over the block);
//   big tiles (21 < k <= 222): u for the tile's rows, then column sums;
//   k > 222: read directly from global memory (two passes).
// y accumulates in a per-CTA shared copy flushed once per CTA (one atomic per
// touched entry) when it fits beside the stages, else in global memory.  Every wait is bounded (2 s by %globaltimer); on a timeout
// the kernel raises ERRBIT_TIMEOUT, waits for its own copies and returns.
#include <algorithm>
#include <vector>

#include "problem.cuh"
#include "ptx.cuh"

namespace sqrtba {

namespace {

constexpr int MV_STAGE_A = 32768;   // bytes of blocks per stage
constexpr int MV_STAGE_C = 1024;    // bytes of camera indices per stage
// Registers are split over the SM's four sub-partitions (16K each) and the
// CTA's 16 warps spread four to a sub-partition: 128 registers per thread.
constexpr int MV_CONSUMERS = 15;    // consumer warps per CTA
constexpr int MV_THREADS = 32 * (MV_CONSUMERS + 1);
constexpr int MV_KSMALL_MAX = 21;   // whole blocks, specialised per k (up to the planner's mv_ksmall)
constexpr int MV_KBIG = 222;        // row ranges, multiples of 4 rows (36k * 4 <= 32 KB)
constexpr int MV_UMAX = 45;         // rows of one big tile (multiple of MV_CONSUMERS)

constexpr int MV_STAGE_R = 2048;    // bytes of c_j values per stage (preconditioner mode)
// Shared-memory layout for NS stages (PC = 1: the preconditioner record
// pass, which also stages c_j values); ACC_OFF starts the matvec's per-CTA
// copy of y.
template <int NS, int PC>
struct Layout {
    static constexpr int STAGE_C_OFF = NS * MV_STAGE_A;
    static constexpr int STAGE_R_OFF = STAGE_C_OFF + NS * MV_STAGE_C;
    static constexpr int U_OFF = STAGE_R_OFF + (PC ? NS * MV_STAGE_R : 0);
    static constexpr int BAR_OFF = (U_OFF + NS * MV_UMAX * 4 + 7) & ~7;
    static constexpr int FLAG_OFF = BAR_OFF + 2 * NS * 8;
    static constexpr int SEQ_OFF = FLAG_OFF + 16;          // tile index each stage holds
    static constexpr int ACC_OFF = SEQ_OFF + 32;
};
constexpr int SMEM_LIMIT = 227 * 1024;
static_assert(Layout<6, 1>::ACC_OFF <= SMEM_LIMIT, "six stages fit the opt-in shared memory");

enum : int16_t { TILE_SMALL = 0, TILE_BIG = 1, TILE_GLOBAL = 2 };

struct MvTile {
    int64_t a_off;    // float offset of the tile's first A float
    int32_t cam_off;  // offset into mv_cam of its first landmark's cameras
    int32_t bytes;    // A bytes to copy (multiple of 16; 0 for TILE_GLOBAL)
    int16_t k;
    int16_t kind;
    int32_t count;    // small: landmarks; big: rows; global: 1
    int32_t r0;       // big: first row
    int32_t first;    // global: storage position of the landmark
};
static_assert(sizeof(MvTile) == 32, "tile record size");

enum : int { MODE_MATVEC = 0, MODE_PRECOND = 1 };
constexpr int REC = 54;  // per-observation record: 45 entries of A_s^T A_s (upper, row-major) + A_s^T c
constexpr int REC_STRIDE = 56;  // floats between records in global memory (16-byte aligned, 2 pad floats)

struct MvArgs {
    const MvTile* tiles;
    const int32_t* tile_begin;
    const float* apool;
    const int32_t* mv_cam;
    const int32_t* lm_by_k;
    const int32_t* pt_off;
    const int32_t* obs_cam_s;
    const int64_t* a_off;
    const float* v;
    float* y;
    int n_cam;
    const PcgScalars* S;
    uint32_t* err;
    const float* cpool;  // preconditioner mode: c_j in storage order
    float* rec;          // preconditioner mode: REC floats per observation (storage order)
    int big8_kmax;       // big tiles with k up to this take eight rows a warp (else four)
    // failure test hooks (defaults WAIT_NS and -1): the limit of the consumer
    // and empty-stage waits, and a tile of CTA 0 the producer does not issue
    // (its consumers' waits then run out and the kernel returns with
    // ERRBIT_TIMEOUT raised).  The producer's final drain keeps WAIT_NS.
    uint64_t wait_ns;
    int fail_tile;
};

// --- consumers ---------------------------------------------------------------------
// Team width of whole-block tiles of k: narrow teams (fewer shuffles per
// element) where their lanes hold at most 7 columns, whole warps from k = 12
// on (measured per k on uniform-k scenes: 8 lanes for k <= 7, 16 for
// 8 <= k <= 11, 32 above).
__host__ __device__ constexpr int small_team_width(int k) { return k <= 7 ? 8 : (k <= 11 ? 16 : 32); }

template <int K>
struct SmallShape {
    static constexpr int NC = 9 * K, NR = 2 * K;
    static constexpr int W = small_team_width(K);
    static constexpr int NM = (NC + W - 1) / W;         // columns per lane
    static constexpr int G = NM <= 6 ? 8 : 4;           // rows per group (G x NM values in registers)
    static constexpr int BF = (18 * K * K + 3) & ~3;  // block floats (padded to 16 bytes)
};

// Rows r0 .. r0 + GR - 1 of one block for a team of W lanes (lane t of the
// team owns columns t + W m): the GR row sums u_r = A_r v are
// reduce-scattered (log2 GR halving shuffles over the team's top lane bits
// leave each lane one row's partial sum, xor shuffles over the remaining
// bits complete it) and broadcast back, then y += u_r A_r.
template <int K, int GR>
__device__ __forceinline__ void small_rows(const float* __restrict__ blk, int r0, const float (&vr)[SmallShape<K>::NM],
                                           float (&yr)[SmallShape<K>::NM], int t, int lane) {
    using S = SmallShape<K>;
    constexpr int W = S::W, NM = S::NM;
    constexpr int LG = GR == 8 ? 3 : (GR == 4 ? 2 : 1);
    static_assert(GR == 8 || GR == 4 || GR == 2, "row group");
    static_assert((GR >> LG) == 1 && GR <= W, "row group within the team");
    float a[GR][NM], cur[GR];
#pragma unroll
    for (int q = 0; q < GR; ++q) {
        cur[q] = 0.f;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const int col = t + W * m;
            a[q][m] = col < S::NC ? blk[(r0 + q) * S::NC + col] : 0.f;
            cur[q] += a[q][m] * vr[m];
        }
    }
#pragma unroll
    for (int st = 0; st < LG; ++st) {
        const int n = GR >> st, o = W >> (st + 1);
        const bool b = lane & o;
#pragma unroll
        for (int i = 0; i < GR / 2; ++i) {
            if (i < n / 2) {
                const float send = b ? cur[i] : cur[i + n / 2], keep = b ? cur[i + n / 2] : cur[i];
                cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    float u = cur[0];
#pragma unroll
    for (int o = W >> (LG + 1); o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    const int tbase = lane & ~(W - 1);
#pragma unroll
    for (int q = 0; q < GR; ++q) {
        int src = tbase;
#pragma unroll
        for (int st = 0; st < LG; ++st)
            if ((q >> (LG - 1 - st)) & 1) src += W >> (st + 1);
        const float uq = __shfl_sync(0xffffffffu, u, src);
#pragma unroll
        for (int m = 0; m < NM; ++m) yr[m] += uq * a[q][m];
    }
}

// One tile of `count` blocks with k = K; consumer warp cw of MV_CONSUMERS.
// Each team of W lanes takes one block: full groups of G rows, then the
// remaining rows in groups of 4 and 2 (2k is even), so no row is padded.
// Teams past the tile's last block read its first block (finite data) with
// v = 0, so they add nothing; their y is not written.
template <int K>
__device__ __forceinline__ void small_tile(const float* __restrict__ sa, const int32_t* __restrict__ sc, int count,
                                           const float* __restrict__ v, float* __restrict__ yt, int cw, int lane) {
    using S = SmallShape<K>;
    constexpr int TPW = 32 / S::W;
    constexpr int T = MV_CONSUMERS * TPW;
    constexpr int FULL = (S::NR / S::G) * S::G, REM = S::NR - FULL;
    constexpr bool R4 = S::G == 8 && REM >= 4;
    constexpr bool R2 = (REM - (R4 ? 4 : 0)) == 2;
    const int t = lane % S::W;
    for (int base = cw * TPW; base < count; base += T) {
        const int l = base + lane / S::W;
        const bool active = l < count;
        const float* blk = sa + (active ? l : 0) * S::BF;
        const int32_t* cams = sc + (active ? l : 0) * K;
        float vr[S::NM], yr[S::NM];
        int yi[S::NM];
#pragma unroll
        for (int m = 0; m < S::NM; ++m) {
            const int col = t + S::W * m;
            const bool ok = active && col < S::NC;
            const int s = col / 9;
            yi[m] = ok ? 9 * cams[s] + (col - 9 * s) : 0;
            vr[m] = ok ? __ldg(v + yi[m]) : 0.f;
            yr[m] = 0.f;
        }
#pragma unroll 1
        for (int r0 = 0; r0 < FULL; r0 += S::G) small_rows<K, S::G>(blk, r0, vr, yr, t, lane);
        if constexpr (R4) small_rows<K, 4>(blk, FULL, vr, yr, t, lane);
        if constexpr (R2) small_rows<K, 2>(blk, S::NR - 2, vr, yr, t, lane);
#pragma unroll
        for (int m = 0; m < S::NM; ++m) {
            const int col = t + S::W * m;
            if (active && col < S::NC) atomicAdd(yt + yi[m], yr[m]);
        }
    }
}

// --- preconditioner mode: per-observation records -----------------------------------
// One thread per observation slot s of a block: over the block's rows r,
// acc += a a^T (upper triangle) and accg += a c_r with a = A_j[r, 9s .. 9s+8].
__device__ __forceinline__ void slot_accumulate(const float* __restrict__ blk, const float* __restrict__ cvals,
                                                int nc, int r0, int r1, int s, float acc[REC]) {
    for (int r = r0; r < r1; ++r) {
        float a[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) a[c] = blk[r * nc + 9 * s + c];
        const float cv = cvals[r];
        int t = 0;
#pragma unroll
        for (int u = 0; u < 9; ++u) {
            acc[45 + u] += a[u] * cv;
#pragma unroll
            for (int v = u; v < 9; ++v) acc[t++] += a[u] * a[v];
        }
    }
}

__device__ __forceinline__ void rec_store(float* __restrict__ rec, const float acc[REC]) {
    float4* r4 = reinterpret_cast<float4*>(rec);
#pragma unroll
    for (int m = 0; m < REC / 4; ++m) r4[m] = make_float4(acc[4 * m], acc[4 * m + 1], acc[4 * m + 2], acc[4 * m + 3]);
    r4[REC / 4] = make_float4(acc[REC - 2], acc[REC - 1], 0.f, 0.f);
}

__device__ __forceinline__ void rec_add(float* __restrict__ rec, const float acc[REC]) {
    float4* r4 = reinterpret_cast<float4*>(rec);
#pragma unroll
    for (int m = 0; m < REC / 4; ++m)
        atomicAdd(r4 + m, make_float4(acc[4 * m], acc[4 * m + 1], acc[4 * m + 2], acc[4 * m + 3]));
    atomicAdd(r4 + REC / 4, make_float4(acc[REC - 2], acc[REC - 1], 0.f, 0.f));
}

// A slot's record is stored in the observation's record in global memory,
// or added there when its block is split over several row tiles.
__device__ __forceinline__ void rec_out(const MvArgs& a, int64_t obs, bool add, const float acc[REC]) {
    if (add) rec_add(a.rec + obs * REC_STRIDE, acc);
    else rec_store(a.rec + obs * REC_STRIDE, acc);
}

// whole staged blocks, one slot per thread
__device__ __forceinline__ void precond_blocks(const MvArgs& a, const MvTile& tile, const float* __restrict__ blocks,
                                               const int32_t* __restrict__ sc, const float* __restrict__ cvals,
                                               int tid) {
    const int k = tile.k, nc = 9 * k, nr = 2 * k;
    const int64_t bf = pad4(18LL * k * k);
    for (int q = tid; q < tile.count * k; q += MV_CONSUMERS * 32) {
        const int l = q / k, s = q - l * k;
        float acc[REC];
#pragma unroll
        for (int m = 0; m < REC; ++m) acc[m] = 0.f;
        slot_accumulate(blocks + l * bf, cvals + l * nr, nc, 0, nr, s, acc);
        rec_out(a, tile.cam_off + q, false, acc);
    }
}

// rows [r0, r0 + nrows) of one block (staged): partial records
__device__ __forceinline__ void precond_rows(const MvArgs& a, const MvTile& tile, const float* __restrict__ sa,
                                             const int32_t* __restrict__ sc, const float* __restrict__ cvals,
                                             int tid) {
    const int k = tile.k, nc = 9 * k;
    for (int s = tid; s < k; s += MV_CONSUMERS * 32) {
        float acc[REC];
#pragma unroll
        for (int m = 0; m < REC; ++m) acc[m] = 0.f;
        slot_accumulate(sa, cvals, nc, 0, tile.count, s, acc);
        rec_out(a, tile.cam_off + s, tile.count < 2 * k, acc);
    }
}

// a block read from global memory (k > MV_KBIG)
__device__ void precond_global(const MvArgs& a, const MvTile& tile, int tid) {
    const int j = a.lm_by_k[tile.first];
    const int k = a.pt_off[j + 1] - a.pt_off[j], nc = 9 * k, nr = 2 * k;
    const float* Aj = a.apool + a.a_off[j];
    const float* cj = a.cpool + 2LL * tile.cam_off;
    for (int s = tid; s < k; s += MV_CONSUMERS * 32) {
        float acc[REC];
#pragma unroll
        for (int m = 0; m < REC; ++m) acc[m] = 0.f;
        slot_accumulate(Aj, cj, nc, 0, nr, s, acc);
        rec_out(a, tile.cam_off + s, false, acc);
    }
}

__device__ __forceinline__ void small_dispatch(int k, const float* sa, const int32_t* sc, int count,
                                               const float* __restrict__ v, float* yt, int cw, int lane) {
    switch (k) {
#define MV_CASE(KK) \
    case KK: small_tile<KK>(sa, sc, count, v, yt, cw, lane); break;
        MV_CASE(2) MV_CASE(3) MV_CASE(4) MV_CASE(5) MV_CASE(6) MV_CASE(7) MV_CASE(8) MV_CASE(9) MV_CASE(10)
        MV_CASE(11) MV_CASE(12) MV_CASE(13) MV_CASE(14) MV_CASE(15) MV_CASE(16) MV_CASE(17) MV_CASE(18)
        MV_CASE(19) MV_CASE(20) MV_CASE(21)
#undef MV_CASE
        default: break;
    }
}

// Rows [r0, r0 + nrows) of one block with k > MV_KSMALL, staged in sa.  Each
// warp owns RPW (4 or 8) consecutive rows (no cross-warp dependency): u_r
// for its rows over all columns, with v gathered once per column chunk for
// all of its rows, then its rows' contribution A[r, col] u_r to every column.
// A tile keeps ceil(nrows / RPW) warps busy; tiles rotate over the warps.
// Eight rows a warp halve the y updates and v gathers per row; four spread a
// short tile (large k) over more warps.  The plan sets the largest k that
// takes eight (big8_kmax).
constexpr int BIG_CH = 4;    // columns per lane per chunk
template <int BIG_RPW>
__device__ __forceinline__ void big_tile(const float* __restrict__ sa, const int32_t* __restrict__ sc, int k,
                                         int nrows, const float* __restrict__ v, float* __restrict__ yt, int vcw,
                                         int lane) {
    const int nc = 9 * k;
    const int ra = vcw * BIG_RPW;
    if (ra >= nrows) return;
    const int nr = min(BIG_RPW, nrows - ra);
    const float* rows = sa + ra * nc;
    float part[BIG_RPW];
#pragma unroll
    for (int q = 0; q < BIG_RPW; ++q) part[q] = 0.f;
    for (int c0 = 0; c0 < nc; c0 += 32 * BIG_CH) {
        float vc[BIG_CH];
#pragma unroll
        for (int m = 0; m < BIG_CH; ++m) {
            const int col = c0 + lane + 32 * m;
            const int s = col / 9;
            vc[m] = col < nc ? __ldg(v + 9 * sc[s] + (col - 9 * s)) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < BIG_RPW; ++q) {
            if (q < nr) {
#pragma unroll
                for (int m = 0; m < BIG_CH; ++m) {
                    const int col = c0 + lane + 32 * m;
                    if (col < nc) part[q] += rows[q * nc + col] * vc[m];
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < BIG_RPW; ++q) part[q] = warp_sum(part[q]);
    for (int c0 = 0; c0 < nc; c0 += 32 * BIG_CH) {
#pragma unroll
        for (int m = 0; m < BIG_CH; ++m) {
            const int col = c0 + lane + 32 * m;
            if (col < nc) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < BIG_RPW; ++q)
                    if (q < nr) acc += rows[q * nc + col] * part[q];
                const int s = col / 9;
                atomicAdd(yt + 9 * sc[s] + (col - 9 * s), acc);
            }
        }
    }
}

// A block read straight from global memory (k > MV_KBIG), one warp, two passes.
__device__ void global_block(const MvArgs& a, int pos, float* __restrict__ ub, float* __restrict__ yt, int lane) {
    const int j = a.lm_by_k[pos];
    const int s0 = a.pt_off[j], k = a.pt_off[j + 1] - s0, nc = 9 * k, nr = 2 * k;
    const float* Aj = a.apool + a.a_off[j];
    for (int r0 = 0; r0 < nr; r0 += MV_UMAX) {
        const int rn = min(MV_UMAX, nr - r0);
        for (int r = 0; r < rn; ++r) {
            float part = 0.f;
            for (int col = lane; col < nc; col += 32) {
                const int s = col / 9;
                part += Aj[(int64_t)(r0 + r) * nc + col] * __ldg(a.v + 9 * a.obs_cam_s[s0 + s] + (col - 9 * s));
            }
            part = warp_sum(part);
            if (lane == 0) ub[r] = part;
        }
        __syncwarp();
        for (int col = lane; col < nc; col += 32) {
            float acc = 0.f;
            for (int r = 0; r < rn; ++r) acc += Aj[(int64_t)(r0 + r) * nc + col] * ub[r];
            const int s = col / 9;
            atomicAdd(yt + 9 * a.obs_cam_s[s0 + s] + (col - 9 * s), acc);
        }
        __syncwarp();
    }
}

// consumer warps a tile keeps busy (at most MV_CONSUMERS)
__device__ __forceinline__ int tile_warps(const MvTile& t, int mode, int big8_kmax) {
    int w;
    if (mode == MODE_MATVEC) {
        if (t.kind == TILE_SMALL) {
            const int tpw = 32 / small_team_width(t.k);
            w = (t.count + tpw - 1) / tpw;
        } else if (t.kind == TILE_BIG) {
            const int rpw = t.k <= big8_kmax ? 8 : 4;
            w = (t.count + rpw - 1) / rpw;
        } else {
            w = 1;
        }
    } else {
        const int slots = t.kind == TILE_SMALL ? t.count * t.k : t.k;
        w = (slots + 31) / 32;
    }
    return w < 1 ? 1 : (w > MV_CONSUMERS ? MV_CONSUMERS : w);
}

// MODE_MATVEC: y (SMEM_ACC: per-CTA copy of y in shared memory);
// MODE_PRECOND: per-observation records (SMEM_ACC false).
template <int MODE, bool SMEM_ACC, int NS>
__global__ void __launch_bounds__(MV_THREADS, 1) k_matvec_tiles(MvArgs a) {
    using L = Layout<NS, MODE == MODE_PRECOND ? 1 : 0>;
    constexpr int MV_STAGES = NS;
    extern __shared__ __align__(128) unsigned char smem[];
    if (a.S != nullptr && a.S->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ys = reinterpret_cast<float*>(smem + L::ACC_OFF);
    static_assert(MODE == MODE_MATVEC || !SMEM_ACC, "records are written to global memory");
    const int acc_n = 9 * a.n_cam;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::FLAG_OFF);
    volatile int* seq = reinterpret_cast<volatile int*>(smem + L::SEQ_OFF);
    const uint32_t bar0 = smem_u32(smem + L::BAR_OFF);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (MV_STAGES + s); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < MV_STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), MV_CONSUMERS);
        }
        *abort_flag = 0;
        for (int q = 0; q < MV_STAGES; ++q) seq[q] = -1;
        mbar_fence_init();
    }
    if (SMEM_ACC)
        for (int i = threadIdx.x; i < acc_n; i += MV_THREADS) ys[i] = 0.f;
    __syncthreads();
    float* yt = SMEM_ACC ? ys : a.y;

    const int tb = a.tile_begin[blockIdx.x], te = a.tile_begin[blockIdx.x + 1];
    if (warp == 0) {
        // producer warp: tile records are fetched 32 at a time (one coalesced
        // load, lane l holds record base + l), lane 0 issues the bulk copies
        int issued = 0;
        bool stop = false;
        for (int base = tb; base < te && !stop; base += 32) {
            MvTile mine{};
            if (base + lane < te) mine = a.tiles[base + lane];
            const int n = min(32, te - base);
            for (int q = 0; q < n; ++q) {
                MvTile tile;
                tile.a_off = __shfl_sync(0xffffffffu, mine.a_off, q);
                tile.cam_off = __shfl_sync(0xffffffffu, mine.cam_off, q);
                tile.bytes = __shfl_sync(0xffffffffu, mine.bytes, q);
                tile.k = (int16_t)__shfl_sync(0xffffffffu, (int)mine.k, q);
                tile.kind = (int16_t)__shfl_sync(0xffffffffu, (int)mine.kind, q);
                tile.count = __shfl_sync(0xffffffffu, mine.count, q);
                tile.r0 = __shfl_sync(0xffffffffu, mine.r0, q);
                tile.first = __shfl_sync(0xffffffffu, mine.first, q);
                int ok = 1;
                if (lane == 0) {
                    const int i = base + q - tb, s = i % MV_STAGES;
                    if (i == a.fail_tile && blockIdx.x == 0) {
                        ok = 0;  // test hook: this tile and the rest of the CTA's range are never issued
                    } else if (i >= MV_STAGES && !mbar_wait(empty_bar(s), ((i / MV_STAGES) - 1) & 1, abort_flag,
                                                            a.err, true, a.wait_ns)) {
                        ok = 0;
                    } else {
                        // the consumer warps the tile does not need arrive on
                        // its empty barrier here, before its data can land
                        const int need = tile_warps(tile, MODE, a.big8_kmax);
                        if (need < MV_CONSUMERS) mbar_arrive_cnt(empty_bar(s), (uint32_t)(MV_CONSUMERS - need));
                        if (tile.kind == TILE_GLOBAL) {
                            mbar_arrive(full_bar(s));
                        } else {
                            const int nc = tile.kind == TILE_SMALL ? tile.count * tile.k : tile.k;
                            const int c4 = tile.cam_off & ~3;
                            const uint32_t cbytes = (uint32_t)(((tile.cam_off - c4 + nc) * 4 + 15) & ~15);
                            // preconditioner mode: c_j values (2k per block, or the tile's rows)
                            const int64_t r_first = 2LL * tile.cam_off + (tile.kind == TILE_BIG ? tile.r0 : 0);
                            const int r_n = tile.kind == TILE_SMALL ? 2 * tile.k * tile.count : tile.count;
                            const int64_t r4 = r_first & ~3LL;
                            const uint32_t rbytes =
                                MODE == MODE_PRECOND ? (uint32_t)(((r_first - r4 + r_n) * 4 + 15) & ~15) : 0u;
                            mbar_expect_tx(full_bar(s), (uint32_t)tile.bytes + cbytes + rbytes);
                            bulk_g2s(smem_u32(smem + s * MV_STAGE_A), a.apool + tile.a_off, (uint32_t)tile.bytes,
                                     full_bar(s));
                            bulk_g2s(smem_u32(smem + L::STAGE_C_OFF + s * MV_STAGE_C), a.mv_cam + c4, cbytes,
                                     full_bar(s));
                            if (MODE == MODE_PRECOND)
                                bulk_g2s(smem_u32(smem + L::STAGE_R_OFF + s * MV_STAGE_R), a.cpool + r4, rbytes,
                                         full_bar(s));
                        }
                        seq[s] = i;  // stage s is armed with tile i
                        ++issued;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    stop = true;
                    break;
                }
            }
        }
        if (lane == 0 && (stop || *abort_flag)) {
            // let the copies already issued land before the CTA exits
            for (int i = max(0, issued - MV_STAGES); i < issued; ++i)
                mbar_wait(full_bar(i % MV_STAGES), (i / MV_STAGES) & 1, abort_flag, a.err, false);
        }
    } else {
        const int cw = warp - 1;
        // Each consumer warp reads the tile records itself and works only on
        // the tiles that need it: successive tiles take successive groups of
        // warps (cyclically), so that the tiles in flight are worked on by
        // disjoint warps.  The producer arrives on a tile's empty barrier for
        // the warps the tile does not need, so a stage is released as soon as
        // its own warps are done.  A warp that skipped tiles first waits until
        // the producer has armed the stage with its tile (seq), so that the
        // parity wait on the full barrier that follows is exact.
        int start = 0;  // first consumer warp of the current tile
        bool stop = false;
        for (int base = tb; base < te && !stop; base += 32) {
            MvTile mine{};
            if (base + lane < te) mine = a.tiles[base + lane];
            const int n = min(32, te - base);
            for (int q = 0; q < n; ++q) {
                MvTile tile;
                tile.a_off = __shfl_sync(0xffffffffu, mine.a_off, q);
                tile.cam_off = __shfl_sync(0xffffffffu, mine.cam_off, q);
                tile.bytes = __shfl_sync(0xffffffffu, mine.bytes, q);
                tile.k = (int16_t)__shfl_sync(0xffffffffu, (int)mine.k, q);
                tile.kind = (int16_t)__shfl_sync(0xffffffffu, (int)mine.kind, q);
                tile.count = __shfl_sync(0xffffffffu, mine.count, q);
                tile.r0 = __shfl_sync(0xffffffffu, mine.r0, q);
                tile.first = __shfl_sync(0xffffffffu, mine.first, q);
                const int need = tile_warps(tile, MODE, a.big8_kmax);
                const int vcw = (cw - start + MV_CONSUMERS) % MV_CONSUMERS;
                start = (start + need) % MV_CONSUMERS;
                if (vcw >= need) continue;
                const int i = base + q - tb, s = i % MV_STAGES;
                if (!seq_wait(seq + s, i, abort_flag, a.err, a.wait_ns) ||
                    !mbar_wait(full_bar(s), (i / MV_STAGES) & 1, abort_flag, a.err, true, a.wait_ns)) {
                    stop = true;
                    break;
                }
                const float* sa = reinterpret_cast<const float*>(smem + s * MV_STAGE_A);
                const int32_t* sc = reinterpret_cast<const int32_t*>(smem + L::STAGE_C_OFF + s * MV_STAGE_C) +
                                    (tile.cam_off & 3);
                float* ub = reinterpret_cast<float*>(smem + L::U_OFF) + s * MV_UMAX;
                if (MODE == MODE_MATVEC) {
                    if (tile.kind == TILE_SMALL) small_dispatch(tile.k, sa, sc, tile.count, a.v, yt, vcw, lane);
                    else if (tile.kind == TILE_BIG && tile.k <= a.big8_kmax)
                        big_tile<8>(sa, sc, tile.k, tile.count, a.v, yt, vcw, lane);
                    else if (tile.kind == TILE_BIG) big_tile<4>(sa, sc, tile.k, tile.count, a.v, yt, vcw, lane);
                    else if (vcw == 0) global_block(a, tile.first, ub, yt, lane);
                } else {
                    const int tid = vcw * 32 + lane;
                    const int64_t r_first = 2LL * tile.cam_off + (tile.kind == TILE_BIG ? tile.r0 : 0);
                    const float* sr = reinterpret_cast<const float*>(smem + L::STAGE_R_OFF + s * MV_STAGE_R) + (r_first & 3);
                    if (tile.kind == TILE_SMALL) precond_blocks(a, tile, sa, sc, sr, tid);
                    else if (tile.kind == TILE_BIG) precond_rows(a, tile, sa, sc, sr, tid);
                    else precond_global(a, tile, tid);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_bar(s));
            }
        }
    }
    __syncthreads();
    if (MODE == MODE_MATVEC && SMEM_ACC) {
        // the CTAs flush at nearly the same time: each starts at its own
        // offset, so that concurrent atomics go to different addresses
        const int i0 = (int)(((int64_t)blockIdx.x * acc_n) / gridDim.x);
        for (int q = threadIdx.x; q < acc_n; q += MV_THREADS) {
            const int i = q + i0 < acc_n ? q + i0 : q + i0 - acc_n;
            const float val = ys[i];
            if (val != 0.f) atomicAdd(a.y + i, val);
        }
    }
}

__global__ void k_add_damping(int n, const float* __restrict__ dp2, float lam, const float* __restrict__ v,
                              float* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += lam * dp2[i] * v[i];
}

// Pipeline depths built: 4, 5 and 6 stages of 32 KB (the planner's tiles do
// not depend on the depth; the autotuner picks it per plan).
template <int PC>
int acc_off_pc(int ns) {
    return ns == 6 ? Layout<6, PC>::ACC_OFF : ns == 5 ? Layout<5, PC>::ACC_OFF : Layout<4, PC>::ACC_OFF;
}
int acc_off(int ns, bool pc) { return pc ? acc_off_pc<1>(ns) : acc_off_pc<0>(ns); }
bool y_fits(const Problem& p, int ns) { return acc_off(ns, false) + 36 * (int64_t)p.n_cam <= SMEM_LIMIT; }
// the depth in use: the plan's, unless the options force one
int depth(const Problem& p, const Problem::TilePlan& plan) {
    return p.opt.pipeline_stages ? p.opt.pipeline_stages : plan.ns;
}
// y is accumulated in shared memory when the plan asks for it and it fits
bool smem_y(const Problem& p, const Problem::TilePlan& plan) { return plan.y_smem && y_fits(p, depth(p, plan)); }
size_t smem_bytes(const Problem& p, const Problem::TilePlan& plan, bool pc) {
    return acc_off(depth(p, plan), pc) + (!pc && smem_y(p, plan) ? 36 * (size_t)p.n_cam : 0);
}

using MvKernel = void (*)(MvArgs);
template <int NS>
MvKernel kernel_ns(bool pc, bool y) {
    if (pc) return k_matvec_tiles<MODE_PRECOND, false, NS>;
    return y ? k_matvec_tiles<MODE_MATVEC, true, NS> : k_matvec_tiles<MODE_MATVEC, false, NS>;
}
MvKernel pick_kernel(const Problem& p, const Problem::TilePlan& plan, bool pc) {
    const bool y = !pc && smem_y(p, plan);
    const int ns = depth(p, plan);
    return ns == 6 ? kernel_ns<6>(pc, y) : ns == 5 ? kernel_ns<5>(pc, y) : kernel_ns<4>(pc, y);
}

MvArgs make_args(Problem& p, const Problem::TilePlan& plan, const float* v, float* y, const PcgScalars* S) {
    return MvArgs{static_cast<const MvTile*>(plan.tiles), plan.begin, p.apool, p.mv_cam, p.lm_by_k, p.pt_off,
                  p.obs_cam_s, p.a_off, v, y, p.n_cam, S, p.err, p.cpool, p.prec, plan.big8_kmax,
                  p.dbg_wait_ns > 0 ? p.dbg_wait_ns : WAIT_NS, &plan == &p.mv_plan ? p.dbg_fail_tile : -1};
}

}  // namespace

// rows of one big tile of a k-block (a multiple of 4)
int big_tile_rows(int k) { return std::min(MV_UMAX & ~3, (MV_STAGE_A / (36 * k)) & ~3); }

// Host planning of the tiles: runs of equal-k blocks in storage order
// (decreasing k), cut into stage-sized tiles, then contiguous tile ranges per
// CTA balanced by bytes.
void plan_tiles(Problem& p, bool pc) {
    Problem::TilePlan& plan = pc ? p.pc_plan : p.mv_plan;
    std::vector<MvTile> tiles;
    const int kmax = p.k_max;
    // records of blocks that are split into row tiles are accumulated
    // atomically: the observations of the landmarks with k above the
    // smallest split k, which come first in storage order, are zeroed before
    // each preconditioner pass (the records of unsplit blocks are stored)
    const int ksmall = std::min(plan.ksmall, MV_KSMALL_MAX);
    const int small_bytes = std::min(plan.small_bytes, MV_STAGE_A);
    plan.n_obs_split = 0;
    auto whole = [&](int k) { return k <= ksmall && 4 * pad4(18LL * k * k) <= MV_STAGE_A; };
    for (int b = 0; b <= kmax && !whole(kmax - b); ++b)
        if (big_tile_rows(kmax - b) < 2 * (kmax - b)) plan.n_obs_split = p.run_co[b + 1];
    for (int b = 0; b <= kmax; ++b) {
        const int k = kmax - b;
        const int64_t cnt = p.k_run_count[b];
        if (cnt == 0 || k < 2) continue;
        const int64_t bf = pad4(18LL * k * k);
        const int64_t pos0 = [&] {
            int64_t q = 0;
            for (int bb = 0; bb < b; ++bb) q += p.k_run_count[bb];
            return q;
        }();
        if (whole(k)) {  // a whole block must fit one stage
            const int64_t per = std::max<int64_t>(1, small_bytes / (4 * bf));
            for (int64_t l = 0; l < cnt; l += per) {
                MvTile t{};
                const int64_t n = std::min(per, cnt - l);
                t.a_off = p.run_off[b] + l * bf;
                t.cam_off = (int32_t)(p.run_co[b] + l * k);
                t.bytes = (int32_t)(4 * n * bf);
                t.k = (int16_t)k;
                t.kind = TILE_SMALL;
                t.count = (int32_t)n;
                t.first = (int32_t)(pos0 + l);
                tiles.push_back(t);
            }
        } else if (k <= MV_KBIG) {
            const int nc = 9 * k, nr = 2 * k;
            // the fewest row tiles that fit a stage, of near-equal size
            // (multiples of 4 rows keep every tile 16-byte aligned)
            const int maxr = big_tile_rows(k), nt = (nr + maxr - 1) / maxr;
            const int rows = std::min(maxr, ((nr + nt - 1) / nt + 3) & ~3);
            for (int64_t l = 0; l < cnt; ++l) {
                for (int r0 = 0; r0 < nr; r0 += rows) {
                    MvTile t{};
                    const int n = std::min(rows, nr - r0);
                    t.a_off = p.run_off[b] + l * bf + (int64_t)r0 * nc;
                    t.cam_off = (int32_t)(p.run_co[b] + l * k);
                    t.bytes = (int32_t)((4LL * n * nc + 15) & ~15LL);
                    t.k = (int16_t)k;
                    t.kind = TILE_BIG;
                    t.count = n;
                    t.r0 = r0;
                    t.first = (int32_t)(pos0 + l);
                    tiles.push_back(t);
                }
            }
        } else {
            for (int64_t l = 0; l < cnt; ++l) {
                MvTile t{};
                t.k = (int16_t)std::min(k, 32767);
                t.kind = TILE_GLOBAL;
                t.count = 1;
                t.first = (int32_t)(pos0 + l);
                // first observation in storage order: the record pass writes
                // the block's records there and reads its c_j from there
                t.cam_off = (int32_t)(p.run_co[b] + l * k);
                t.bytes = 0;
                tiles.push_back(t);
            }
        }
    }
    // CTA b takes tiles b, b + G, b + 2G, ... of the k-sorted list, so every
    // SM gets the same mix of block sizes (work per byte differs strongly with
    // k); stored as contiguous ranges of a permuted list
    const int grid = p.mv_grid;
    std::vector<MvTile> perm;
    perm.reserve(tiles.size());
    std::vector<int32_t> begin(grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        begin[c] = (int32_t)perm.size();
        for (size_t i = c; i < tiles.size(); i += grid) perm.push_back(tiles[i]);
    }
    begin[grid] = (int32_t)perm.size();
    tiles.swap(perm);
    plan.n = (int)tiles.size();
    if (!plan.tiles || plan.cap < plan.n) {
        // re-planning (autotuner) reuses the allocation when it is large enough
        plan.cap = std::max(1, plan.n);
        plan.tiles = dalloc<MvTile>(p, plan.cap);
    }
    if (!plan.begin) plan.begin = dalloc<int32_t>(p, grid + 1);
    if (!tiles.empty())
        BA_CUDA_TRY(cudaMemcpyAsync(plan.tiles, tiles.data(), sizeof(MvTile) * tiles.size(), cudaMemcpyHostToDevice,
                                    p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(plan.begin, begin.data(), sizeof(int32_t) * (grid + 1), cudaMemcpyHostToDevice,
                                p.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
}

void plan_matvec(Problem& p) {
    plan_tiles(p, false);
    plan_tiles(p, true);
}

int matvec_ctas_per_sm() { return 1; }
int matvec_ksmall_limit() { return MV_KSMALL_MAX; }
bool matvec_y_in_smem(const Problem& p) { return smem_y(p, p.mv_plan); }
int matvec_stage_bytes() { return MV_STAGE_A; }

void configure_matvec(Problem&) {
    // every variant may take the whole opt-in shared memory: the attribute is
    // per kernel, not per problem, so it must hold for any problem's plan
    for (int ns = 4; ns <= 6; ++ns)
        for (int v = 0; v < 3; ++v) {
            const MvKernel k = ns == 6 ? kernel_ns<6>(v == 2, v == 1) : ns == 5 ? kernel_ns<5>(v == 2, v == 1)
                                                                          : kernel_ns<4>(v == 2, v == 1);
            BA_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT));
        }
}

void launch_matvec_raw(Problem& p, const float* v, float* y, const PcgScalars* S) {
    if (p.implicit) {
        launch_matvec_implicit(p, v, y, S);
        return;
    }
    if (p.schur) {
        launch_schur_matvec(p, v, y, S);
        return;
    }
    const MvArgs a = make_args(p, p.mv_plan, v, y, S);
    pick_kernel(p, p.mv_plan, false)<<<p.mv_grid, MV_THREADS, smem_bytes(p, p.mv_plan, false), p.stream>>>(a);
    BA_LAUNCH_CHECK();
}

// K3, first half, streamed through the same tile pipeline: one record of
// REC floats per observation (A_s^T A_s upper triangle and A_s^T c_j), in
// storage order.  Records of blocks split over row tiles are accumulated, so
// their prefix is zeroed first.
void launch_precond_records(Problem& p) {
    if (!p.prec) p.prec = dalloc<float>(p, REC_STRIDE * p.n_obs);  // on first use
    const MvArgs a = make_args(p, p.pc_plan, nullptr, nullptr, nullptr);
    if (p.pc_plan.n_obs_split > 0)
        BA_CUDA_TRY(cudaMemsetAsync(p.prec, 0, sizeof(float) * REC_STRIDE * p.pc_plan.n_obs_split, p.stream));
    pick_kernel(p, p.pc_plan, true)<<<p.mv_grid, MV_THREADS, smem_bytes(p, p.pc_plan, true), p.stream>>>(a);
    BA_LAUNCH_CHECK();
}

void launch_matvec(Problem& p, const float* v, float* y, bool add_damping) {
    count_launches(p, 1 + (add_damping ? 1 : 0));
    BA_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(float) * 9 * p.n_cam, p.stream));
    launch_matvec_raw(p, v, y, nullptr);
    if (add_damping) {
        k_add_damping<<<ceil_div(9 * (int64_t)p.n_cam, 256), 256, 0, p.stream>>>(9 * p.n_cam, p.dp2,
                                                                                 (float)p.lambda_damped, v, y);
        BA_LAUNCH_CHECK();
    }
}

}  // namespace sqrtba
