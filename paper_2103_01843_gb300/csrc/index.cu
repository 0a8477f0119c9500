// K0: input validation and grouping of the observations by landmark
// (Sec. 5.1: "we group the residuals by landmarks"), plus the camera-side
// index and the landmark-block offsets.  Integer work; the result is unique
// (observations sorted by (landmark, camera), camera lists in increasing
// sorted position), so it is bit-exact whatever the thread schedule.
#include <algorithm>
#include <vector>

#include "problem.cuh"

namespace sqrtba {

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_PER = 16;
constexpr int SCAN_B = SCAN_T * SCAN_PER;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        sh[32 + lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) sh[64] = wi;
    }
    __syncthreads();
    total = sh[64];
    int64_t res = sh[32 + wid] + inc - v;
    __syncthreads();
    return res;
}

template <typename TIn>
__global__ void k_scan_blocksum(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
    __shared__ int64_t sh[65];
    const int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_PER;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    int64_t total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_bsums(int64_t* bsum, int nb) {
    __shared__ int64_t sh[65];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t total;
        int64_t ex = block_exclusive_scan(v, sh, total);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

template <typename TIn, typename TOut>
__global__ void k_scan_final(const TIn* __restrict__ in, int64_t n, const int64_t* __restrict__ bex,
                             TOut* __restrict__ out) {
    __shared__ int64_t sh[65];
    const int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_PER;
    int64_t vals[SCAN_PER];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        vals[i] = base + i < n ? (int64_t)in[base + i] : 0;
        s += vals[i];
    }
    int64_t total;
    int64_t run = bex[blockIdx.x] + block_exclusive_scan(s, sh, total);
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        if (base + i < n) out[base + i] = (TOut)run;
        if (base + i == n - 1) out[n] = (TOut)(run + vals[i]);
        run += vals[i];
    }
}

// exclusive scan of n values into out[0..n]; tmp holds >= ceil(n / SCAN_B) int64
template <typename TIn, typename TOut>
void exclusive_scan(const TIn* in, int64_t n, TOut* out, int64_t* tmp, cudaStream_t st) {
    if (n <= 0) {
        BA_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(TOut), st));
        return;
    }
    const int nb = ceil_div(n, SCAN_B);
    k_scan_blocksum<TIn><<<nb, SCAN_T, 0, st>>>(in, n, tmp);
    k_scan_bsums<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_final<TIn, TOut><<<nb, SCAN_T, 0, st>>>(in, n, tmp, out);
    BA_LAUNCH_CHECK();
}

__global__ void k_convert_params(const double* __restrict__ in, int64_t n, float* __restrict__ out,
                                 uint32_t* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i];
        if (!isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
        out[i] = (float)v;
    }
}

__global__ void k_validate_count(const int32_t* __restrict__ oc, const int32_t* __restrict__ op,
                                 const double* __restrict__ xy, int64_t n, int n_cam, int n_pt,
                                 int32_t* cnt_pt, int32_t* cnt_cam, uint32_t* err) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int c = oc[o], j = op[o];
        if (c < 0 || c >= n_cam || j < 0 || j >= n_pt) {
            atomicOr(err, ERRBIT_INDEX);
            continue;
        }
        if (!isfinite(xy[2 * o]) || !isfinite(xy[2 * o + 1])) atomicOr(err, ERRBIT_NONFINITE);
        atomicAdd(&cnt_pt[j], 1);
        atomicAdd(&cnt_cam[c], 1);
    }
}

// observation o into its landmark's segment as the key (camera << 32 | o):
// the segment sorts then compare one contiguous array (camera first, the
// observation index breaks ties, so every key is unique)
__global__ void k_scatter_pt(const int32_t* __restrict__ op, const int32_t* __restrict__ oc, int64_t n,
                             const int32_t* __restrict__ pt_off, int32_t* cursor, uint64_t* __restrict__ kv) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int j = op[o];
        const int pos = pt_off[j] + atomicAdd(&cursor[j], 1);
        kv[pos] = ((uint64_t)(uint32_t)oc[o] << 32) | (uint64_t)(uint32_t)o;
    }
}

__device__ __forceinline__ void write_sorted(int i, int j, uint64_t key, const double* __restrict__ xy,
                                             int32_t* __restrict__ perm, int32_t* __restrict__ obs_cam_s,
                                             int32_t* __restrict__ obs_pt_s, float2* __restrict__ obs_xy_s) {
    const int o = (int)(uint32_t)key;
    perm[i] = o;
    obs_cam_s[i] = (int)(key >> 32);
    obs_pt_s[i] = j;
    obs_xy_s[i] = make_float2((float)xy[2 * o], (float)xy[2 * o + 1]);
}

// One thread per landmark: its size, the checks (k < 2), and for k <= 32 the
// order of its observations by camera (insertion sort of the keys), the
// duplicate check and the sorted observation arrays; k > 32 is left to
// k_sort_segments_big.
__global__ void k_sort_segments(int n_pt, const int32_t* __restrict__ pt_off, uint64_t* kv,
                                const double* __restrict__ xy, int32_t* __restrict__ perm,
                                int32_t* __restrict__ obs_cam_s, int32_t* __restrict__ obs_pt_s,
                                float2* __restrict__ obs_xy_s, int32_t* __restrict__ kcount, int32_t* kmax,
                                int32_t* nbig, uint32_t* err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pt) return;
    const int a = pt_off[j], b = pt_off[j + 1], k = b - a;
    kcount[j] = k;
    atomicMax(kmax, k);
    if (k > 32) {
        atomicAdd(nbig, 1);
        return;
    }
    if (k < 2) atomicOr(err, ERRBIT_FEWOBS);
    for (int i = a + 1; i < b; ++i) {
        const uint64_t v = kv[i];
        int m = i - 1;
        while (m >= a && kv[m] > v) {
            kv[m + 1] = kv[m];
            --m;
        }
        kv[m + 1] = v;
    }
    uint64_t prev = ~0ull;
    for (int i = a; i < b; ++i) {
        const uint64_t key = kv[i];
        if ((key >> 32) == (prev >> 32)) atomicOr(err, ERRBIT_DUPLICATE);
        prev = key;
        write_sorted(i, j, key, xy, perm, obs_cam_s, obs_pt_s, obs_xy_s);
    }
}

// k > 32: one warp per landmark, each key placed at its rank among the
// segment's keys (the keys are unique), then the duplicate check against the
// neighbour in the sorted order.
__global__ void k_sort_segments_big(int n_pt, const int32_t* __restrict__ pt_off, const uint64_t* __restrict__ kv,
                                    const double* __restrict__ xy, int32_t* __restrict__ perm,
                                    int32_t* __restrict__ obs_cam_s, int32_t* __restrict__ obs_pt_s,
                                    float2* __restrict__ obs_xy_s, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (j >= n_pt) return;
    const int a = pt_off[j], k = pt_off[j + 1] - a;
    if (k <= 32) return;  // whole warp
    for (int i = lane; i < k; i += 32) {
        const uint64_t key = kv[a + i];
        int rank = 0;
        for (int m = 0; m < k; ++m) rank += kv[a + m] < key ? 1 : 0;
        write_sorted(a + rank, j, key, xy, perm, obs_cam_s, obs_pt_s, obs_xy_s);
    }
    __syncwarp();
    for (int i = a + 1 + lane; i < a + k; i += 32)
        if (obs_cam_s[i] == obs_cam_s[i - 1]) atomicOr(err, ERRBIT_DUPLICATE);
}

// --- camera lists: a stable counting sort by camera over tiles --------------
__global__ void k_tile_hist(const int32_t* __restrict__ cam_s, int64_t n, int n_cam, int tile,
                            int32_t* hist) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[(s / tile) * n_cam + cam_s[s]], 1);
}

// One warp per camera: its counts over the tiles turned into the tiles'
// running bases (an exclusive scan in tile order, 32 tiles per step)
__global__ void k_tile_base(int32_t* hist, int n_tiles, int n_cam, const int32_t* __restrict__ cam_off) {
    const int lane = threadIdx.x & 31;
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= n_cam) return;  // whole warp
    int run = cam_off[c];
    for (int t0 = 0; t0 < n_tiles; t0 += 32) {
        const int t = t0 + lane;
        const int64_t i = (int64_t)t * n_cam + c;
        const int h = t < n_tiles ? hist[i] : 0;
        int inc = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (t < n_tiles) hist[i] = run + inc - h;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// one warp per tile, 32 observations at a time in increasing order
__global__ void k_tile_place(const int32_t* __restrict__ cam_s, int64_t n, int n_cam, int tile,
                             int n_tiles, int32_t* base, int32_t* __restrict__ cam_list) {
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n_tiles) return;
    const int64_t s_end = min((int64_t)(t + 1) * tile, n);
    for (int64_t c0 = (int64_t)t * tile; c0 < s_end; c0 += 32) {
        const int64_t s = c0 + lane;
        const bool valid = s < s_end;
        const int cam = valid ? cam_s[s] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, cam);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1u));
        int b = 0;
        if (valid && lane == leader) b = base[(int64_t)t * n_cam + cam];
        b = __shfl_sync(0xffffffffu, b, leader);
        if (valid) cam_list[b + rank] = (int32_t)s;
        if (valid && lane == leader) base[(int64_t)t * n_cam + cam] = b + __popc(grp);
        __syncwarp();
    }
}

// --- block sizes and work lists ---------------------------------------------
__global__ void k_ksq(int n_pt, const int32_t* __restrict__ kcount, int64_t* __restrict__ k2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pt) return;
    const int64_t k = kcount[j];
    k2[j] = k * k;
}

__global__ void k_khist(int n_pt, const int32_t* __restrict__ kcount, int kmax, int32_t* hist) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pt) return;
    atomicAdd(&hist[kmax - kcount[j]], 1);  // decreasing k
}

__global__ void k_kscatter(int n_pt, const int32_t* __restrict__ kcount, int kmax,
                           const int32_t* __restrict__ koff, int32_t* cursor, int32_t* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pt) return;
    const int b = kmax - kcount[j];
    out[koff[b] + atomicAdd(&cursor[b], 1)] = j;
}

// Block offsets in storage order (decreasing k, then the order of lm_by_k)
// and the cameras of every observation in that order (the matvec's stream).
__global__ void k_storage(int n_pt, const int32_t* __restrict__ order, const int32_t* __restrict__ kcount,
                          int kmax, const int32_t* __restrict__ ko, const int64_t* __restrict__ run_off,
                          const int64_t* __restrict__ run_co, const int32_t* __restrict__ pt_off,
                          const int32_t* __restrict__ obs_cam_s, int64_t* __restrict__ a_off,
                          int32_t* __restrict__ mv_cam, int32_t* __restrict__ c_off,
                          int32_t* __restrict__ obs_store, int32_t* __restrict__ lm_pos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pt) return;
    const int j = order[i];
    lm_pos[j] = i;
    const int64_t k = kcount[j];
    const int b = kmax - (int)k;
    const int64_t idx = i - ko[b];
    a_off[j] = run_off[b] + idx * pad4(18 * k * k);
    const int64_t co = run_co[b] + idx * k;
    const int s0 = pt_off[j];
    c_off[j] = (int32_t)(2 * co);
    for (int s = 0; s < k; ++s) {
        mv_cam[co + s] = obs_cam_s[s0 + s];
        obs_store[s0 + s] = (int32_t)(co + s);
    }
}

__global__ void k_map_list(int64_t n, const int32_t* __restrict__ list, const int32_t* __restrict__ map,
                           int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = map[list[e]];
}

__global__ void k_chunk_count(int n_cam, const int32_t* __restrict__ cam_off, int32_t* __restrict__ cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cam) cnt[c] = (cam_off[c + 1] - cam_off[c] + PG_CHUNK - 1) / PG_CHUNK;
}

__global__ void k_chunk_fill(int n_cam, const int32_t* __restrict__ chunk_off, int32_t* __restrict__ chunk_cam) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cam) return;
    for (int q = chunk_off[c]; q < chunk_off[c + 1]; ++q) chunk_cam[q] = c;
}

}  // namespace

void build_index(Problem& p, const int32_t* d_oc, const int32_t* d_op, const double* d_xy,
                 const double* d_cams, const double* d_pts) {
    cudaStream_t st = p.stream;
    const int64_t n = p.n_obs;
    const int TPB = 256;
    const int gsz = std::max(1, std::min(ceil_div(n, TPB), p.sm_count * 8));

    // temporaries, freed at the end of this call
    std::vector<void*> tmps;
    auto tmp_alloc = [&](size_t bytes) {
        void* ptr = nullptr;
        BA_CUDA_TRY(cudaMallocFromPoolAsync(&ptr, bytes ? bytes : 1, device_pool(), st));
        tmps.push_back(ptr);
        return ptr;
    };
    struct Guard {
        std::vector<void*>* v;
        cudaStream_t st;
        ~Guard() {
            for (void* q : *v) cudaFreeAsync(q, st);
        }
    } guard{&tmps, st};

    int32_t* cnt_pt = (int32_t*)tmp_alloc(sizeof(int32_t) * (p.n_pt + 1));
    int32_t* cnt_cam = (int32_t*)tmp_alloc(sizeof(int32_t) * (p.n_cam + 1));
    int64_t* scan_tmp = (int64_t*)tmp_alloc(sizeof(int64_t) * (ceil_div(n + p.n_pt + p.n_cam + 1, SCAN_B) + 2));
    BA_CUDA_TRY(cudaMemsetAsync(cnt_pt, 0, sizeof(int32_t) * (p.n_pt + 1), st));
    BA_CUDA_TRY(cudaMemsetAsync(cnt_cam, 0, sizeof(int32_t) * (p.n_cam + 1), st));
    BA_CUDA_TRY(cudaMemsetAsync(p.err, 0, sizeof(uint32_t), st));

    k_convert_params<<<gsz, TPB, 0, st>>>(d_cams, 9 * (int64_t)p.n_cam, p.cams, p.err);
    k_convert_params<<<gsz, TPB, 0, st>>>(d_pts, 3 * (int64_t)p.n_pt, p.pts, p.err);
    k_validate_count<<<gsz, TPB, 0, st>>>(d_oc, d_op, d_xy, n, p.n_cam, p.n_pt, cnt_pt, cnt_cam, p.err);
    BA_LAUNCH_CHECK();
    uint32_t herr = 0;
    BA_CUDA_TRY(cudaMemcpyAsync(&herr, p.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & ERRBIT_INDEX) throw Error{BA_ERR_INVALID_ARG, "observation index out of range"};
    if (herr & ERRBIT_NONFINITE) throw Error{BA_ERR_INVALID_ARG, "non-finite camera, point or observation value"};

    exclusive_scan(cnt_pt, p.n_pt, p.pt_off, scan_tmp, st);
    exclusive_scan(cnt_cam, p.n_cam, p.cam_off, scan_tmp, st);

    int32_t* cursor = cnt_pt;  // reuse as scatter cursors
    BA_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (p.n_pt + 1), st));
    uint64_t* kv = (uint64_t*)tmp_alloc(sizeof(uint64_t) * n);
    k_scatter_pt<<<gsz, TPB, 0, st>>>(d_op, d_oc, n, p.pt_off, cursor, kv);
    int32_t* kcount = (int32_t*)tmp_alloc(sizeof(int32_t) * (p.n_pt + 1));
    int32_t* kmax_d = (int32_t*)tmp_alloc(2 * sizeof(int32_t));
    BA_CUDA_TRY(cudaMemsetAsync(kmax_d, 0, 2 * sizeof(int32_t), st));
    k_sort_segments<<<ceil_div(p.n_pt, 128), 128, 0, st>>>(p.n_pt, p.pt_off, kv, d_xy, p.perm, p.obs_cam_s,
                                                           p.obs_pt_s, p.obs_xy_s, kcount, kmax_d, kmax_d + 1,
                                                           p.err);
    k_sort_segments_big<<<ceil_div((int64_t)p.n_pt * 32, 128), 128, 0, st>>>(p.n_pt, p.pt_off, kv, d_xy, p.perm,
                                                                              p.obs_cam_s, p.obs_pt_s,
                                                                              p.obs_xy_s, p.err);
    BA_LAUNCH_CHECK();

    // camera lists
    int64_t n_tiles = std::max<int64_t>(1, std::min<int64_t>((n + 2047) / 2048, ((int64_t)1 << 25) / p.n_cam));
    int64_t tile = ((n + n_tiles - 1) / n_tiles + 31) / 32 * 32;
    n_tiles = std::max<int64_t>(1, (n + tile - 1) / tile);
    int32_t* hist = (int32_t*)tmp_alloc(sizeof(int32_t) * n_tiles * p.n_cam);
    BA_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int32_t) * n_tiles * p.n_cam, st));
    k_tile_hist<<<gsz, TPB, 0, st>>>(p.obs_cam_s, n, p.n_cam, (int)tile, hist);
    k_tile_base<<<ceil_div((int64_t)p.n_cam * 32, 128), 128, 0, st>>>(hist, (int)n_tiles, p.n_cam, p.cam_off);
    k_tile_place<<<ceil_div(n_tiles * 32, 128), 128, 0, st>>>(p.obs_cam_s, n, p.n_cam, (int)tile,
                                                              (int)n_tiles, hist, p.cam_list);
    BA_LAUNCH_CHECK();

    // sum of k^2 (reported), error checks and k_max
    int64_t* k2 = (int64_t*)tmp_alloc(sizeof(int64_t) * (p.n_pt + 1));
    int64_t* k2off = (int64_t*)tmp_alloc(sizeof(int64_t) * (p.n_pt + 1));
    k_ksq<<<ceil_div(p.n_pt, 256), 256, 0, st>>>(p.n_pt, kcount, k2);
    exclusive_scan(k2, p.n_pt, k2off, scan_tmp, st);

    int32_t kinfo[2] = {0, 0};
    int64_t sumk2 = 0;
    BA_CUDA_TRY(cudaMemcpyAsync(&herr, p.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemcpyAsync(kinfo, kmax_d, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemcpyAsync(&sumk2, k2off + p.n_pt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & ERRBIT_FEWOBS) throw Error{BA_ERR_INVALID_ARG, "a landmark has fewer than two observations"};
    if (herr & ERRBIT_DUPLICATE) throw Error{BA_ERR_INVALID_ARG, "duplicate (camera, landmark) observation"};
    const int32_t kmax = kinfo[0];
    p.k_max = kmax;
    p.n_big = kinfo[1];
    p.sum_k2 = sumk2;

    // landmarks by decreasing k; the work order of the per-landmark kernels
    // and the storage order of the landmark blocks (equal-k blocks adjacent)
    int32_t* kh = (int32_t*)tmp_alloc(sizeof(int32_t) * (kmax + 2));
    int32_t* ko = (int32_t*)tmp_alloc(sizeof(int32_t) * (kmax + 2));
    BA_CUDA_TRY(cudaMemsetAsync(kh, 0, sizeof(int32_t) * (kmax + 2), st));
    k_khist<<<ceil_div(p.n_pt, 256), 256, 0, st>>>(p.n_pt, kcount, kmax, kh);
    exclusive_scan(kh, kmax + 1, ko, scan_tmp, st);
    p.k_run_count.assign(kmax + 1, 0);
    BA_CUDA_TRY(cudaMemcpyAsync(p.k_run_count.data(), kh, sizeof(int32_t) * (kmax + 1), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaMemsetAsync(kh, 0, sizeof(int32_t) * (kmax + 2), st));
    k_kscatter<<<ceil_div(p.n_pt, 256), 256, 0, st>>>(p.n_pt, kcount, kmax, ko, kh, p.lm_by_k);
    BA_LAUNCH_CHECK();
    BA_CUDA_TRY(cudaStreamSynchronize(st));

    // run b holds the landmarks with k = kmax - b: block offsets (floats) and
    // offsets into the camera stream of the matvec (one int per observation)
    p.run_off.assign(kmax + 2, 0);
    p.run_co.assign(kmax + 2, 0);
    for (int b = 0; b <= kmax; ++b) {
        const int64_t k = kmax - b, cnt = p.k_run_count[b];
        p.run_off[b + 1] = p.run_off[b] + cnt * pad4(18 * k * k);
        p.run_co[b + 1] = p.run_co[b] + cnt * k;
    }
    p.a_floats = p.run_off[kmax + 1];
    int64_t* d_run = (int64_t*)tmp_alloc(sizeof(int64_t) * 2 * (kmax + 2));
    BA_CUDA_TRY(cudaMemcpyAsync(d_run, p.run_off.data(), sizeof(int64_t) * (kmax + 2), cudaMemcpyHostToDevice, st));
    BA_CUDA_TRY(cudaMemcpyAsync(d_run + kmax + 2, p.run_co.data(), sizeof(int64_t) * (kmax + 2),
                                cudaMemcpyHostToDevice, st));
    BA_CUDA_TRY(cudaMemcpyAsync(p.a_off + p.n_pt, &p.run_off[kmax + 1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int32_t* obs_store = (int32_t*)tmp_alloc(sizeof(int32_t) * n);
    p.lm_pos = dalloc<int32_t>(p, p.n_pt);
    k_storage<<<ceil_div(p.n_pt, 256), 256, 0, st>>>(p.n_pt, p.lm_by_k, kcount, kmax, ko, d_run, d_run + kmax + 2,
                                                     p.pt_off, p.obs_cam_s, p.a_off, p.mv_cam, p.c_off, obs_store,
                                                     p.lm_pos);
    k_map_list<<<gsz, TPB, 0, st>>>(n, p.cam_list, obs_store, p.cam_list_st);
    BA_LAUNCH_CHECK();

    // chunks of the camera lists for the Gram-form preconditioner
    int32_t* nch = (int32_t*)tmp_alloc(sizeof(int32_t) * (p.n_cam + 1));
    k_chunk_count<<<ceil_div(p.n_cam, 256), 256, 0, st>>>(p.n_cam, p.cam_off, nch);
    p.pg_chunk_off = dalloc<int32_t>(p, p.n_cam + 1);
    exclusive_scan(nch, p.n_cam, p.pg_chunk_off, scan_tmp, st);
    BA_CUDA_TRY(cudaMemcpyAsync(&p.pg_chunks, p.pg_chunk_off + p.n_cam, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BA_CUDA_TRY(cudaStreamSynchronize(st));
    p.pg_chunk_cam = dalloc<int32_t>(p, p.pg_chunks);
    p.pg_part = dalloc<float>(p, 56LL * p.pg_chunks);
    k_chunk_fill<<<ceil_div(p.n_cam, 256), 256, 0, st>>>(p.n_cam, p.pg_chunk_off, p.pg_chunk_cam);
    BA_LAUNCH_CHECK();

    BA_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace sqrtba
