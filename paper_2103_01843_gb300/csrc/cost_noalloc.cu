// Allocation-free variant of the energy evaluation (K7) for callers that
// cannot allocate device memory: code on a latency-critical path where
// cudaMalloc/cudaFree would synchronise the device, and hosts whose device
// memory is entirely owned by another allocator (a framework caching
// allocator, a fixed arena).
//
// The per-block FP64 partial sums live in one file-scope __device__ array of
// NA_MAX_BLOCKS doubles (128 KiB), which every GPU that loads the library
// holds until the process exits.  Each call writes only the partials it
// reads back, so nothing needs clearing between calls; calls that overlap on
// the GPU (different streams, or other threads) share the array and race.
#include <mutex>

#include "camera.cuh"
#include "common.cuh"

namespace sqrtba {
void set_create_error(const std::string& m);

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_OBS_PER_BLOCK = 1024;
constexpr int NA_MAX_BLOCKS = 16384;  // 128 KiB of partial sums
constexpr int64_t NA_MAX_OBS = (int64_t)NA_MAX_BLOCKS * NA_OBS_PER_BLOCK;
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

std::mutex g_setup_mu;
double* g_partials_ptr[NA_MAX_DEVICES] = {};

// Block b sums ||r||^2 over observations [b * 1024, (b + 1) * 1024) in the
// caller's order.  An index out of range makes the cost NaN (no access).
__global__ void __launch_bounds__(NA_THREADS)
k_cost_partials_noalloc(int64_t n_obs, int n_cam, int n_pt, const float* __restrict__ cams,
                        const float* __restrict__ pts, const int32_t* __restrict__ obs_cam,
                        const int32_t* __restrict__ obs_pt, const float* __restrict__ obs_xy,
                        double* __restrict__ partials) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t base = (int64_t)blockIdx.x * NA_OBS_PER_BLOCK;
    for (int i = threadIdx.x; i < NA_OBS_PER_BLOCK; i += NA_THREADS) {
        const int64_t o = base + i;
        if (o >= n_obs) break;
        const int c = obs_cam[o], j = obs_pt[o];
        if (c < 0 || c >= n_cam || j < 0 || j >= n_pt) {
            acc += __longlong_as_double(0x7ff8000000000000ll);  // NaN
            continue;
        }
        float r0, r1;
        project_residual(cams + 9 * (int64_t)c, pts[3 * (int64_t)j], pts[3 * (int64_t)j + 1],
                         pts[3 * (int64_t)j + 2], obs_xy[2 * o], obs_xy[2 * o + 1], r0, r1);
        acc += (double)r0 * (double)r0 + (double)r1 * (double)r1;
    }
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(1024)
k_sum_partials_noalloc(const double* __restrict__ partials, int n, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace
}  // namespace sqrtba

using namespace sqrtba;

extern "C" ba_status ba_eval_cost_noalloc(const float* d_cams, int32_t n_cam, const float* d_pts, int32_t n_pt,
                                          const int32_t* d_obs_cam, const int32_t* d_obs_pt,
                                          const float* d_obs_xy, int64_t n_obs, double* d_cost,
                                          void* cuda_stream) {
    if (!d_cams || !d_pts || !d_obs_cam || !d_obs_pt || !d_obs_xy || !d_cost || n_cam < 1 || n_pt < 1 ||
        n_obs < 1) {
        set_create_error("ba_eval_cost_noalloc: null pointer or empty problem");
        return BA_ERR_INVALID_ARG;
    }
    if (n_obs > NA_MAX_OBS) {
        set_create_error("ba_eval_cost_noalloc: n_obs exceeds 16777216, the limit of its fixed 128 KiB "
                         "device scratch (16384 partial sums of 1024 observations each)");
        return BA_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        set_create_error(std::string("ba_eval_cost_noalloc: no usable current device: ") + cudaGetErrorString(e));
        return BA_ERR_CUDA;
    }
    if (cuda_stream) {
        // the launches below go to the current device: the stream must be one of its streams
        int sdev = -1;
        e = cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev);
        if (e != cudaSuccess || sdev != dev) {
            set_create_error(e != cudaSuccess
                                 ? std::string("ba_eval_cost_noalloc: invalid stream: ") + cudaGetErrorString(e)
                                 : std::string("ba_eval_cost_noalloc: the stream belongs to another device than "
                                               "the current one"));
            return BA_ERR_INVALID_ARG;
        }
    }
    double* partials = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_partials_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
            if (e != cudaSuccess || !ptr) {
                set_create_error(std::string("ba_eval_cost_noalloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
                return BA_ERR_CUDA;
            }
            g_partials_ptr[dev] = static_cast<double*>(ptr);
        }
        partials = g_partials_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (int)((n_obs + NA_OBS_PER_BLOCK - 1) / NA_OBS_PER_BLOCK);
    k_cost_partials_noalloc<<<nb, NA_THREADS, 0, st>>>(n_obs, n_cam, n_pt, d_cams, d_pts, d_obs_cam, d_obs_pt,
                                                      d_obs_xy, partials);
    k_sum_partials_noalloc<<<1, 1024, 0, st>>>(partials, nb, d_cost);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_create_error(std::string("ba_eval_cost_noalloc: launch failed: ") + cudaGetErrorString(e));
        return BA_ERR_CUDA;
    }
    return BA_OK;
}
