// Shared device/host helpers of the sqrtba CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sqrtba.h"

#define BA_WARP 32

namespace sqrtba {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
struct Error {
    ba_status code;
    std::string msg;
};

#define BA_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            if (e_ == cudaErrorMemoryAllocation) {                                 \
                cudaGetLastError();                                                \
                throw ::sqrtba::Error{BA_ERR_OOM, std::string(#expr) + ": " +      \
                                                      cudaGetErrorString(e_)};     \
            }                                                                      \
            throw ::sqrtba::Error{BA_ERR_CUDA,                                     \
                                  std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
        }                                                                          \
    } while (0)

#define BA_LAUNCH_CHECK() BA_CUDA_TRY(cudaGetLastError())

// error bits written by kernels into a device word
enum : uint32_t {
    ERRBIT_INDEX = 1u << 0,      // observation index out of range
    ERRBIT_NONFINITE = 1u << 1,  // non-finite input value
    ERRBIT_FEWOBS = 1u << 2,     // landmark with < 2 observations
    ERRBIT_DUPLICATE = 1u << 3,  // duplicate (landmark, camera) pair
    ERRBIT_PRECOND = 1u << 4,    // a preconditioner block was not positive definite
    ERRBIT_TIMEOUT = 1u << 5,    // a bounded device-side wait gave up
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum, result broadcast to every thread.  scratch: >= 32 floats.
// Must be called by all threads of the block.
__device__ __forceinline__ float block_sum(float v, float* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    float t = lane < nw ? scratch[lane] : 0.0f;
    t = warp_sum(t);
    return t;
}

__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = lane < nw ? scratch[lane] : 0.0;
    t = warp_sum_d(t);
    return t;
}

__host__ __device__ __forceinline__ int64_t pad4(int64_t n) { return (n + 3) & ~int64_t(3); }

// Givens rotation m (0..5) of the landmark damping (Sec. 5.3) acts on R1 row c
// and damping row d: (d, c) = (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
__host__ __device__ __forceinline__ void givens_pair(int m, int& c, int& d) {
    c = m < 3 ? m : (m < 5 ? m - 2 : 2);
    d = m < 3 ? 0 : (m < 5 ? 1 : 2);
}

// Float offset of landmark j's top block (3 rows x (9k + 4)).
__host__ __device__ __forceinline__ int64_t top_offset(int64_t obs_off_j, int64_t j) {
    return 3 * (9 * obs_off_j + 4 * j);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace sqrtba
