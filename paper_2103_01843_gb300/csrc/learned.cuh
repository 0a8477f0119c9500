// The learned warm start and block-preconditioner correction (K8 inference,
// K9 training): a per-camera MLP 19 -> 256 -> 256 -> 256 -> 54 with GELU,
// BF16 weights and activations on the tensor cores (tcgen05, FP32
// accumulation in tensor memory), FP32 master weights, backward and Adam.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace sqrtba {

struct Problem;

constexpr int ML_IN = 19, ML_H = 256, ML_OUT = 54;
constexpr int ML_ROWS = 128;   // rows of one tensor-core tile (the MMA's M)
constexpr int ML_AUX = 72;     // per-sample head inputs: L (45, lower, row by row), w, s, z* (9 each)
// flat parameter vector: W0 (256 x 19), b0, W1 (256 x 256), b1, W2, b2, W3 (54 x 256), b3
constexpr int64_t ML_P = 256LL * 19 + 256 + 2 * (256LL * 256 + 256) + 54LL * 256 + 54;

struct Mlp {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float* master = nullptr;   // ML_P FP32 master parameters
    float* grad = nullptr;     // ML_P
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t adam_t = 0;
    uint8_t* wimg = nullptr;   // BF16 operand images of W0..W3 (tensor-core layout)
    // per-call buffers, grown on demand (rows padded to ML_ROWS)
    int cap = 0;
    uint8_t* ximg = nullptr;   // feature tiles, BF16 operand images
    float* xf = nullptr;       // [cap][19] features (FP32)
    float* z = nullptr;        // [3][cap][256] hidden pre-activations
    float* y = nullptr;        // [cap][64] outputs
    float* dy = nullptr;       // [cap][64]
    float* dza = nullptr;      // [cap][256]
    float* dzb = nullptr;      // [cap][256]
    double* loss = nullptr;    // device accumulator
    double* loss_host = nullptr;
    uint32_t* err = nullptr;
    std::vector<void*> allocations;
    std::string last_error;
};

void mlp_init(Mlp& m, const float* host_params, cudaStream_t stream);
void mlp_free(Mlp& m);
void mlp_reserve(Mlp& m, int n);
// features (n x 19 FP32, device) -> outputs (n x 54 FP32, device)
void mlp_forward(Mlp& m, const float* feats, int n, float* out);
// mean loss over n samples and (optionally) its gradient in m.grad
double mlp_loss_grad(Mlp& m, const float* feats, const float* aux, int n);
void mlp_adam(Mlp& m, float lr, float beta1, float beta2, float eps);
// per-sample features and head inputs from (M_i, g_i, x*_i, count_i)
void mlp_prepare(cudaStream_t st, const float* M, const float* g, const float* xstar, const int32_t* count, int n,
                 float* feats, float* aux);
// in the solver: features of every camera, MLP, warm start into p.x and the
// corrected blocks into p.minv_l
void learned_apply(Problem& p, Mlp& m);

}  // namespace sqrtba
