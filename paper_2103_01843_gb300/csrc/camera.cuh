// FP32 BAL camera model on the device (Sec. 6.2: Snavely model with one
// focal length and two radial distortion parameters).
//
//   P = R(w) X + t,   p = -P_xy / P_z,   pixel = f (1 + k1 |p|^2 + k2 |p|^4) p
//   residual = pixel - z
//
// Pose Jacobian columns: (dw, t, f, k1, k2) with the rotation increment taken
// from the left, R <- Exp(dw) R, hence dP/d(dw) = -[R X]_x.
#pragma once

#include <cuda_runtime.h>

namespace sqrtba {

// R = cos(th) I + (sin(th)/th) [w]_x + ((1 - cos th)/th^2) w w^T, row-major.
// 1 - cos(th) is evaluated as 2 sin^2(th/2) to keep FP32 accuracy at small th.
__device__ __forceinline__ void rotation_matrix(const float w0, const float w1, const float w2,
                                                float R[9]) {
    const float th2 = w0 * w0 + w1 * w1 + w2 * w2;
    float a, b, c;
    if (th2 < 1e-8f) {
        a = 1.0f - th2 * (1.0f / 6.0f);
        b = 0.5f - th2 * (1.0f / 24.0f);
        c = 1.0f - 0.5f * th2;
    } else {
        const float th = sqrtf(th2);
        float s, co;
        sincosf(th, &s, &co);
        const float sh = sinf(0.5f * th);
        a = s / th;
        b = 2.0f * sh * sh / th2;
        c = co;
    }
    R[0] = c + b * w0 * w0;
    R[1] = -a * w2 + b * w0 * w1;
    R[2] = a * w1 + b * w0 * w2;
    R[3] = a * w2 + b * w1 * w0;
    R[4] = c + b * w1 * w1;
    R[5] = -a * w0 + b * w1 * w2;
    R[6] = -a * w1 + b * w2 * w0;
    R[7] = a * w0 + b * w2 * w1;
    R[8] = c + b * w2 * w2;
}

// Residual only.
__device__ __forceinline__ void project_residual(const float* __restrict__ cam, float X0, float X1,
                                                 float X2, float z0, float z1, float& r0,
                                                 float& r1) {
    float R[9];
    rotation_matrix(cam[0], cam[1], cam[2], R);
    const float P0 = R[0] * X0 + R[1] * X1 + R[2] * X2 + cam[3];
    const float P1 = R[3] * X0 + R[4] * X1 + R[5] * X2 + cam[4];
    const float P2 = R[6] * X0 + R[7] * X1 + R[8] * X2 + cam[5];
    const float iz = 1.0f / P2;
    const float p0 = -P0 * iz, p1 = -P1 * iz;
    const float r2 = p0 * p0 + p1 * p1;
    const float fd = cam[6] * (1.0f + cam[7] * r2 + cam[8] * r2 * r2);
    r0 = fd * p0 - z0;
    r1 = fd * p1 - z1;
}

// Residual r[2], pose Jacobian Jp[18] (2x9 row-major), landmark Jacobian
// Jl[6] (2x3 row-major).
__device__ __forceinline__ void project_jacobians(const float* __restrict__ cam, float X0, float X1,
                                                  float X2, float z0, float z1, float r[2],
                                                  float Jp[18], float Jl[6]) {
    float R[9];
    rotation_matrix(cam[0], cam[1], cam[2], R);
    const float Y0 = R[0] * X0 + R[1] * X1 + R[2] * X2;
    const float Y1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
    const float Y2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
    const float P0 = Y0 + cam[3], P1 = Y1 + cam[4], P2 = Y2 + cam[5];
    const float f = cam[6], k1 = cam[7], k2 = cam[8];
    const float iz = 1.0f / P2;
    const float p0 = -P0 * iz, p1 = -P1 * iz;
    const float r2 = p0 * p0 + p1 * p1;
    const float d = 1.0f + k1 * r2 + k2 * r2 * r2;
    r[0] = f * d * p0 - z0;
    r[1] = f * d * p1 - z1;

    // d pixel / d p = f (d I + g p p^T), g = 2 (k1 + 2 k2 |p|^2)
    const float g = 2.0f * (k1 + 2.0f * k2 * r2);
    const float D00 = f * (d + g * p0 * p0), D01 = f * g * p0 * p1, D11 = f * (d + g * p1 * p1);
    // d p / d P = [[-iz, 0, P0 iz^2], [0, -iz, P1 iz^2]]
    const float iz2 = iz * iz;
    float A[6];  // d pixel / d P
    A[0] = -D00 * iz;
    A[1] = -D01 * iz;
    A[2] = (D00 * P0 + D01 * P1) * iz2;
    A[3] = -D01 * iz;
    A[4] = -D11 * iz;
    A[5] = (D01 * P0 + D11 * P1) * iz2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float a0 = A[3 * i], a1 = A[3 * i + 1], a2 = A[3 * i + 2];
        // A * (-[Y]_x), -[Y]_x = [[0, Y2, -Y1], [-Y2, 0, Y0], [Y1, -Y0, 0]]
        Jp[9 * i + 0] = -a1 * Y2 + a2 * Y1;
        Jp[9 * i + 1] = a0 * Y2 - a2 * Y0;
        Jp[9 * i + 2] = -a0 * Y1 + a1 * Y0;
        Jp[9 * i + 3] = a0;
        Jp[9 * i + 4] = a1;
        Jp[9 * i + 5] = a2;
        const float pi = i == 0 ? p0 : p1;
        Jp[9 * i + 6] = d * pi;
        Jp[9 * i + 7] = f * r2 * pi;
        Jp[9 * i + 8] = f * r2 * r2 * pi;
        Jl[3 * i + 0] = a0 * R[0] + a1 * R[3] + a2 * R[6];
        Jl[3 * i + 1] = a0 * R[1] + a1 * R[4] + a2 * R[7];
        Jl[3 * i + 2] = a0 * R[2] + a1 * R[5] + a2 * R[8];
    }
}

// Robust norm (the Huber norm of Sec. 6.2, read as iteratively reweighted
// least squares): for s = ||r||^2, rho(s) = s if s <= delta^2, else
// 2 delta sqrt(s) - delta^2; the linearised rows [J | r] of an observation are
// scaled by sqrt(w), w = rho'(s) = min(1, delta / ||r||).  delta <= 0: the
// squared norm (rho(s) = s, w = 1).
__device__ __forceinline__ float huber_weight(float delta, float r0, float r1) {
    const float s = r0 * r0 + r1 * r1;
    return (delta > 0.f && s > delta * delta) ? delta * rsqrtf(s) : 1.f;
}
__device__ __forceinline__ double huber_rho(double delta, double s) {
    return (delta > 0.0 && s > delta * delta) ? 2.0 * delta * sqrt(s) - delta * delta : s;
}
// One observation's energy term rho(r0^2 + r1^2) from FP32 residuals, for an
// FP64 sum: the square in FP32 (relative error 2^-23 at most, below that of
// the FP32 residual itself), then one conversion; FP64 arithmetic only on the
// robust branch.  GB300 issues FP64 at a small fraction of its FP32 rate, and
// the squares in FP64 made the per-observation sums FP64-bound.
__device__ __forceinline__ double energy_term(float delta, float r0, float r1) {
    const float s = r0 * r0 + r1 * r1;
    return (delta > 0.f && s > delta * delta) ? huber_rho((double)delta, (double)s) : (double)s;
}
__device__ __forceinline__ void huber_scale_rows(float delta, float r[2], float Jp[18], float Jl[6]) {
    const float w = huber_weight(delta, r[0], r[1]);
    if (w == 1.f) return;
    const float sw = sqrtf(w);
#pragma unroll
    for (int i = 0; i < 2; ++i) r[i] *= sw;
#pragma unroll
    for (int i = 0; i < 18; ++i) Jp[i] *= sw;
#pragma unroll
    for (int i = 0; i < 6; ++i) Jl[i] *= sw;
}

// Camera frames: the rotation matrix evaluated once per camera and state,
// 16 floats per camera (R row-major, t, f, k1, k2, 0), 16-byte aligned, so
// that the per-observation kernels skip the trigonometry of R(w).
constexpr int FRAME = 16;

__device__ __forceinline__ void make_frame(const float* __restrict__ cam, float* __restrict__ fr) {
    float R[9];
    rotation_matrix(cam[0], cam[1], cam[2], R);
    float4* o = reinterpret_cast<float4*>(fr);
    o[0] = make_float4(R[0], R[1], R[2], R[3]);
    o[1] = make_float4(R[4], R[5], R[6], R[7]);
    o[2] = make_float4(R[8], cam[3], cam[4], cam[5]);
    o[3] = make_float4(cam[6], cam[7], cam[8], 0.f);
}

struct Frame {
    float R[9], t[3], f, k1, k2;
};

__device__ __forceinline__ Frame load_frame(const float* __restrict__ fr) {
    const float4* q = reinterpret_cast<const float4*>(fr);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    return Frame{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x}, {c.y, c.z, c.w}, d.x, d.y, d.z};
}

// Residual from a camera frame (same arithmetic as project_residual).
__device__ __forceinline__ void frame_residual(const float* __restrict__ fr, float X0, float X1, float X2, float z0,
                                               float z1, float& r0, float& r1) {
    const Frame F = load_frame(fr);
    const float P0 = F.R[0] * X0 + F.R[1] * X1 + F.R[2] * X2 + F.t[0];
    const float P1 = F.R[3] * X0 + F.R[4] * X1 + F.R[5] * X2 + F.t[1];
    const float P2 = F.R[6] * X0 + F.R[7] * X1 + F.R[8] * X2 + F.t[2];
    const float iz = 1.0f / P2;
    const float p0 = -P0 * iz, p1 = -P1 * iz;
    const float r2 = p0 * p0 + p1 * p1;
    const float fd = F.f * (1.0f + F.k1 * r2 + F.k2 * r2 * r2);
    r0 = fd * p0 - z0;
    r1 = fd * p1 - z1;
}

// Residual and Jacobians from a camera frame (same arithmetic as
// project_jacobians).
__device__ __forceinline__ void frame_jacobians(const float* __restrict__ fr, float X0, float X1, float X2, float z0,
                                                float z1, float r[2], float Jp[18], float Jl[6]) {
    const Frame F = load_frame(fr);
    const float* R = F.R;
    const float Y0 = R[0] * X0 + R[1] * X1 + R[2] * X2;
    const float Y1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
    const float Y2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
    const float P0 = Y0 + F.t[0], P1 = Y1 + F.t[1], P2 = Y2 + F.t[2];
    const float f = F.f, k1 = F.k1, k2 = F.k2;
    const float iz = 1.0f / P2;
    const float p0 = -P0 * iz, p1 = -P1 * iz;
    const float r2 = p0 * p0 + p1 * p1;
    const float d = 1.0f + k1 * r2 + k2 * r2 * r2;
    r[0] = f * d * p0 - z0;
    r[1] = f * d * p1 - z1;
    const float g = 2.0f * (k1 + 2.0f * k2 * r2);
    const float D00 = f * (d + g * p0 * p0), D01 = f * g * p0 * p1, D11 = f * (d + g * p1 * p1);
    const float iz2 = iz * iz;
    float A[6];
    A[0] = -D00 * iz;
    A[1] = -D01 * iz;
    A[2] = (D00 * P0 + D01 * P1) * iz2;
    A[3] = -D01 * iz;
    A[4] = -D11 * iz;
    A[5] = (D01 * P0 + D11 * P1) * iz2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float a0 = A[3 * i], a1 = A[3 * i + 1], a2 = A[3 * i + 2];
        Jp[9 * i + 0] = -a1 * Y2 + a2 * Y1;
        Jp[9 * i + 1] = a0 * Y2 - a2 * Y0;
        Jp[9 * i + 2] = -a0 * Y1 + a1 * Y0;
        Jp[9 * i + 3] = a0;
        Jp[9 * i + 4] = a1;
        Jp[9 * i + 5] = a2;
        const float pi = i == 0 ? p0 : p1;
        Jp[9 * i + 6] = d * pi;
        Jp[9 * i + 7] = f * r2 * pi;
        Jp[9 * i + 8] = f * r2 * r2 * pi;
        Jl[3 * i + 0] = a0 * R[0] + a1 * R[3] + a2 * R[6];
        Jl[3 * i + 1] = a0 * R[1] + a1 * R[4] + a2 * R[7];
        Jl[3 * i + 2] = a0 * R[2] + a1 * R[5] + a2 * R[8];
    }
}

// w_out = Log(Exp(dw) Exp(w)) through unit quaternions (angle kept in [0, pi]).
__device__ __forceinline__ void compose_rotation(const float dw[3], const float w[3], float out[3]) {
    float qa[4], qb[4];
    const float* src[2] = {dw, w};
    float* dst[2] = {qa, qb};
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float* v = src[m];
        const float th = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        float s, c;
        sincosf(0.5f * th, &s, &c);
        const float sc = th < 1e-4f ? 0.5f - th * th * (1.0f / 48.0f) : s / th;
        dst[m][0] = c;
        dst[m][1] = sc * v[0];
        dst[m][2] = sc * v[1];
        dst[m][3] = sc * v[2];
    }
    float q0 = qa[0] * qb[0] - qa[1] * qb[1] - qa[2] * qb[2] - qa[3] * qb[3];
    float q1 = qa[0] * qb[1] + qa[1] * qb[0] + qa[2] * qb[3] - qa[3] * qb[2];
    float q2 = qa[0] * qb[2] - qa[1] * qb[3] + qa[2] * qb[0] + qa[3] * qb[1];
    float q3 = qa[0] * qb[3] + qa[1] * qb[2] - qa[2] * qb[1] + qa[3] * qb[0];
    const float n = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    q0 *= n; q1 *= n; q2 *= n; q3 *= n;
    if (q0 < 0.0f) { q0 = -q0; q1 = -q1; q2 = -q2; q3 = -q3; }
    const float vn = sqrtf(q1 * q1 + q2 * q2 + q3 * q3);
    const float fct = vn < 1e-7f ? 2.0f / q0 : 2.0f * atan2f(vn, q0) / vn;
    out[0] = fct * q1;
    out[1] = fct * q2;
    out[2] = fct * q3;
}

}  // namespace sqrtba
