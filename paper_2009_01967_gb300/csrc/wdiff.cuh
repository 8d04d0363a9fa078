// Compensated FP32 arithmetic for the energy and occupation differences of
// the delta epilogues (paper Eq. phase_space: w +- w' - w'' and n' - n'').
//
// A frequency or an occupation number is carried as an unevaluated pair
// hi + lo of FP32 values (hi = fl(x), lo = fl(x - hi), x the FP64 value), so
// that a difference of nearly equal quantities -- the energy mismatch inside
// the delta window, or n' - n'' when w is small -- is formed from the pair
// parts and keeps a relative error of a few FP32 ulps of the difference
// itself, instead of an absolute error of an ulp of the largest frequency.
// The sum w + w' of two pairs uses Knuth's two-sum (exact for the hi parts).
#pragma once

#include <cmath>

#include "kald_internal.h"

namespace kald {

struct F2 {
    float h, l;
};

__host__ __device__ __forceinline__ F2 f2_of(double x) {
    F2 r;
    r.h = (float)x;
    r.l = (float)(x - (double)r.h);
    return r;
}

// a + b as a pair: two-sum of the hi parts (exact), lo parts added to the error.
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float v = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
    F2 r;
    r.h = s;
    r.l = e + (a.l + b.l);
    return r;
}

__device__ __forceinline__ F2 f2_neg(F2 a) {
    F2 r;
    r.h = -a.h;
    r.l = -a.l;
    return r;
}

// (a - b) rounded to FP32: hi parts first (exact when a and b are within a
// factor of two of each other), then the lo parts.
__device__ __forceinline__ float f2_diff(F2 a, F2 b) {
    return __fadd_rn(__fsub_rn(a.h, b.h), __fsub_rn(a.l, b.l));
}

// Energy-delta shapes of the epilogues, without their normalisation (applied
// per mode at the end, delta_norm): 0 Gaussian exp(-a d^2), a = 1/(2 sigma^2);
// 1 Lorentzian 1/(1 + a d^2), a = 1/sigma^2; 2 triangle max(0, 1 - a |d|),
// a = 1/sigma.  The shape is uniform over a launch (no divergence).
enum : int { kDeltaGauss = 0, kDeltaLorentz = 1, kDeltaTriangle = 2 };
__device__ __forceinline__ float delta_shape(float d, int shape, float a) {
    if (shape == kDeltaGauss) return __expf(-d * d * a);
    if (shape == kDeltaLorentz) return 1.0f / fmaf(d * d, a, 1.0f);
    return fmaxf(0.0f, 1.0f - fabsf(d) * a);
}
// The same on a pair of values (packed FP32x2 arithmetic; per component the
// operations and their rounding are those of delta_shape).
__device__ __forceinline__ float2 delta_shape2(float2 d, int shape, float a) {
    const float2 d2 = __fmul2_rn(d, d);
    if (shape == kDeltaGauss) {
        const float2 x = __fmul2_rn(d2, make_float2(-a, -a));
        return make_float2(__expf(x.x), __expf(x.y));
    }
    if (shape == kDeltaLorentz) {
        const float2 x = __ffma2_rn(d2, make_float2(a, a), make_float2(1.0f, 1.0f));
        return make_float2(1.0f / x.x, 1.0f / x.y);
    }
    return make_float2(fmaxf(0.0f, 1.0f - fabsf(d.x) * a), fmaxf(0.0f, 1.0f - fabsf(d.y) * a));
}
__device__ __forceinline__ double delta_shape(double d, int shape, double a) {
    if (shape == kDeltaGauss) return exp(-d * d * a);
    if (shape == kDeltaLorentz) return 1.0 / fma(d * d, a, 1.0);
    return fmax(0.0, 1.0 - fabs(d) * a);
}
// Host side: the parameter a of a shape and width sigma (rad/ps), and the
// normalisation that makes the shape a density in angular frequency.
__host__ __device__ inline double delta_param(int shape, double sigma) {
    return shape == kDeltaGauss ? 0.5 / (sigma * sigma) : shape == kDeltaLorentz ? 1.0 / (sigma * sigma) : 1.0 / sigma;
}
inline double delta_norm(int shape, double sigma) {
    return shape == kDeltaGauss ? 1.0 / (std::sqrt(kTwoPi) * sigma)       // 1 / (sqrt(2 pi) sigma)
           : shape == kDeltaLorentz ? 1.0 / (kPi * sigma)
                                    : 1.0 / sigma;
}

}  // namespace kald
