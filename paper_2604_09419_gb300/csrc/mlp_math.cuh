// The warm-start MLP's activation: GELU(a) = a Phi(a) with the exact normal
// CDF Phi(a) = (1 + erf(a / sqrt 2)) / 2 (Hendrycks and Gimpel, 2016), and
// its derivative Phi(a) + a phi(a).  gelu() and gelu_grad() use the CUDA
// erff and serve the FP32-activation path; gelu_bf16out2() and
// gelu_grad_fast2() serve the tensor-core products of the BF16-activation
// path (its forward activations are rounded to BF16).
#pragma once

namespace line {

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float a) {
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

// GELU through erf by Abramowitz and Stegun, Handbook of Mathematical
// Functions, formula 7.1.26 (Hastings' approximation):
//   erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),
//   t = 1 / (1 + p x), x >= 0, erf(-x) = -erf(x),
// with |error| <= 1.5e-7, plus the FP32 rounding of its evaluation here (a
// hardware reciprocal and base-2 exponential).  For activations that are then
// rounded to BF16 (relative spacing 2^-8) this matches gelu() at far fewer
// instructions.  Two values at a time: the multiplies and fused multiply-adds
// are the packed FP32 pairs of sm_100 and later (each half rounded as the
// scalar instruction would be), the reciprocal and the exponential one value
// at a time.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// The shared part of GELU and GELU': x = |a| / sqrt 2, the polynomial times
// t, and exp(-x^2) = exp(-a^2 / 2).
__device__ __forceinline__ void erf_parts(float2 a, float2& poly, float2& e) {
    const float2 x = __fmul2_rn(make_float2(fabsf(a.x), fabsf(a.y)), f2(0.70710678118654752f));
    const float2 d = __ffma2_rn(f2(0.3275911f), x, f2(1.0f));
    float2 t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.x) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.y) : "f"(d.y));
    poly = __ffma2_rn(t, f2(1.061405429f), f2(-1.453152027f));
    poly = __ffma2_rn(t, poly, f2(1.421413741f));
    poly = __ffma2_rn(t, poly, f2(-0.284496736f));
    poly = __ffma2_rn(t, poly, f2(0.254829592f));
    poly = __fmul2_rn(poly, t);
    const float2 arg = __fmul2_rn(__fmul2_rn(make_float2(-x.x, -x.y), x), f2(1.4426950408889634f));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(arg.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(arg.y));
}

// erf(a / sqrt 2) from the parts: 1 - poly e with the sign of a.
__device__ __forceinline__ float2 erf_of(float2 a, float2 poly, float2 e) {
    const float2 m = __ffma2_rn(make_float2(-poly.x, -poly.y), e, f2(1.0f));
    return make_float2(copysignf(m.x, a.x), copysignf(m.y, a.y));
}

// GELU(a) = h (1 + erf), h = a / 2.
__device__ __forceinline__ float2 gelu_bf16out2(float2 a) {
    float2 poly, e;
    erf_parts(a, poly, e);
    const float2 h = __fmul2_rn(f2(0.5f), a);
    return __ffma2_rn(h, erf_of(a, poly, e), h);
}

// GELU'(a) = Phi(a) + a phi(a) by the same formula: its exp(-x^2) is
// exp(-a^2/2), so phi(a) = exp(-a^2/2)/sqrt(2 pi) comes at no extra cost:
// (a e) / sqrt(2 pi) + (erf + 1) / 2.  For the backward products that feed
// BF16-activation training.
__device__ __forceinline__ float2 gelu_grad_fast2(float2 a) {
    float2 poly, e;
    erf_parts(a, poly, e);
    const float2 phi_half = __ffma2_rn(f2(0.5f), erf_of(a, poly, e), f2(0.5f));
    return __ffma2_rn(__fmul2_rn(a, e), f2(0.39894228040143268f), phi_half);
}

}  // namespace line
