// The warm-start MLP's activation: GELU(a) = a Phi(a) with the exact normal
// CDF Phi(a) = (1 + erf(a / sqrt 2)) / 2 (Hendrycks and Gimpel, 2016), and
// its derivative Phi(a) + a phi(a).  gelu() and gelu_grad() use the CUDA
// erff and serve the FP32-activation path; gelu_bf16out() and
// gelu_grad_fast() serve the tensor-core products of the BF16-activation
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
// instructions.
__device__ __forceinline__ float gelu_bf16out(float a) {
    const float x = fabsf(a) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-x * x * 1.4426950408889634f));
    const float erf_abs = fmaf(-poly, e, 1.0f);
    const float erf = copysignf(erf_abs, a);
    const float h = 0.5f * a;
    return fmaf(h, erf, h);
}

// GELU'(a) = Phi(a) + a phi(a) by the same formula: its exp(-x^2), x =
// |a|/sqrt 2, is exp(-a^2/2), so phi(a) = exp(-a^2/2)/sqrt(2 pi) comes at no
// extra cost.  For the backward products that feed BF16-activation training.
__device__ __forceinline__ float gelu_grad_fast(float a) {
    const float x = fabsf(a) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-x * x * 1.4426950408889634f));
    const float erf = copysignf(fmaf(-poly, e, 1.0f), a);
    return fmaf(0.5f, erf, 0.5f) + a * e * 0.39894228040143268f;
}

}  // namespace line
