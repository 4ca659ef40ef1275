// Check-node arithmetic shared by the BP kernels (Sec. 4.1, Eq. 2), FP32.
// For an input x (a variable->check message) the pair t = tanh(|x|/2),
// d = 1 - t = 2 e^{-|x|} / (1 + e^{-|x|}) is formed without cancellation;
// products of pairs are (tA tB, dA + tA dB), exact algebra, so P = prod t and
// D = 1 - P stay accurate even when P rounds to 1 in FP32; the output
// magnitude is 2 atanh(P) = log((1 + P) / D).
#pragma once

#include <cstdint>

namespace t3d {
namespace bpm {

struct TD {
    float t;  // tanh(|x|/2)
    float d;  // 1 - tanh(|x|/2)
};

__device__ __forceinline__ TD td_mul(TD A, TD B) { return TD{A.t * B.t, fmaf(A.t, B.d, A.d)}; }

// MUFU approximations (PTX ex2/rcp/lg2 .approx.ftz, a few ulp); the
// formulations below only feed them arguments where that relative accuracy
// carries through without cancellation.
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// (tanh(|x|/2), 1 - tanh(|x|/2)) = ((1 - E), 2E) / (1 + E) with E = e^{-|x|}.
// For |x| < 0.1 the difference 1 - E is taken from its Taylor series
// |x| - |x|^2/2 + |x|^3/6 - |x|^4/24 (truncation < 1e-6 relative) instead of
// subtracting two nearly equal numbers; above 0.1 the subtraction loses at
// most a factor E/(1-E) < 10 on E's few-ulp error.  Both forms are evaluated
// and one selected.
__device__ __forceinline__ TD td_of(float x)
{
    const float a = fabsf(x);
    const float E = ex2_approx(-a * kLog2e);
    const float r = rcp_approx(1.0f + E);
    float h = fmaf(a, -1.0f / 24.0f, 1.0f / 6.0f);
    h = fmaf(a, h, -0.5f);
    h = fmaf(a, h, 1.0f);
    const float om = (a < 0.1f) ? a * h : 1.0f - E;
    return TD{om * r, (E + E) * r};
}

// 2 atanh(P) for P = prod t, D = 1 - P: for P < 0.05 the odd series
// 2P (1 + P^2/3 + P^4/5) (truncation < 3e-10 relative); above it
// log((1 + P) / D), whose argument exceeds 1.1 so the approximate logarithm's
// absolute error stays below 2e-6 of the result.  D = 0 (underflow) gives +inf,
// which the clamp turns into 30.
__device__ __forceinline__ float two_atanh(float P, float D)
{
    const float u = P * P;
    const float series = 2.0f * P * fmaf(u, fmaf(u, 1.0f / 5.0f, 1.0f / 3.0f), 1.0f);
    const float logv = kLn2 * lg2_approx((1.0f + P) * rcp_approx(D));
    return (P < 0.05f) ? series : logv;
}

}  // namespace bpm
}  // namespace t3d
