// Check-node arithmetic shared by the BP kernels (Sec. 4.1, Eq. 2), FP32.
// For an input x (a variable->check message) the pair t = tanh(|x|/2),
// d = 1 - t = 2 e^{-|x|} / (1 + e^{-|x|}) is formed without cancellation;
// products of pairs are (tA tB, dA + tA dB), exact algebra, so P = prod t and
// D = 1 - P stay accurate even when P rounds to 1 in FP32; the output
// magnitude is 2 atanh(P) = log((1 + P) / D).  Also the flooding check node
// over a fixed number of inputs built from those pairs, and the four-samples-
// per-thread row accessors of the sample-innermost message layouts.
#pragma once

#include <cuda_runtime.h>

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


// Flooding check node over K inputs (Eq. 2): out[i] = (-1)^{syn} times the
// product of the other inputs' signs times 2 atanh(prod_{j != i} tanh(|x_j|/2)),
// from prefix and suffix products of the (t, d) pairs, clamped to |M| <= 30.
constexpr float kCheckClamp = 30.0f;

template <int K>
__device__ __forceinline__ void check_node(const float (&x)[K], bool syn, float (&out)[K])
{
    TD v[K], pre[K], suf[K];
    uint32_t sgn_all = syn ? 0x80000000u : 0u;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        v[i] = td_of(x[i]);
        sgn_all ^= __float_as_uint(x[i]);
    }
    pre[0] = TD{1.0f, 0.0f};
#pragma unroll
    for (int i = 1; i < K; ++i) pre[i] = td_mul(pre[i - 1], v[i - 1]);
    suf[K - 1] = TD{1.0f, 0.0f};
#pragma unroll
    for (int i = K - 2; i >= 0; --i) suf[i] = td_mul(v[i + 1], suf[i + 1]);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const TD o = td_mul(pre[i], suf[i]);
        const float mag = fminf(two_atanh(o.t, o.d), kCheckClamp);
        const uint32_t sgn = (sgn_all ^ __float_as_uint(x[i])) & 0x80000000u;
        out[i] = __uint_as_float(__float_as_uint(mag) | sgn);
    }
}

// Sample-innermost message rows (samples of a chunk padded to 64): a thread
// takes four consecutive samples of one row with 16-byte loads and stores.
__device__ __forceinline__ float4 ld4(const float* base, int64_t row, int64_t S, int64_t smp)
{
    return __ldg(reinterpret_cast<const float4*>(base + row * S + smp));
}

__device__ __forceinline__ void st4(float* base, int64_t row, int64_t S, int64_t smp, float4 v)
{
    *reinterpret_cast<float4*>(base + row * S + smp) = v;
}

__device__ __forceinline__ float comp(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }

}  // namespace bpm
}  // namespace t3d
