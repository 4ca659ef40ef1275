// Learned local pre-decoder (not in the paper): a periodic 3-D convolutional
// network that maps the last two measured syndromes of every site to flip
// probabilities of the site's three edges, trained on pairs the simulator
// generates.  It stands in for BP ahead of the flip / p-flip schedule.
//
// Network: conv 3x3x3 (6 -> 16) + ReLU, conv 3x3x3 (16 -> 16) + ReLU,
// conv 3x3x3 (16 -> 16) + ReLU, 1x1x1 head (16 -> 3), sigmoid; 16,515
// parameters.  Input channels of site r: s_{t-1}(n, r) and s_t(n, r) for the
// three face normals n, as 0/1.  Output d of site r: the edge (d, r).
//
// Layout: activations are BF16 [site][sample][16] (32 bytes per site and
// sample), so a 3x3x3 convolution is 27 accumulated GEMMs of
// (samples x 16 input channels) . (16 x 16 output channels): one warp computes
// 32 samples x 16 channels of one site with mma.sync m16n8k16 (BF16 inputs,
// FP32 accumulation), reading the neighbour site's 32 x 16 input tile directly
// as A fragments and the offset's 16 x 16 weights from shared memory.
// Hidden activations are rounded to BF16 between layers; the head reads the
// third layer's output in FP32.
//
// Training: forward with the labels fused into the third layer's epilogue
// (BCE gradient, head gradient, ReLU mask), backward data by the same
// tensor-core convolution with flipped and transposed weights, weight and
// bias gradients by a CUDA-core reduction, Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "t3d_cnn.cuh"
#include "t3d_device.cuh"
#include "t3d_host.hpp"

namespace t3d {
namespace cnn {

constexpr int kThreads = 256;   // 8 warps
constexpr int kTile = 32;       // samples per warp tile

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t u)
{
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(v);
}

// D (16x8, f32) += A (16x16, bf16, row) * B (16x8, bf16, col).
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Neighbour site r + (dx, dy, dz) with periodic wrap.
__device__ __forceinline__ int neighbour(const Lattice& lat, const Coord& rc, int k)
{
    const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
    int x = rc.x[0] + dx, y = rc.x[1] + dy, z = rc.x[2] + dz;
    x = x < 0 ? x + lat.L : (x >= lat.L ? x - lat.L : x);
    y = y < 0 ? y + lat.L : (y >= lat.L ? y - lat.L : y);
    z = z < 0 ? z + lat.L : (z >= lat.L ? z - lat.L : z);
    return (z * lat.L + y) * lat.L + x;
}

enum InMode { kInBits = 0, kInAct = 1 };
enum OutMode { kOutRelu = 0, kOutMask = 1, kOutHeadDecide = 2, kOutHeadTrain = 3 };

struct ConvArgs {
    Lattice lat;
    int64_t Sp;                    // padded samples of the activation buffers (multiple of 32)
    int64_t n_samples;             // valid samples
    int64_t W;                     // words per bit-sliced row
    const uint64_t* s_prev;        // kInBits
    const uint64_t* s_cur;
    const uint32_t* x;             // kInAct: BF16 pairs [site][Sp][8]
    const __nv_bfloat16* w;        // [27][co][ci]
    const float* bias;             // [16] (relu / head modes)
    const float* w4;               // [3][16] head
    const float* b4;               // [3]
    uint32_t* y;                   // BF16 output [site][Sp][8] (relu / mask / head-train dPre)
    const uint32_t* mask;          // kOutMask: forward activation whose sign gates the gradient
    uint32_t* e32;                 // head decide: error words as 32-bit halves
    uint32_t* dec32;               // head decide: decision words, [word][site][8] 32-bit halves
    float* logits;                 // optional [3][L^3][n_samples]
    const uint64_t* label;         // head train: bit-sliced e_t
    float inv_n;                   // head train: 1 / (3 L^3 n_samples)
    float* grad_w4;                // head train: [3][16] accumulated
    float* grad_b4;                // [3]
    float* loss;                   // [1]
};

template <int kIn, int kOut>
__global__ void __launch_bounds__(kThreads)
k_conv(const ConvArgs a)
{
    __shared__ __align__(16) __nv_bfloat16 sw[kOff][kC][kC];
    __shared__ float sred[kThreads / 32][3 * kC + 3 + 1];
    for (int i = threadIdx.x; i < kOff * kC * kC / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(&sw[0][0][0])[i] = reinterpret_cast<const uint32_t*>(a.w)[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int r = blockIdx.x * (kThreads / 32) + warp;
    const int64_t m0 = (int64_t)blockIdx.y * kTile;
    const bool active = r < a.lat.L3;
    float acc[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.0f;
    if (active) {
        const Coord rc = site_coord(a.lat, r);
        for (int k = 0; k < kOff; ++k) {
            const int rn = neighbour(a.lat, rc, k);
            uint32_t A[2][4];
            if (kIn == kInAct) {
                const uint32_t* base = a.x + ((int64_t)rn * a.Sp + m0) * (kC / 2);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const uint32_t* row0 = base + (mt * 16 + g) * (kC / 2);
                    const uint32_t* row8 = row0 + 8 * (kC / 2);
                    A[mt][0] = row0[t];
                    A[mt][1] = row8[t];
                    A[mt][2] = row0[t + 4];
                    A[mt][3] = row8[t + 4];
                }
            } else {
                // channel c < 3: s_{t-1}(n = c); 3 <= c < 6: s_t(n = c - 3); others zero
                const int64_t wd = m0 / 64;
                const int sh = (int)(m0 % 64);
                uint64_t wp[3], wc[3];
#pragma unroll
                for (int n = 0; n < 3; ++n) {
                    wp[n] = a.s_prev[((int64_t)n * a.lat.L3 + rn) * a.W + wd] >> sh;
                    wc[n] = a.s_cur[((int64_t)n * a.lat.L3 + rn) * a.W + wd] >> sh;
                }
                auto bitv = [&](int c, int row) -> float {
                    uint64_t w = c < 3 ? wp[c] : wc[c - 3];
                    return ((w >> row) & 1ULL) ? 1.0f : 0.0f;
                };
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int ra = mt * 16 + g, rb = ra + 8;
                    const int c0 = 2 * t, c1 = 2 * t + 1;
                    A[mt][0] = c0 < kInC ? pack_bf16(bitv(c0, ra), c1 < kInC ? bitv(c1, ra) : 0.0f) : 0u;
                    A[mt][1] = c0 < kInC ? pack_bf16(bitv(c0, rb), c1 < kInC ? bitv(c1, rb) : 0.0f) : 0u;
                    A[mt][2] = 0u;  // channels 8..15
                    A[mt][3] = 0u;
                }
            }
            uint32_t B[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const uint32_t* wrow = reinterpret_cast<const uint32_t*>(&sw[k][nt * 8 + g][0]);
                B[nt][0] = wrow[t];
                B[nt][1] = wrow[t + 4];
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma_bf16(acc[mt][nt], A[mt], B[nt]);
        }
    }
    // this thread holds rows {mt*16 + g, mt*16 + g + 8} x channels {nt*8 + 2t, nt*8 + 2t + 1}
    if (kOut == kOutRelu || kOut == kOutMask) {
        if (!active) return;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int64_t row = m0 + mt * 16 + g + 8 * half;
                uint32_t* out = a.y + ((int64_t)r * a.Sp + row) * (kC / 2);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const int c = nt * 8 + 2 * t;
                    float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
                    if (kOut == kOutRelu) {
                        v0 = fmaxf(v0 + a.bias[c], 0.0f);
                        v1 = fmaxf(v1 + a.bias[c + 1], 0.0f);
                    } else {
                        const float2 m = unpack_bf16(a.mask[((int64_t)r * a.Sp + row) * (kC / 2) + c / 2]);
                        v0 = m.x > 0.0f ? v0 : 0.0f;
                        v1 = m.y > 0.0f ? v1 : 0.0f;
                    }
                    out[c / 2] = pack_bf16(v0, v1);
                }
            }
        return;
    }
    // head: y3 = relu(acc + b3) in FP32; z_d = sum_c y3_c w4[d][c] + b4[d]
    float y3[2][2][2][2];  // [mt][half][nt][j]
    float z[2][2][3];      // [mt][half][d]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
            for (int d = 0; d < 3; ++d) z[mt][half][d] = 0.0f;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int c = nt * 8 + 2 * t + j;
                    const float v = fmaxf(acc[mt][nt][2 * half + j] + a.bias[c], 0.0f);
                    y3[mt][half][nt][j] = v;
#pragma unroll
                    for (int d = 0; d < 3; ++d) z[mt][half][d] += v * a.w4[d * kC + c];
                }
        }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float v = z[mt][half][d];
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                z[mt][half][d] = v + a.b4[d];
            }
    // the logit of sample row l (= mt*16 + half*8 + g) into lane l
    float zl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float cand[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) cand[q] = __shfl_sync(0xffffffffu, z[q >> 1][q & 1][d], 4 * (lane & 7));
        const int q = lane >> 3;
        zl[d] = q == 0 ? cand[0] : (q == 1 ? cand[1] : (q == 2 ? cand[2] : cand[3]));
    }
    const int64_t sample = m0 + lane;
    const bool valid = active && sample < a.n_samples;
    if (a.logits && valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) a.logits[((int64_t)d * a.lat.L3 + r) * a.n_samples + sample] = zl[d];
    }
    if (kOut == kOutHeadDecide) {
        const int64_t wd = m0 / 64;
        const int hw = (int)((m0 / 32) & 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const uint32_t bits = __ballot_sync(0xffffffffu, valid && zl[d] > 0.0f);
            if (active && lane == 0) {
                if (bits) a.e32[2 * (((int64_t)d * a.lat.L3 + r) * a.W + wd) + hw] ^= bits;
                a.dec32[(wd * a.lat.L3 + r) * 8 + 2 * d + hw] = bits;
            }
        }
        return;
    }
    // training: BCE gradient dz = (sigmoid(z) - y) / N, loss, head gradients, dPre3
    float dzl[3];
    float loss = 0.0f;
    {
        const int64_t wd = m0 / 64;
        const int sh = (int)(m0 % 64);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float y = 0.0f;
            if (active) y = (float)((a.label[((int64_t)d * a.lat.L3 + r) * a.W + wd] >> (sh + lane)) & 1ULL);
            const float zz = zl[d];
            const float sig = 1.0f / (1.0f + expf(-zz));
            dzl[d] = valid ? (sig - y) * a.inv_n : 0.0f;
            if (valid) loss += fmaxf(zz, 0.0f) - zz * y + log1pf(expf(-fabsf(zz)));
        }
    }
    // back to fragment rows: the dz of rows held by this lane
    float dz[2][2][3];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int d = 0; d < 3; ++d) dz[mt][half][d] = __shfl_sync(0xffffffffu, dzl[d], mt * 16 + half * 8 + g);
    float gw4[3][4], gb4[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        gb4[d] = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) gw4[d][i] = 0.0f;
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int64_t row = m0 + mt * 16 + g + 8 * half;
            uint32_t* out = a.y + ((int64_t)r * a.Sp + row) * (kC / 2);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float dv[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int c = nt * 8 + 2 * t + j;
                    float dy = 0.0f;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        dy += dz[mt][half][d] * a.w4[d * kC + c];
                        gw4[d][nt * 2 + j] += y3[mt][half][nt][j] * dz[mt][half][d];
                    }
                    dv[j] = y3[mt][half][nt][j] > 0.0f ? dy : 0.0f;
                }
                if (active) out[(nt * 8 + 2 * t) / 2] = pack_bf16(dv[0], dv[1]);
            }
        }
    // t == 0 lanes of each group hold rows' dz for bias: sum dz over the warp's 32 rows once
#pragma unroll
    for (int d = 0; d < 3; ++d) gb4[d] = dzl[d];
    // reduce over the warp: head weights over groups (lanes with equal t), bias and loss over all
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float v = gw4[d][i];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            gw4[d][i] = v;
        }
        float b = gb4[d];
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        gb4[d] = b;
    }
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane < 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int i = 0; i < 4; ++i) sred[warp][d * kC + (i >> 1) * 8 + 2 * lane + (i & 1)] = gw4[d][i];
    }
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) sred[warp][3 * kC + d] = gb4[d];
        sred[warp][3 * kC + 3] = loss;
    }
    __syncthreads();
    if (threadIdx.x < 3 * kC + 4) {
        float v = 0.0f;
        for (int wi = 0; wi < kThreads / 32; ++wi) v += sred[wi][threadIdx.x];
        if (threadIdx.x < 3 * kC) atomicAdd(&a.grad_w4[threadIdx.x], v);
        else if (threadIdx.x < 3 * kC + 3) atomicAdd(&a.grad_b4[threadIdx.x - 3 * kC], v);
        else atomicAdd(a.loss, v);
    }
}

// Input features for training (BF16 [site][Sp][16]): the six syndrome bits.
__global__ void k_features(Lattice lat, int64_t Sp, int64_t W, const uint64_t* __restrict__ s_prev,
                           const uint64_t* __restrict__ s_cur, uint32_t* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (site, sample)
    if (i >= (int64_t)lat.L3 * Sp) return;
    const int r = (int)(i / Sp);
    const int64_t s = i - (int64_t)r * Sp;
    float v[kInC];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        v[n] = (float)((s_prev[((int64_t)n * lat.L3 + r) * W + s / 64] >> (s % 64)) & 1ULL);
        v[3 + n] = (float)((s_cur[((int64_t)n * lat.L3 + r) * W + s / 64] >> (s % 64)) & 1ULL);
    }
    uint32_t* out = x + i * (kC / 2);
    out[0] = pack_bf16(v[0], v[1]);
    out[1] = pack_bf16(v[2], v[3]);
    out[2] = pack_bf16(v[4], v[5]);
#pragma unroll
    for (int c = 3; c < kC / 2; ++c) out[c] = 0u;
}

// Weight and bias gradients of one convolution layer (CUDA cores):
// gw[k][co][ci] = sum over sites r and samples s of x[r + off_k][s][ci] dpre[r][s][co],
// gb[co] = sum dpre[r][s][co].  Block (k, sample chunk of 64); thread (co, ci);
// partial sums per chunk go to part[chunk][k][co][ci] (+ bias at k = 27).
constexpr int kChunk = 64;

__global__ void __launch_bounds__(256)
k_wgrad(Lattice lat, int64_t Sp, int64_t n_samples, const uint32_t* __restrict__ x,
        const uint32_t* __restrict__ dpre, float* __restrict__ part)
{
    __shared__ float sx[kChunk][kC + 1];
    __shared__ float sd[kChunk][kC + 1];
    const int k = blockIdx.x;            // 0..26, 27 = bias
    const int64_t s0 = (int64_t)blockIdx.y * kChunk;
    const int co = threadIdx.x / kC, ci = threadIdx.x % kC;
    float acc = 0.0f;
    for (int r = 0; r < lat.L3; ++r) {
        const int rn = (k < kOff) ? neighbour(lat, site_coord(lat, r), k) : r;
        for (int i = threadIdx.x; i < kChunk * (kC / 2); i += blockDim.x) {
            const int s = i / (kC / 2), c2 = i % (kC / 2);
            const bool ok = s0 + s < n_samples;
            const float2 vx = ok ? unpack_bf16(x[((int64_t)rn * Sp + s0 + s) * (kC / 2) + c2]) : make_float2(0, 0);
            const float2 vd = ok ? unpack_bf16(dpre[((int64_t)r * Sp + s0 + s) * (kC / 2) + c2]) : make_float2(0, 0);
            sx[s][2 * c2] = vx.x;
            sx[s][2 * c2 + 1] = vx.y;
            sd[s][2 * c2] = vd.x;
            sd[s][2 * c2 + 1] = vd.y;
        }
        __syncthreads();
        if (k < kOff) {
#pragma unroll 8
            for (int s = 0; s < kChunk; ++s) acc += sx[s][ci] * sd[s][co];
        } else if (ci == 0) {
            for (int s = 0; s < kChunk; ++s) acc += sd[s][co];
        }
        __syncthreads();
    }
    part[((int64_t)blockIdx.y * (kOff + 1) + k) * kC * kC + co * kC + ci] = acc;
}

__global__ void k_wgrad_reduce(int chunks, const float* __restrict__ part, float* __restrict__ gw,
                               float* __restrict__ gb, int c_in)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // (k, co, ci) or bias
    if (i >= (kOff + 1) * kC * kC) return;
    float v = 0.0f;
    for (int c = 0; c < chunks; ++c) v += part[(int64_t)c * (kOff + 1) * kC * kC + i];
    const int k = i / (kC * kC), co = (i / kC) % kC, ci = i % kC;
    if (k < kOff) {
        if (ci < c_in) gw[(co * c_in + ci) * kOff + k] = v;   // PyTorch order [co][ci][k]
    } else if (ci == 0) {
        gb[co] = v;
    }
}

// FP32 master -> blob (forward weights, transposed-flipped weights, biases, head).
__global__ void k_prepare(const float* __restrict__ p, Blob* __restrict__ blob)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * kOff * kC * kC) {
        const int l = i / (kOff * kC * kC), k = (i / (kC * kC)) % kOff, co = (i / kC) % kC, ci = i % kC;
        const int c_in = l == 0 ? kInC : kC;
        const int base = l == 0 ? P_W1 : (l == 1 ? P_W2 : P_W3);
        const float w = ci < c_in ? p[base + (co * c_in + ci) * kOff + k] : 0.0f;
        blob->wf[l][k][co][ci] = __float2bfloat16_rn(w);
        blob->wt[l][kOff - 1 - k][ci][co] = __float2bfloat16_rn(w);
    }
    if (i < 3 * kC) {
        const int l = i / kC, c = i % kC;
        blob->bias[l][c] = p[(l == 0 ? P_B1 : (l == 1 ? P_B2 : P_B3)) + c];
        blob->w4[l][c] = p[P_W4 + l * kC + c];
    }
    if (i < 3) blob->b4[i] = p[P_B4 + i];
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters.
__global__ void k_adam(int n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// e ^= d and s ^= H d from the decision words left by the head: dec[word][site]
// holds the three edges' words (as 32-bit halves) at the site.
__global__ void k_dec_apply(Lattice lat, int64_t W, int64_t words, const uint64_t* __restrict__ dec,
                            uint64_t* __restrict__ e, uint64_t* __restrict__ s)
{
    const int64_t w = (int64_t)blockIdx.y * 32 + (threadIdx.x & 31);
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (w >= words || r >= lat.L3) return;
    const Coord rc = site_coord(lat, r);
    const int step[3] = {1, lat.L, lat.L2};
    int nb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nb[a] = r + ((rc.x[a] + 1 == lat.L) ? step[a] * (1 - lat.L) : step[a]);
    const uint64_t* D = dec + w * (int64_t)lat.L3 * 4;
    auto Dd = [&](int site, int d) { return D[(int64_t)site * 4 + d]; };
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const uint64_t own = Dd(r, d);
        if (own) e[((int64_t)d * lat.L3 + r) * W + w] ^= own;
    }
    const uint64_t par0 = Dd(r, 1) ^ Dd(nb[2], 1) ^ Dd(r, 2) ^ Dd(nb[1], 2);
    const uint64_t par1 = Dd(r, 0) ^ Dd(nb[2], 0) ^ Dd(r, 2) ^ Dd(nb[0], 2);
    const uint64_t par2 = Dd(r, 0) ^ Dd(nb[1], 0) ^ Dd(r, 1) ^ Dd(nb[0], 1);
    if (par0) s[((int64_t)0 * lat.L3 + r) * W + w] ^= par0;
    if (par1) s[((int64_t)1 * lat.L3 + r) * W + w] ^= par1;
    if (par2) s[((int64_t)2 * lat.L3 + r) * W + w] ^= par2;
}

int64_t padded(int64_t n) { return (n + kTile - 1) / kTile * kTile; }
size_t act_bytes(int L, int64_t n) { return (size_t)L * L * L * (size_t)padded(n) * kC * 2; }
size_t round256(size_t x) { return (x + 255) / 256 * 256; }

dim3 conv_grid(int L, int64_t n) { return dim3((unsigned)((L * L * L + 7) / 8), (unsigned)(padded(n) / kTile)); }

}  // namespace cnn
}  // namespace t3d

using namespace t3d;
using namespace t3d::cnn;

extern "C" int toric3d_cnn_param_count(void) { return kParams; }

extern "C" size_t toric3d_cnn_blob_bytes(void) { return sizeof(Blob); }

extern "C" t3d_status toric3d_cnn_prepare(const float* params, void* blob, t3d_stream stream)
{
    clear_error();
    T3D_REQUIRE(params != nullptr && aligned(params, 4), "params must be a device float array");
    T3D_REQUIRE(blob != nullptr && aligned(blob, 16), "blob must be 16-byte aligned");
    k_prepare<<<(3 * kOff * kC * kC + 255) / 256, 256, 0, as_stream(stream)>>>(params, static_cast<Blob*>(blob));
    T3D_LAUNCH_CHECK("cnn prepare");
    return T3D_OK;
}

extern "C" t3d_status toric3d_cnn_status(void)
{
    clear_error();
    return tc_status();
}

extern "C" t3d_status toric3d_cnn_debug_wait_limit(uint64_t ns)
{
    clear_error();
    return tc_set_wait_limit(ns);
}

extern "C" size_t toric3d_cnn_workspace_bytes(int L, int64_t n_samples)
{
    if (L < 2 || L > 128 || n_samples < 1) return 0;
    return cnn_workspace_bytes(L, n_samples);
}

static t3d_status cnn_checks(int L, int64_t n_samples)
{
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(L <= 128, "the pre-decoder supports L <= 128");
    T3D_REQUIRE(n_samples >= 1 && padded(n_samples) / kTile <= 65535, "n_samples out of range");
    return T3D_OK;
}

namespace t3d {

// The decode pass on n_samples samples whose bit-sliced rows have stride W
// words (a chunk of a larger batch when the pointers are offset).
t3d_status launch_cnn_decode(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, uint64_t* s,
                             uint64_t* e, const void* blob, float* logits_out, void* work, cudaStream_t st)
{
    using namespace t3d::cnn;
    const int64_t words = words_for(n_samples);
    uint64_t* dec = reinterpret_cast<uint64_t*>(work);
    void* fwd = static_cast<char*>(work) + round256((size_t)words * L * L * L * 32);
    T3D_TRY(launch_forward_tc(L, n_samples, W, s_prev, s, dec, static_cast<const Blob*>(blob), logits_out, fwd, st));
    ProfScope prof(T3D_K_CNN, st);
    const Lattice lat = make_lattice_host(L);
    dim3 sg((unsigned)((L * L * L + 7) / 8), (unsigned)((words + 31) / 32));
    k_dec_apply<<<sg, 256, 0, st>>>(lat, W, words, dec, e, s);
    T3D_LAUNCH_CHECK("cnn correction");
    return T3D_OK;
}

size_t cnn_workspace_bytes(int L, int64_t n_samples)
{
    using namespace t3d::cnn;
    return round256((size_t)words_for(n_samples) * L * L * L * 32) + tc_workspace_bytes(L, n_samples);
}

// e ^= d, s ^= H d from decision words dec[word][site][4] (the three edges'
// words at the site as 32-bit halves; slot 3 unused).
t3d_status launch_dec_apply(const Lattice& lat, int64_t W, int64_t words, const uint64_t* dec, uint64_t* e,
                            uint64_t* s, cudaStream_t st)
{
    dim3 sg((unsigned)((lat.L3 + 7) / 8), (unsigned)((words + 31) / 32));
    cnn::k_dec_apply<<<sg, 256, 0, st>>>(lat, W, words, dec, e, s);
    T3D_LAUNCH_CHECK("decision apply");
    return T3D_OK;
}

}  // namespace t3d

extern "C" t3d_status toric3d_cnn_decode(int L, int64_t n_samples, const uint64_t* s_prev, uint64_t* s,
                                         uint64_t* e, const void* blob, float* logits_out, void* work,
                                         size_t work_bytes, t3d_stream stream)
{
    clear_error();
    T3D_TRY(cnn_checks(L, n_samples));
    T3D_TRY(check_words(s_prev, "s_prev"));
    T3D_TRY(check_words(s, "s"));
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(blob != nullptr && aligned(blob, 16), "blob must be 16-byte aligned");
    T3D_REQUIRE(work != nullptr && aligned(work, 256), "work must be 256-byte aligned");
    T3D_REQUIRE(work_bytes >= toric3d_cnn_workspace_bytes(L, n_samples), "workspace too small: %zu < %zu",
                work_bytes, toric3d_cnn_workspace_bytes(L, n_samples));
    return launch_cnn_decode(L, n_samples, words_for(n_samples), s_prev, s, e, blob, logits_out, work,
                             as_stream(stream));
}

extern "C" size_t toric3d_cnn_train_workspace_bytes(int L, int64_t n_samples)
{
    if (L < 2 || L > 128 || n_samples < 1) return 0;
    const size_t ab = round256(act_bytes(L, n_samples));
    const size_t part = round256((size_t)((padded(n_samples) + kChunk - 1) / kChunk) * (kOff + 1) * kC * kC * 4);
    return 5 * ab + part + round256(kParams * 4) + 256;
}

extern "C" t3d_status toric3d_cnn_train_step(int L, int64_t n_samples, const uint64_t* s_prev,
                                             const uint64_t* s, const uint64_t* e_label, float* params,
                                             float* adam_m, float* adam_v, int step, float lr,
                                             void* blob, float* grads_out, float* loss_out, void* work,
                                             size_t work_bytes, t3d_stream stream)
{
    clear_error();
    T3D_TRY(cnn_checks(L, n_samples));
    T3D_TRY(check_words(s_prev, "s_prev"));
    T3D_TRY(check_words(s, "s"));
    T3D_TRY(check_words(e_label, "e_label"));
    T3D_REQUIRE(params && adam_m && adam_v && blob && loss_out, "params, adam state, blob and loss_out are required");
    T3D_REQUIRE(step >= 1, "Adam step counts from 1");
    T3D_REQUIRE(work != nullptr && aligned(work, 256), "work must be 256-byte aligned");
    T3D_REQUIRE(work_bytes >= toric3d_cnn_train_workspace_bytes(L, n_samples), "workspace too small");
    cudaStream_t st = as_stream(stream);
    Blob* b = static_cast<Blob*>(blob);
    char* base = static_cast<char*>(work);
    const size_t ab = round256(act_bytes(L, n_samples));
    uint32_t* x0 = reinterpret_cast<uint32_t*>(base);
    uint32_t* y1 = reinterpret_cast<uint32_t*>(base + ab);
    uint32_t* y2 = reinterpret_cast<uint32_t*>(base + 2 * ab);
    uint32_t* g3 = reinterpret_cast<uint32_t*>(base + 3 * ab);   // dPre3, later dPre1
    uint32_t* g2 = reinterpret_cast<uint32_t*>(base + 4 * ab);   // dPre2
    const int chunks = (int)((padded(n_samples) + kChunk - 1) / kChunk);
    float* part = reinterpret_cast<float*>(base + 5 * ab);
    float* grads = reinterpret_cast<float*>(base + 5 * ab +
                                            round256((size_t)chunks * (kOff + 1) * kC * kC * 4));
    if (grads_out) grads = grads_out;
    const Lattice lat = make_lattice_host(L);
    const int64_t Sp = padded(n_samples), W = words_for(n_samples);
    T3D_CUDA_CHECK(cudaMemsetAsync(grads, 0, kParams * sizeof(float), st));
    T3D_CUDA_CHECK(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
    const dim3 grid = conv_grid(L, n_samples);
    ProfScope prof(T3D_K_CNN, st);
    k_features<<<(unsigned)(((int64_t)lat.L3 * Sp + 255) / 256), 256, 0, st>>>(lat, Sp, W, s_prev, s, x0);
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.lat = lat;
    a.Sp = Sp;
    a.n_samples = n_samples;
    a.W = W;
    a.s_prev = s_prev;
    a.s_cur = s;
    // forward
    a.w = &b->wf[0][0][0][0];
    a.bias = b->bias[0];
    a.y = y1;
    k_conv<kInBits, kOutRelu><<<grid, kThreads, 0, st>>>(a);
    a.x = y1;
    a.w = &b->wf[1][0][0][0];
    a.bias = b->bias[1];
    a.y = y2;
    k_conv<kInAct, kOutRelu><<<grid, kThreads, 0, st>>>(a);
    a.x = y2;
    a.w = &b->wf[2][0][0][0];
    a.bias = b->bias[2];
    a.w4 = &b->w4[0][0];
    a.b4 = b->b4;
    a.y = g3;
    a.label = e_label;
    a.inv_n = 1.0f / (3.0f * (float)lat.L3 * (float)n_samples);
    a.grad_w4 = grads + P_W4;
    a.grad_b4 = grads + P_B4;
    a.loss = loss_out;
    k_conv<kInAct, kOutHeadTrain><<<grid, kThreads, 0, st>>>(a);
    T3D_LAUNCH_CHECK("cnn forward");
    // backward: layer 3 weights, then data gradient into layer 2 (masked by y2 > 0), ...
    const dim3 wg(kOff + 1, (unsigned)chunks);
    const int red = ((kOff + 1) * kC * kC + 255) / 256;
    k_wgrad<<<wg, 256, 0, st>>>(lat, Sp, n_samples, y2, g3, part);
    k_wgrad_reduce<<<red, 256, 0, st>>>(chunks, part, grads + P_W3, grads + P_B3, kC);
    ConvArgs bk;
    std::memset(&bk, 0, sizeof(bk));
    bk.lat = lat;
    bk.Sp = Sp;
    bk.n_samples = n_samples;
    bk.W = W;
    bk.x = g3;
    bk.w = &b->wt[2][0][0][0];
    bk.mask = y2;
    bk.y = g2;
    k_conv<kInAct, kOutMask><<<grid, kThreads, 0, st>>>(bk);
    k_wgrad<<<wg, 256, 0, st>>>(lat, Sp, n_samples, y1, g2, part);
    k_wgrad_reduce<<<red, 256, 0, st>>>(chunks, part, grads + P_W2, grads + P_B2, kC);
    bk.x = g2;
    bk.w = &b->wt[1][0][0][0];
    bk.mask = y1;
    bk.y = g3;  // dPre1
    k_conv<kInAct, kOutMask><<<grid, kThreads, 0, st>>>(bk);
    k_wgrad<<<wg, 256, 0, st>>>(lat, Sp, n_samples, x0, g3, part);
    k_wgrad_reduce<<<red, 256, 0, st>>>(chunks, part, grads + P_W1, grads + P_B1, kInC);
    T3D_LAUNCH_CHECK("cnn backward");
    if (lr > 0.0f) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
        k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(kParams, params, adam_m, adam_v, grads, lr, b1, b2, 1e-8f,
                                                       c1, c2);
        k_prepare<<<(3 * kOff * kC * kC + 255) / 256, 256, 0, st>>>(params, b);
        T3D_LAUNCH_CHECK("cnn update");
    }
    return T3D_OK;
}
