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
// The convolutions of inference and training run on the tcgen05 tensor
// cores (t3d_cnn_tc.cu): activations are BF16 and tile-major, FP32
// accumulation in TMEM; hidden activations are rounded to BF16 between layers
// and the head reads the third layer's output in FP32.
//
// Training: the forward pass with the labels in the third layer's epilogue
// (BCE gradient, the head's gradients, the ReLU mask), backward data by the
// same tensor-core convolution with flipped and transposed weights and a
// masking epilogue, weight and bias gradients by a CUDA-core reduction over
// sites and samples, Adam.
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

constexpr int kTile = 128;      // samples per tensor-core tile

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
size_t round256(size_t x) { return (x + 255) / 256 * 256; }


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
    // (the weight-gradient grid has one row per 64 samples; 2,097,120 samples in all)
    T3D_REQUIRE(n_samples >= 1 && padded(n_samples) <= 65535LL * 32, "n_samples out of range");
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
    // features, y1, y2, two gradient buffers, two channel-major copies, the ones tile, grads
    return tc_act_bytes(L, n_samples, 8) + 6 * tc_act_bytes(L, n_samples, kC) + 4096 + round256(kParams * 4) + 256;
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
    uint8_t* base = static_cast<uint8_t*>(work);
    const size_t xb = tc_act_bytes(L, n_samples, 8), ab = tc_act_bytes(L, n_samples, kC);
    uint8_t* x0 = base;                 // the syndrome features
    uint8_t* y1 = base + xb;
    uint8_t* y2 = y1 + ab;
    uint8_t* g3 = y2 + ab;              // dPre3, later dPre1
    uint8_t* g2 = g3 + ab;              // dPre2
    uint8_t* xt = g2 + ab;              // channel-major copies for the weight gradients
    uint8_t* dt = xt + ab;
    uint8_t* ones = dt + ab;
    float* grads = reinterpret_cast<float*>(ones + 4096);
    if (grads_out) grads = grads_out;
    const int64_t W = words_for(n_samples);
    T3D_CUDA_CHECK(cudaMemsetAsync(grads, 0, kParams * sizeof(float), st));
    T3D_CUDA_CHECK(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
    T3D_TRY(tc_fill_ones(ones, st));
    // forward, with the BCE gradient and the head's gradients in the last layer's epilogue
    T3D_TRY(tc_train_forward(L, n_samples, W, s_prev, s, e_label, b, x0, y1, y2, g3, grads + P_W4, grads + P_B4,
                             loss_out, st));
    // backward: layer 3's weights, the data gradient into layer 2 (gated by y2 > 0), ...
    T3D_TRY(tc_weight_grad(L, n_samples, kC, kC, y2, g3, xt, dt, ones, grads + P_W3, grads + P_B3, st));
    T3D_TRY(tc_backward_data(L, n_samples, &b->wt[2][0][0][0], g3, y2, g2, st));
    T3D_TRY(tc_weight_grad(L, n_samples, kC, kC, y1, g2, xt, dt, ones, grads + P_W2, grads + P_B2, st));
    T3D_TRY(tc_backward_data(L, n_samples, &b->wt[1][0][0][0], g2, y1, g3, st));   // dPre1
    T3D_TRY(tc_weight_grad(L, n_samples, 8, kInC, x0, g3, xt, dt, ones, grads + P_W1, grads + P_B1, st));
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
