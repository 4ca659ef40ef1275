// Learned pre-decoder: network constants and the prepared weight blob shared
// by the training kernels (mma.sync) and the inference kernels (tcgen05).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/toric3d.h"

namespace t3d {
namespace cnn {

constexpr int kC = 16;          // channels of every hidden layer
constexpr int kInC = 6;         // input channels
constexpr int kOff = 27;        // 3x3x3 offsets: k = (dz+1)*9 + (dy+1)*3 + (dx+1), neighbour r + (dx, dy, dz)

// Master parameters (FP32), PyTorch order.
constexpr int P_W1 = 0;                          // [16][6][27]
constexpr int P_B1 = P_W1 + kC * kInC * kOff;    // [16]
constexpr int P_W2 = P_B1 + kC;                  // [16][16][27]
constexpr int P_B2 = P_W2 + kC * kC * kOff;
constexpr int P_W3 = P_B2 + kC;
constexpr int P_B3 = P_W3 + kC * kC * kOff;
constexpr int P_W4 = P_B3 + kC;                  // [3][16]
constexpr int P_B4 = P_W4 + 3 * kC;              // [3]
constexpr int kParams = P_B4 + 3;                // 16,515

// Prepared device blob.
struct Blob {
    __nv_bfloat16 wf[3][kOff][kC][kC];   // forward: [layer][k][co][ci] (layer 1: ci >= 6 zero)
    __nv_bfloat16 wt[3][kOff][kC][kC];   // backward data: [layer][k][ci][co] = wf[layer][26-k][co][ci]
    float bias[3][kC];
    float w4[3][kC];
    float b4[3];
};

// The tensor-core inference forward pass (conv 1..3 + head) on n_samples
// samples whose bit-sliced rows have stride W words: leaves the decisions
// (logit > 0) in dec ([word][site][4] uint64, the three edges' words at the
// site; e and s are updated from them by the caller).  work:
// tc_workspace_bytes(L, n_samples).
size_t tc_workspace_bytes(int L, int64_t n_samples);
t3d_status launch_forward_tc(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, const uint64_t* s,
                             uint64_t* dec, const Blob* blob, float* logits_out, void* work, cudaStream_t st);
// Per-device launch attributes of the tensor-core kernels (call before any
// stream capture; idempotent).
t3d_status tc_prepare();
// T3D_OK, or T3D_ETIMEOUT if a tensor-core kernel gave up a bounded wait since
// the last call (reads and clears the device flag; synchronises the device).
t3d_status tc_status();
t3d_status tc_set_wait_limit(uint64_t ns);

// Training on the same tensor-core convolutions.  Activations and gradients are
// tile-major: the 128-sample tile t of site r is one block at byte
// (t L^3 + r) * (256 * channels), [sample/8][channel/8][8 samples][8 channels]
// BF16 for 16 channels, [sample][8] for the first layer's 8 (6 used).
// tc_act_bytes: one such buffer.
size_t tc_act_bytes(int L, int64_t n_samples, int channels);
// Forward pass with the labels: x0 (8 channels) the syndrome features, y1 and y2
// the hidden activations, g3 the gradient at the third layer's pre-activation of
// the mean BCE; the head's gradients and the summed BCE are added to grad_w4
// [3][16], grad_b4 [3] and loss [1].
t3d_status tc_train_forward(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, const uint64_t* s,
                            const uint64_t* label, const Blob* blob, uint8_t* x0, uint8_t* y1, uint8_t* y2,
                            uint8_t* g3, float* grad_w4, float* grad_b4, float* loss, cudaStream_t st);
// Backward data through one convolution: g_out = conv(g_in; wt) where the forward
// activation mask_act is non-zero, else 0 (wt: the transposed, flipped weights).
t3d_status tc_backward_data(int L, int64_t n_samples, const __nv_bfloat16* wt, const uint8_t* g_in,
                            const uint8_t* mask_act, uint8_t* g_out, cudaStream_t st);
// Weight and bias gradients of one convolution on the tensor cores: x (x_ch = 8 or 16
// channels) and d (16) tile-major; xt, dt scratch of tc_act_bytes(L, n_samples, 16) for
// their channel-major copies; ones: a 4 KiB tile of BF16 ones (tc_fill_ones).  Adds
// gw[co][ci][27] (ci < cin_kept) and gb[16].
t3d_status tc_fill_ones(uint8_t* tile, cudaStream_t st);
t3d_status tc_weight_grad(int L, int64_t n_samples, int x_ch, int cin_kept, const uint8_t* x, const uint8_t* d,
                          uint8_t* xt, uint8_t* dt, const uint8_t* ones, float* gw, float* gb, cudaStream_t st);

}  // namespace cnn
}  // namespace t3d
