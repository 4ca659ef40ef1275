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

}  // namespace cnn
}  // namespace t3d
