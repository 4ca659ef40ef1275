// The learned pre-decoder's convolutions on the fifth-generation tensor cores
// (tcgen05 MMA with TMEM accumulators, operands staged in shared memory): the
// inference forward pass, and for training the forward pass with the loss and
// the backward-data passes (the same kernel with another epilogue).
//
// Each 3x3x3 convolution (16 output channels) is a sum of GEMMs over the input
// sites: for an input site i and every output site o within one step of it,
//   D_o[sample][co] += A_i[sample][ci] . W(i - o)[co][ci],   M = 128, K = 16,
// where A_i is the 128-sample activation tile of site i.  A tcgen05.mma with
// M = 128, K = 16 takes about as long for N = 16 as for N = 64 (the issue
// floor, about 53 cycles; N = 128 takes 64 and N = 256 128, the bf16 peak), so
// one MMA serves every output of a work unit that an input tile reaches: its N
// stacks those outputs' weight blocks (the column kernel below).
//
// Work unit: one 128-sample tile x one 2 x 2 column of output sites running
// through all L planes in z.  The CTA streams the unit's input planes
// z = -1 .. L, each the 4 x 4 input sites around the column (periodic wrap);
// each input tile reaches shared memory once and is multiplied, by one MMA,
// into every column site of the three output planes it touches.  TMEM keeps a
// ring of eight output planes; the epilogue drains a plane once its last
// input plane has been multiplied.
//
// Warp roles (192 threads, one CTA per SM):
//   warps 0-3  epilogue: tcgen05.ld of a finished plane (warp w reads TMEM lanes
//              32w..32w+31 = samples), then by mode (TcMode): bias + ReLU +
//              BF16 store of the next layer's input; the 16 -> 3 head and the
//              hard decisions; the head with the BCE gradient, the head's
//              gradients and the gradient at the pre-activation; or the
//              backward-data gradient gated by the forward activation;
//   warp 4     producer: sixteen lanes issue the bulk copies of a plane's 16
//              tiles at once (first layer: four lanes copy a row's four 2 KiB
//              tiles each as one run) into a ring of shared-memory slots;
//   warp 5     MMA issuer: one thread issues the MMAs and commits their
//              completion to the slot's "empty" barrier and to the output
//              plane's "accumulators full" barrier.
// Every wait is bounded (one second; toric3d_cnn_debug_wait_limit shortens the
// waits that may give up, so a test can make them run out); a wait that gives
// up sets the device error flag and the CTA winds down (waiting, again bounded
// but always by the full second, for its copies and MMAs in flight, and
// freeing its TMEM) so the context stays usable.
//
// Shared-memory operand layout ("no swizzle", K-major): core matrices of 8 rows
// x 16 bytes stored contiguously.  Hidden activations in global memory use the
// same layout, [sample/8][channel/8][8 samples][8 channels] BF16 per tile, and
// the tile of (site, 128-sample tile m) starts at byte (m L^3 + site) 4096, so
// a tile is one contiguous 4 KiB block (K-direction core-matrix stride (LBO)
// 128 B, M-direction stride (SBO) 256 B).  The first layer's input tile (6 of 8
// channels used: s_{t-1} then s_t of the three faces) is [sample][8], 2 KiB
// (SBO 128 B); two x-adjacent sites form one K = 16 operand as its two K chunks
// (LBO 2 KiB).  Weight blocks: [co/8][ci/8][co%8][ci%8] (512 B, LBO 128 B,
// SBO 256 B).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "t3d_cnn.cuh"
#include "t3d_device.cuh"
#include "t3d_host.hpp"

namespace t3d {
namespace cnn {
namespace {

constexpr int kTileM = 128;                         // samples per tile (MMA M)
constexpr uint32_t kTmemCols = 512;
constexpr int kSlotBytes = 4096;                    // one hidden-layer tile
constexpr int kEpiWarps = 4;
constexpr int kProducerWarp = 4;
constexpr int kIssuerWarp = 5;
constexpr int kTcThreads = 32 * (kIssuerWarp + 1);
constexpr uint64_t kWaitNs = 1000000000ull;         // bound of every wait

__device__ unsigned int g_tc_error;   // bit 0: a bounded wait gave up
// bound of the waits that may give up (the wind-down drains always use kWaitNs)
__device__ unsigned long long g_tc_wait_ns = kWaitNs;

// What the epilogue makes of a finished output plane.
enum TcMode {
    kTcRelu = 0,        // bias + ReLU, BF16 activations for the next layer
    kTcHead = 1,        // bias + ReLU, the 16 -> 3 head, hard decisions (and optional logits)
    kTcHeadTrain = 2,   // training: the head, the BCE gradient against the labels, the head's
                        // gradients and the loss, and the gradient at the layer's pre-activation
    kTcMask = 3,        // backward data: the gradient gated by the forward activation's sign
};
__host__ __device__ constexpr bool tc_head(int mode) { return mode == kTcHead || mode == kTcHeadTrain; }

struct TcArgs {
    int L, L3;
    int64_t Sp;                 // padded samples of the activation buffers (multiple of 128)
    int64_t n_samples;
    int64_t W;                  // row stride of the bit-sliced arrays (words)
    int64_t words;              // words of this pass
    int ncx;                    // 2 x 2 columns per axis (ceil(L / 2))
    int64_t n_units;
    const uint8_t* in;          // input activations
    uint8_t* out;               // output activations / gradients (all modes but kTcHead)
    const __nv_bfloat16* w;     // [27][co][ci]
    const float* bias;          // [16]
    const float* w4;            // head [3][16]
    const float* b4;            // [3]
    uint32_t* dec32;            // kTcHead: decision words [word][site][8] 32-bit halves
    float* logits;              // kTcHead: optional [3][L^3][n_samples]
    const uint64_t* label;      // kTcHeadTrain: bit-sliced labels [3][L^3][W]
    float inv_n;                // kTcHeadTrain: 1 / (3 L^3 n_samples)
    float* grad_w4;             // kTcHeadTrain: [3][16], accumulated
    float* grad_b4;             // kTcHeadTrain: [3], accumulated
    float* loss;                // kTcHeadTrain: [1], accumulated
    const uint8_t* mask_act;    // kTcMask: the forward activation at the output sites
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity.  Gives up after
// g_tc_wait_ns, or early once another role of the CTA has given up (abort
// flag), unless ignore_abort (the final drain of work in flight, bounded by
// kWaitNs whatever the debug limit).
__device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile uint32_t* abort_flag, bool ignore_abort = false)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    const uint64_t limit = ignore_abort ? kWaitNs : *(volatile unsigned long long*)&g_tc_wait_ns;
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (!ignore_abort && *abort_flag) return false;
        if (global_ns() - t0 > limit) {
            *abort_flag = 1;
            atomicOr(&g_tc_error, 1u);
            return false;
        }
    }
}

// Wait for phase 0 of a barrier that completes only at the end of a long launch: gives up
// (error flag, abort) once *progress has not changed for g_tc_wait_ns.
__device__ bool wait_bar_progress(uint32_t bar, volatile uint32_t* progress, volatile uint32_t* abort_flag)
{
    uint64_t t0 = global_ns();
    uint32_t last = *progress;
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, 0)) return true;
        if (*abort_flag) return false;
        const uint32_t now_p = *progress;
        const uint64_t now = global_ns();
        if (now_p != last) {
            last = now_p;
            t0 = now;
        } else if (now - t0 > *(volatile unsigned long long*)&g_tc_wait_ns) {
            *abort_flag = 1;
            atomicOr(&g_tc_error, 1u);
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Whole warp: allocate ncols TMEM columns; the base address goes to smem.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// D += A . B^T with the instruction descriptor of this MMA (N varies).
__device__ __forceinline__ void mma_bf16_n(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc)
{
    asm volatile(
        "{\n"
        ".reg .pred pa;\n"
        "setp.ne.b32 pa, 1, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n"
        "}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc)
        : "memory");
}

// D = A . B^T, not accumulating (the first MMA into an accumulator).
__device__ __forceinline__ void mma_bf16_overwrite(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc)
{
    asm volatile(
        "{\n"
        ".reg .pred pa;\n"
        "setp.ne.b32 pa, 0, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n"
        "}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc)
        : "memory");
}

// Warp: zero 32 TMEM lanes x 16 consecutive 32-bit columns (one lane per thread).
__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr),
        "r"(z)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Arrive on the barrier once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Warp: 32 TMEM lanes x 16 consecutive 32-bit columns, one lane per thread
// (asynchronous: the registers are valid after tmem_wait_ld).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// ------------------------------------------------------------------ schedule
struct Unit {
    int64_t m0;      // first sample of the tile
    int x0, y;       // column origin (even)
};

// v in [-L, 2L): periodic coordinate
__device__ __forceinline__ int wrap(int v, int L)
{
    return v < 0 ? v + L : (v >= L ? v - L : v);
}

// Activation layout: the tile of (site, 128-sample tile m) starts at byte
// (m L^3 + site) tile_bytes, so a tile is contiguous and so are the tiles of
// x-adjacent sites of one row (bulk copies of whole runs of a row move more
// bytes per clock than one copy per tile).
__device__ __forceinline__ int64_t tile_off(int64_t site, int64_t m0, int L3, uint32_t tile_bytes)
{
    return ((m0 >> 7) * L3 + site) * (int64_t)tile_bytes;
}

// Copy the tiles of sites row + wrap(x0 + i), i = 0 .. n - 1, to dst + i tile_bytes: one bulk
// copy per run of consecutive sites (a row wraps at x = L at most once when n <= L + 2, twice
// for the smallest lattices).
__device__ __forceinline__ void copy_row(uint32_t dst, const uint8_t* in, int64_t row, int x0, int n, int L, int L3,
                                         int64_t m0, uint32_t tile_bytes, uint32_t bar)
{
    int i = 0;
    while (i < n) {
        const int x = wrap(x0 + i, L);
        int k = 1;
        while (i + k < n && x + k < L && wrap(x0 + i + k, L) == x + k) ++k;
        bulk_load(dst + (uint32_t)i * tile_bytes, in + tile_off(row + x, m0, L3, tile_bytes), (uint32_t)k * tile_bytes,
                  bar);
        i += k;
    }
}

// ------------------------------------------------------------------ column kernel
// The convolution with dense operands: a work unit is one 128-sample tile x one
// 2 x 2 column of output sites (x0, x0 + 1) x (y0, y0 + 1) run through all L
// planes in z.  Every input site (xi, yi) of an input plane zi with
// xi = x0 - 1 .. x0 + 2, yi = y0 - 1 .. y0 + 2 feeds the column sites within
// one step of it in x and y, in the three output planes zi - 1, zi, zi + 1;
// TMEM keeps eight output planes of 64 columns (4 sites x 16 channels, site
// j = jx + 2 jy) in a ring, so one MMA covers the input tile's whole reach:
// the columns from (plane zi - 1, its lowest site lo) to (plane zi + 1, its
// highest site hi), N = 16 (4 (P2 - P1) + hi - lo + 1) for the planes P1..P2
// that exist (N = 192 for the four inner sites).  Its B operand is a window of
// one per-position sequence of weight blocks [plane zi - 1: sites lo..3 |
// plane zi: 0..3 | plane zi + 1: 0..hi], W(xi - xo, yi - yo, zi - zo) or zero
// where the site is out of reach; of the blocks multiplied 64% are non-zero
// (108 of 168 per plane).  A window that would cross
// the ring's end is split in two MMAs.  TMEM columns are zeroed by the
// epilogue after it drains a plane (and once at the start), so every MMA
// accumulates.  The first layer pairs x-adjacent input sites in one K = 16
// operand (chunk c = site 2p - 1 + c of the row; LBO 2 KiB steps to the second site).
// Input ring of 128 KiB: two planes of 16 x 4 KiB tiles (hidden layers) or four of 16 x 2 KiB
// (first layer).
constexpr int kColRingBytes = 32 * kSlotBytes;
__host__ __device__ constexpr int col_in_slots(bool bits_in) { return bits_in ? 4 : 2; }
constexpr int kColInMax = 4;
constexpr int kColSlots = 8;                              // output planes resident in TMEM
constexpr int kColPlaneCols = 4 * kC;                     // 64
constexpr int kColWBlocks = 168;                          // windows of the 16 positions (hidden layers)
constexpr int kColOffW = kColRingBytes;
constexpr int kColOffBar = kColOffW + kColWBlocks * 512;
constexpr int kColNumBars = 2 * kColInMax + 2 * kColSlots + 1;   // full, empty, acc_full, acc_empty, done
constexpr int kColOffMisc = kColOffBar + kColNumBars * 8;
constexpr int kColOffPos = kColOffMisc + 16;              // ColPos[16]
constexpr int kColSmemBytes = kColOffPos + 16 * 12 + 1024;
static_assert(kColSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kColSlots * kColPlaneCols == 512, "TMEM ring");

// Operand position p of a row (hidden: the site x0 - 1 + p; first layer: the
// pair x0 - 1 + 2p, x0 + 2p) at row b (yi = y0 - 1 + b): the column sites in
// reach span lo..hi, and its weight sequence starts at block base.
struct ColPos {
    int base, lo, hi;
};

__host__ __device__ constexpr int col_chunk_dx(bool bits_in, int p, int c) { return bits_in ? 2 * p - 1 + c : p - 1; }

__host__ __device__ constexpr bool col_reach(bool bits_in, int p, int jx)
{
    for (int c = 0; c < 2; ++c) {
        const int dx = col_chunk_dx(bits_in, p, c) - jx;
        if (dx >= -1 && dx <= 1) return true;
    }
    return false;
}

__host__ __device__ constexpr ColPos col_pos(bool bits_in, int p, int b)
{
    const int P = bits_in ? 2 : 4;
    int base = 0;
    ColPos r = {0, 0, 0};
    for (int bb = 0; bb < 4; ++bb)
        for (int pp = 0; pp < P; ++pp) {
            int jx_lo = 2, jx_hi = -1;
            for (int jx = 0; jx < 2; ++jx)
                if (col_reach(bits_in, pp, jx)) {
                    jx_lo = jx < jx_lo ? jx : jx_lo;
                    jx_hi = jx;
                }
            const int jy_lo = bb == 3 ? 1 : 0, jy_hi = bb == 0 ? 0 : 1;   // yi - yo in -1..1
            const int lo = jx_lo + 2 * jy_lo, hi = jx_hi + 2 * jy_hi;
            if (bb == b && pp == p) {
                r.base = base;
                r.lo = lo;
                r.hi = hi;
            }
            base += (4 - lo) + 4 + (hi + 1);
        }
    return r;
}

// The positions' table, evaluated at compile time so the issuer's unrolled loops
// see constants.
struct ColTable {
    ColPos pos[16];
};

__host__ __device__ constexpr ColTable make_col_table(bool bits_in)
{
    ColTable t = {};
    const int P = bits_in ? 2 : 4;
    for (int b = 0; b < 4; ++b)
        for (int p = 0; p < P; ++p) t.pos[b * P + p] = col_pos(bits_in, p, b);
    return t;
}

__device__ __forceinline__ Unit col_unit_of(const TcArgs& a, int64_t u)
{
    const int64_t cols = (int64_t)a.ncx * a.ncx;
    const int64_t tile = u / cols;
    const int rem = (int)(u - tile * cols);
    Unit t;
    t.m0 = tile * kTileM;
    t.y = (rem / a.ncx) * 2;
    t.x0 = (rem % a.ncx) * 2;
    return t;
}

template <int kMode, bool kBitsIn>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_col(const __grid_constant__ TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t ring = smem_u32(sm);
    const uint32_t wsm = ring + kColOffW;
    const uint32_t bars = ring + kColOffBar;
    constexpr int kColIn = col_in_slots(kBitsIn);
    constexpr uint32_t kColInBytes = (uint32_t)(kColRingBytes / kColIn);
    auto full_bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    auto empty_bar = [&](int i) { return bars + 8u * (uint32_t)(kColInMax + i); };
    auto accf_bar = [&](int i) { return bars + 8u * (uint32_t)(2 * kColInMax + i); };
    auto acce_bar = [&](int i) { return bars + 8u * (uint32_t)(2 * kColInMax + kColSlots + i); };
    const uint32_t done_bar = bars + 8u * (uint32_t)(2 * kColInMax + 2 * kColSlots);
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + kColOffMisc);   // [0] TMEM base, [1] abort flag
    volatile uint32_t* abort_flag = misc + 1;
    ColPos* s_pos = reinterpret_cast<ColPos*>(sm + kColOffPos);   // [b * P + p]
    constexpr int P = kBitsIn ? 2 : 4;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x < 4 * P) s_pos[threadIdx.x] = col_pos(kBitsIn, threadIdx.x % P, threadIdx.x / P);
    __syncthreads();
    // weight windows: for every position (p, b) and element e of its sequence, block
    // W(dx, dy, dz) in the B-operand layout [co/8][chunk][co%8][ci%8], zero out of reach
    {
        const ColPos last = s_pos[4 * P - 1];
        const int n_blocks = last.base + (4 - last.lo) + 4 + (last.hi + 1);
        for (int i = threadIdx.x; i < n_blocks * 256; i += blockDim.x) {
            const int blk = i >> 8, co = (i >> 4) & 15, kk = i & 15;   // kk = chunk * 8 + ci
            // the position owning block blk
            int pb = 0;
            while (pb + 1 < 4 * P && s_pos[pb + 1].base <= blk) ++pb;
            const ColPos pos = s_pos[pb];
            const int p = pb % P, b = pb / P;
            const int e = blk - pos.base;
            const int part = (e + pos.lo) >> 2, j = (e + pos.lo) & 3;   // block index = 4 part + j - lo
            const int jx = j & 1, jy = j >> 1;
            const int c = kk >> 3, ci = kk & 7;
            const int dx = col_chunk_dx(kBitsIn, p, c) - jx;
            const int dy = (b - 1) - jy;
            const int dz = 1 - part;
            __nv_bfloat16 w = __float2bfloat16_rn(0.0f);
            const int ch = kBitsIn ? ci : c * 8 + ci;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
                const int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                w = a.w[(k * kC + co) * kC + ch];
            }
            *reinterpret_cast<__nv_bfloat16*>(sm + kColOffW + blk * 512 + (co >> 3) * 256 + c * 128 + (co & 7) * 16 +
                                              ci * 2) = w;
        }
    }
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        for (int i = 0; i < kColIn; ++i) {
            mbar_init(full_bar(i), 1);
            mbar_init(empty_bar(i), 1);
        }
        for (int i = 0; i < kColSlots; ++i) {
            mbar_init(accf_bar(i), 1);
            mbar_init(acce_bar(i), kEpiWarps);
        }
        mbar_init(done_bar, 1);
        misc[1] = 0;
        fence_mbar_init();
    }
    if (warp == kIssuerWarp) tmem_alloc(smem_u32(misc), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    // every accumulator starts at zero (the epilogue re-zeroes a plane after draining it)
    if (warp < kEpiWarps) {
#pragma unroll 4
        for (int c = 0; c < kColSlots * kColPlaneCols; c += 16) tmem_zero16(tmem + ((uint32_t)(warp * 32) << 16) + c);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int L = a.L;
    const uint32_t in_row = kBitsIn ? 16u : 32u;
    const uint32_t tile_bytes = kTileM * in_row;

    if (warp == kProducerWarp) {
        // one input plane (the 4 x 4 tiles around the column) per slot, one barrier phase each;
        // lane 4 b + i copies the tile at (x0 - 1 + i, y0 - 1 + b).  Sixteen lanes issuing 4 KiB
        // copies at once measured faster here than four lanes issuing a row's 16 KiB each.
        uint32_t pseq = 0;
        bool ok = true;
        const int b = (lane >> 2) & 3, i = lane & 3;
        for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit t = col_unit_of(a, u);
            const int64_t xy = (int64_t)wrap(t.y - 1 + b, L) * L + wrap(t.x0 - 1 + i, L);
            for (int zi = -1; zi <= L; ++zi) {
                const int g = (int)(pseq % kColIn);
                const uint32_t use = pseq / kColIn;
                int good = 1;
                if (lane == 0 && use > 0) good = wait_bar(empty_bar(g), (use - 1) & 1u, abort_flag) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, good, 0)) {
                    ok = false;
                    break;
                }
                if (lane == 0) mbar_arrive_expect_tx(full_bar(g), 16u * tile_bytes);
                __syncwarp();
                if (kBitsIn) {
                    // 2 KiB tiles: lane b copies row b's four contiguous tiles (8 KiB) in one run
                    if (lane < 4)
                        copy_row(ring + (uint32_t)g * kColInBytes + (uint32_t)lane * 4u * tile_bytes, a.in,
                                 ((int64_t)wrap(zi, L) * L + wrap(t.y - 1 + lane, L)) * L, t.x0 - 1, 4, L, a.L3, t.m0,
                                 tile_bytes, full_bar(g));
                } else if (lane < 16) {
                    bulk_load(ring + (uint32_t)g * kColInBytes + (uint32_t)lane * tile_bytes,
                              a.in + tile_off((int64_t)wrap(zi, L) * L * L + xy, t.m0, a.L3, tile_bytes), tile_bytes,
                              full_bar(g));
                }
                ++pseq;
            }
        }
        // copies still in flight land before the CTA exits
        if (lane == 0) {
            const uint32_t last = pseq < (uint32_t)kColIn ? pseq : (uint32_t)kColIn;
            for (uint32_t g = 0; g < last; ++g) {
                const uint32_t q = pseq - 1 - ((pseq - 1 - g) % kColIn);
                wait_bar(full_bar((int)g), (q / kColIn) & 1u, abort_flag, true);
            }
        }
        __syncwarp();
    } else if (warp == kIssuerWarp) {
        if (lane == 0) {
            uint32_t pseq = 0;
            int64_t qbase = 0;
            bool ok = true;
            const uint32_t a_lbo = kBitsIn ? 2048u : 128u, a_sbo = kBitsIn ? 128u : 256u;
            const uint64_t bdesc0 = smem_desc(wsm, 128u, 256u);   // + 32 per 512-byte block
            constexpr uint32_t kIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileM >> 4) << 24);
            for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
                for (int zi = -1; zi <= L && ok; ++zi) {
                    // output plane zi + 1 is first written by this input plane: its slot must be drained
                    if (zi + 1 <= L - 1) {
                        const int64_t q = qbase + zi + 1;
                        const uint32_t v = (uint32_t)(q >> 3);
                        if (v > 0 && !wait_bar(acce_bar((int)(q & 7)), (v - 1) & 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    const int t1 = zi - 1 < 0 ? 0 : zi - 1, t2 = zi + 1 > L - 1 ? L - 1 : zi + 1;
                    const int P1 = t1 - (zi - 1), P2 = t2 - (zi - 1);           // parts 0..2
                    const int s1 = (int)((qbase + t1) & 7);
                    const int wrap_at = s1 + (t2 - t1) > 7 ? t1 + (8 - s1) : -1;   // first plane in slot 0
                    // the window of position (b, p): blocks 4 P1 .. 4 P2 + hi - lo of its sequence
                    // into TMEM column 64 s1 + 16 lo, N = 16 (4 (P2 - P1) + hi - lo + 1)
                    const uint64_t bdesc_plane = bdesc0 + (uint64_t)(128 * P1);
                    const uint32_t idesc_plane = kIdescBase + ((uint32_t)(8 * (P2 - P1)) << 17);
                    const uint32_t col_plane = tmem + (uint32_t)(s1 * kColPlaneCols);
                    constexpr ColTable kTab = make_col_table(kBitsIn);
                    const int g = (int)(pseq % kColIn);
                    if (!wait_bar(full_bar(g), (pseq / kColIn) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint64_t adesc0 =
                            smem_desc(ring + (uint32_t)g * kColInBytes + (uint32_t)b * 4u * tile_bytes, a_lbo, a_sbo);
                        if (wrap_at < 0) {
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const ColPos pos = kTab.pos[b * P + p];
                                mma_bf16_n(col_plane + (uint32_t)(pos.lo * kC),
                                           adesc0 + (uint64_t)(p * (kSlotBytes >> 4)),
                                           bdesc_plane + (uint64_t)(32 * pos.base),
                                           idesc_plane + ((uint32_t)(2 * (pos.hi - pos.lo + 1)) << 17));
                            }
                        } else {
                            // the window crosses the ring's end: split at slot 0
                            const int Pw = wrap_at - (zi - 1);
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const ColPos pos = kTab.pos[b * P + p];
                                const uint64_t adesc = adesc0 + (uint64_t)(p * (kSlotBytes >> 4));
                                auto issue = [&](int pa, int ja, int pz, int jz, uint32_t col) {
                                    // blocks (pa, ja) .. (pz, jz) of the sequence into TMEM column col
                                    const int b0 = 4 * pa + ja - pos.lo, nb = 4 * (pz - pa) + jz - ja + 1;
                                    mma_bf16_n(tmem + col, adesc, bdesc0 + (uint64_t)(32 * (pos.base + b0)),
                                               kIdescBase | ((uint32_t)(nb * 2) << 17));
                                };
                                issue(P1, pos.lo, Pw - 1, 3, (uint32_t)(s1 * kColPlaneCols + pos.lo * kC));
                                issue(Pw, 0, P2, pos.hi, 0u);
                            }
                        }
                    }
                    mma_commit(empty_bar(g));
                    ++pseq;
                    // output plane zi - 1 has received its last contribution
                    if (zi - 1 >= 0) mma_commit(accf_bar((int)((qbase + zi - 1) & 7)));
                }
                qbase += L;
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(done_bar);
            wait_bar(done_bar, 0, abort_flag, true);
        }
        __syncwarp();
    } else {
        // epilogue: warp w owns TMEM lanes (= tile rows = samples) 32w .. 32w + 31
        const int r = warp * 32 + lane;
        constexpr bool kHead = tc_head(kMode);
        float bias[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) bias[c] = kMode == kTcMask ? 0.0f : a.bias[c];
        float w4[kHead ? 3 * kC : 1];
        float b4[3] = {0.0f, 0.0f, 0.0f};
        if (kHead) {
#pragma unroll
            for (int i = 0; i < 3 * kC; ++i) w4[i] = a.w4[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) b4[d] = a.b4[d];
        }
        // training: this thread's share of the head's gradients and of the loss
        constexpr int kAcc = kMode == kTcHeadTrain ? 3 * kC + 3 + 1 : 1;
        float acc[kAcc];
#pragma unroll
        for (int i = 0; i < kAcc; ++i) acc[i] = 0.0f;
        int64_t q = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit t = col_unit_of(a, u);
            const int64_t sample = t.m0 + r;
            const bool valid = sample < a.n_samples;
            for (int zo = 0; zo < L; ++zo, ++q) {
                const int s = (int)(q & 7);
                int got = 1;
                if (lane == 0) got = wait_bar(accf_bar(s), (uint32_t)(q >> 3) & 1u, abort_flag) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kColPlaneCols);
                uint32_t raw[4][16];
#pragma unroll
                for (int j = 0; j < 4; ++j) tmem_ld16(lane_base + (uint32_t)(j * kC), raw[j]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 4; ++j) tmem_zero16(lane_base + (uint32_t)(j * kC));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int xo = t.x0 + (j & 1), yo = t.y + (j >> 1);
                    if (xo >= L || yo >= L) continue;   // the odd lattice's last column
                    const int64_t site = ((int64_t)zo * L + yo) * L + xo;
                    const int64_t row_off = tile_off(site, t.m0, a.L3, 4096) + (r >> 3) * 256 + (r & 7) * 16;
                    float v[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(raw[j][c]);
                    if (kMode == kTcRelu || kMode == kTcMask) {
                        uint32_t pk[8];
                        if (kMode == kTcRelu) {
#pragma unroll
                            for (int c = 0; c < kC; c += 2)
                                pk[c / 2] = pack2(fmaxf(v[c] + bias[c], 0.0f), fmaxf(v[c + 1] + bias[c + 1], 0.0f));
                        } else {
                            // the gradient passes where the forward activation (a ReLU output,
                            // so never negative) is non-zero
                            const uint4 m0v = *reinterpret_cast<const uint4*>(a.mask_act + row_off);
                            const uint4 m1v = *reinterpret_cast<const uint4*>(a.mask_act + row_off + 128);
                            const uint32_t mw[8] = {m0v.x, m0v.y, m0v.z, m0v.w, m1v.x, m1v.y, m1v.z, m1v.w};
#pragma unroll
                            for (int c = 0; c < kC; c += 2)
                                pk[c / 2] = pack2((mw[c / 2] & 0x7FFFu) ? v[c] : 0.0f,
                                                  (mw[c / 2] & 0x7FFF0000u) ? v[c + 1] : 0.0f);
                        }
                        uint8_t* dst = a.out + row_off;
                        *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
                        float y3[kC];
                        float z[3] = {b4[0], b4[1], b4[2]};
#pragma unroll
                        for (int c = 0; c < kC; ++c) {
                            y3[c] = fmaxf(v[c] + bias[c], 0.0f);
#pragma unroll
                            for (int d = 0; d < 3; ++d) z[d] = fmaf(y3[c], w4[d * kC + c], z[d]);
                        }
                        const int64_t wd = (t.m0 + warp * 32) / 64;
                        const int hw = warp & 1;
                        if (kMode == kTcHead) {
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                if (a.logits && valid)
                                    a.logits[((int64_t)d * a.L3 + site) * a.n_samples + sample] = z[d];
                                const uint32_t bits = __ballot_sync(0xffffffffu, valid && z[d] > 0.0f);
                                if (lane == 0 && wd < a.words) a.dec32[(wd * a.L3 + site) * 8 + 2 * d + hw] = bits;
                            }
                        } else {
                            // binary cross-entropy of the logits against the labels (the mean over
                            // edges and samples is what training minimises): dL/dz = (sigmoid(z) - y) / N
                            float dz[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                const uint64_t lw = wd < a.words ? a.label[((int64_t)d * a.L3 + site) * a.W + wd] : 0ull;
                                const float yv = (float)((uint32_t)(lw >> (32 * hw + lane)) & 1u);
                                const float sig = 1.0f / (1.0f + expf(-z[d]));
                                dz[d] = valid ? (sig - yv) * a.inv_n : 0.0f;
                                if (valid) acc[3 * kC + 3] += fmaxf(z[d], 0.0f) - z[d] * yv + log1pf(expf(-fabsf(z[d])));
                                acc[3 * kC + d] += dz[d];
                            }
                            uint32_t pk[8];
#pragma unroll
                            for (int c = 0; c < kC; c += 2) {
                                float g2[2];
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    float dy = 0.0f;
#pragma unroll
                                    for (int d = 0; d < 3; ++d) {
                                        dy = fmaf(dz[d], w4[d * kC + c + h], dy);
                                        acc[d * kC + c + h] = fmaf(y3[c + h], dz[d], acc[d * kC + c + h]);
                                    }
                                    g2[h] = y3[c + h] > 0.0f ? dy : 0.0f;
                                }
                                pk[c / 2] = pack2(g2[0], g2[1]);
                            }
                            uint8_t* dst = a.out + row_off;
                            *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        }
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce_bar(s));
            }
        }
        if (kMode == kTcHeadTrain) {
            // the warp's sums, then one atomic per value and warp
#pragma unroll
            for (int i = 0; i < kAcc; ++i) {
                float x = acc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0 && x != 0.0f) {
                    float* dst = i < 3 * kC ? a.grad_w4 + i : (i < 3 * kC + 3 ? a.grad_b4 + (i - 3 * kC) : a.loss);
                    atomicAdd(dst, x);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kIssuerWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// First layer's input: [site][sample][8] BF16, channels s_{t-1}(n) then s_t(n)
// for n = 0..2, then two zeros.  Rows past n_samples are zero.  One warp per
// site and 256 samples (4 words): lanes 0..23 load the 6 channels x 4 words,
// and store j of the warp writes samples 32j .. 32j + 31 (512 contiguous bytes).
__global__ void k_expand_bits(int L3, int64_t Sp, int64_t W, int64_t words, const uint64_t* __restrict__ s_prev,
                              const uint64_t* __restrict__ s_cur, uint4* __restrict__ out)
{
    const int64_t site = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * 256;
    if (site >= L3) return;
    uint64_t v = 0;
    if (lane < 24) {
        const int c = lane >> 2;
        const int64_t w = (m0 >> 6) + (lane & 3);
        if (w < words) {
            const uint64_t* src = c < 3 ? s_prev : s_cur;
            v = __ldg(&src[((int64_t)(c % 3) * L3 + site) * W + w]);
        }
    }
    constexpr uint32_t one = 0x3F80u;   // BF16 1.0
    // tile-major layout: samples m0 .. m0 + 127 in tile m0 / 128 of the site, the next 128 in
    // the next tile (L3 tiles further)
    uint4* dst = out + ((m0 >> 7) * L3 + site) * kTileM + lane;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (m0 + 32 * j >= Sp) break;
        const uint32_t half = (uint32_t)(v >> (32 * (j & 1)));
        uint32_t h[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) h[c] = ((__shfl_sync(0xffffffffu, half, c * 4 + (j >> 1)) >> lane) & 1u) * one;
        dst[(j >> 2) * (int64_t)L3 * kTileM + 32 * (j & 3)] =
            make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), 0u);
    }
}

// ------------------------------------------------------------------ weight gradients
// Weight and bias gradients of one convolution as a GEMM over samples:
//   G[(k, ci)][co] = sum over sites r and samples s of x[r + off_k][s][ci] . d[r][s][co],
// M = 128 rows (8 offsets x 16 input channels; the first layer 16 x 8), N = 16 output
// channels, K = 16 samples per MMA.  The reduction runs over samples, so both operands are
// channel-major copies of the tiles (k_channel_major): a tile of C channels x 128 samples is
// [C/8][sample/8][8 channels][8 samples] BF16, K-major core matrices with LBO 128 B (the next
// 8 samples) and SBO 2048 B (the next 8 channels -- also the step to the next tile of an M
// group, so the 8 (16) neighbour tiles of a group sit at a uniform stride).  The 28th
// "offset" is a tile of ones: its rows give the bias gradient sum d[r][s][co].  Work item:
// one (128-sample tile, site); per item the d tile and, per M group, its neighbour tiles are
// copied into rings of slots, and the group's accumulator in TMEM (16 columns) takes 8 MMAs.
// The accumulators live for the whole launch and are added to the gradients at the end.
// Rows beyond offset 27 multiply whatever the slot holds and are never read.
constexpr int kWgX = 6;                       // group slots, 32 KiB each
constexpr int kWgD = 4;                       // d-tile slots, 4 KiB each
constexpr int kWgOffD = kWgX * 32768;
constexpr int kWgOffBar = kWgOffD + kWgD * 4096;
constexpr int kWgNumBars = 2 * kWgX + 2 * kWgD + 1;   // x full, x empty, d full, d empty, done
constexpr int kWgOffMisc = kWgOffBar + kWgNumBars * 8;
constexpr int kWgSmemBytes = kWgOffMisc + 16 + 1024;
static_assert(kWgSmemBytes <= 227 * 1024, "shared memory budget");

struct WgArgs {
    int L, L3;
    int64_t n_items;            // 128-sample tiles x L^3 sites
    const uint8_t* xt;          // channel-major x tiles (kCin channels)
    const uint8_t* dt;          // channel-major d tiles (16 channels)
    const uint8_t* ones;        // one x tile of BF16 ones
    int cin;                    // input channels kept in gw (6 for the first layer)
    float* gw;                  // [co][cin][27], accumulated
    float* gb;                  // [16], accumulated
};

// Site r + offset k (k = (dz + 1) 9 + (dy + 1) 3 + (dx + 1)), periodic.
__device__ __forceinline__ int64_t wg_neighbour(int r, int k, int L)
{
    const int x = r % L, y = (r / L) % L, z = r / (L * L);
    const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
    return ((int64_t)wrap(z + dz, L) * L + wrap(y + dy, L)) * L + wrap(x + dx, L);
}

template <int kCin>
__global__ void __launch_bounds__(kTcThreads, 1) k_wgrad_tc(const __grid_constant__ WgArgs a)
{
    constexpr uint32_t kTileB = kCin * 256;
    constexpr int kPer = 128 / kCin;                         // offsets per M group
    constexpr int kGroups = (kOff + 1 + kPer - 1) / kPer;    // 4, or 2 for the first layer
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t base = smem_u32(sm);
    const uint32_t bars = base + kWgOffBar;
    auto xfull = [&](int i) { return bars + 8u * (uint32_t)i; };
    auto xempty = [&](int i) { return bars + 8u * (uint32_t)(kWgX + i); };
    auto dfull = [&](int i) { return bars + 8u * (uint32_t)(2 * kWgX + i); };
    auto dempty = [&](int i) { return bars + 8u * (uint32_t)(2 * kWgX + kWgD + i); };
    const uint32_t done_bar = bars + 8u * (uint32_t)(2 * kWgX + 2 * kWgD);
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + kWgOffMisc);   // [0] TMEM base, [1] abort, [2] progress
    volatile uint32_t* abort_flag = misc + 1;
    volatile uint32_t* progress = misc + 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        misc[2] = 0;
        for (int i = 0; i < kWgX; ++i) {
            mbar_init(xfull(i), 1);
            mbar_init(xempty(i), 1);
        }
        for (int i = 0; i < kWgD; ++i) {
            mbar_init(dfull(i), 1);
            mbar_init(dempty(i), 1);
        }
        mbar_init(done_bar, 1);
        misc[1] = 0;
        fence_mbar_init();
    }
    if (warp == kIssuerWarp) tmem_alloc(smem_u32(misc), 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    const int L = a.L;

    if (warp == kProducerWarp) {
        uint32_t xs = 0, ds = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.n_items && ok; u += gridDim.x) {
            const int64_t t = u / a.L3;
            const int r = (int)(u - t * a.L3);
            {
                const int g = (int)(ds % kWgD);
                const uint32_t use = ds / kWgD;
                int good = 1;
                if (lane == 0 && use > 0) good = wait_bar(dempty(g), (use - 1) & 1u, abort_flag) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, good, 0)) break;
                if (lane == 0) {
                    mbar_arrive_expect_tx(dfull(g), 4096u);
                    bulk_load(base + kWgOffD + (uint32_t)g * 4096u, a.dt + (t * a.L3 + r) * 4096, 4096u, dfull(g));
                }
                ++ds;
            }
            for (int grp = 0; grp < kGroups; ++grp) {
                const int g = (int)(xs % kWgX);
                const uint32_t use = xs / kWgX;
                int good = 1;
                if (lane == 0 && use > 0) good = wait_bar(xempty(g), (use - 1) & 1u, abort_flag) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, good, 0)) {
                    ok = false;
                    break;
                }
                const int k0 = grp * kPer;
                const int n_real = min(kPer, kOff + 1 - k0);     // offsets and the ones tile
                if (lane == 0) mbar_arrive_expect_tx(xfull(g), (uint32_t)n_real * kTileB);
                __syncwarp();
                if (lane < n_real) {
                    const int k = k0 + lane;
                    const uint8_t* src = k < kOff ? a.xt + (t * a.L3 + wg_neighbour(r, k, L)) * kTileB : a.ones;
                    bulk_load(base + (uint32_t)g * 32768u + (uint32_t)lane * kTileB, src, kTileB, xfull(g));
                }
                ++xs;
            }
        }
        // copies still in flight land before the CTA exits
        if (lane == 0) {
            const uint32_t lx = xs < (uint32_t)kWgX ? xs : (uint32_t)kWgX;
            for (uint32_t g = 0; g < lx; ++g) {
                const uint32_t q = xs - 1 - ((xs - 1 - g) % kWgX);
                wait_bar(xfull((int)g), (q / kWgX) & 1u, abort_flag, true);
            }
            const uint32_t ld = ds < (uint32_t)kWgD ? ds : (uint32_t)kWgD;
            for (uint32_t g = 0; g < ld; ++g) {
                const uint32_t q = ds - 1 - ((ds - 1 - g) % kWgD);
                wait_bar(dfull((int)g), (q / kWgD) & 1u, abort_flag, true);
            }
        }
        __syncwarp();
    } else if (warp == kIssuerWarp) {
        if (lane == 0) {
            constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                                        ((uint32_t)(kTileM >> 4) << 24);
            uint32_t xs = 0, ds = 0;
            bool ok = true, first = true;
            for (int64_t u = blockIdx.x; u < a.n_items && ok; u += gridDim.x) {
                const int gd = (int)(ds % kWgD);
                if (!wait_bar(dfull(gd), (ds / kWgD) & 1u, abort_flag)) break;
                tc_fence_after();
                const uint64_t bdesc = smem_desc(base + kWgOffD + (uint32_t)gd * 4096u, 128u, 2048u);
                for (int grp = 0; grp < kGroups; ++grp) {
                    const int g = (int)(xs % kWgX);
                    if (!wait_bar(xfull(g), (xs / kWgX) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc = smem_desc(base + (uint32_t)g * 32768u, 128u, 2048u);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        // 16 samples per step: two core matrices (256 B) further along K
                        const uint64_t step = (uint64_t)((kk * 256) >> 4);
                        if (first && kk == 0)
                            mma_bf16_overwrite(tmem + (uint32_t)(grp * 16), adesc + step, bdesc + step, kIdesc);
                        else
                            mma_bf16_n(tmem + (uint32_t)(grp * 16), adesc + step, bdesc + step, kIdesc);
                    }
                    mma_commit(xempty(g));
                    ++xs;
                }
                first = false;
                mma_commit(dempty(gd));
                ++ds;
                *progress = ds;
            }
            mma_commit(done_bar);
            wait_bar(done_bar, 0, abort_flag, true);
        }
        __syncwarp();
    } else if (warp < kEpiWarps) {
        // every MMA has completed: add the accumulators to the gradients; TMEM lane = M row
        int got = 1;
        if (lane == 0) got = wait_bar_progress(done_bar, progress, abort_flag) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        tc_fence_after();
        if (got && !*abort_flag) {
            const int row = warp * 32 + lane;
#pragma unroll
            for (int grp = 0; grp < kGroups; ++grp) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(grp * 16), v);
                tmem_wait_ld();
                const int k = grp * kPer + row / kCin, ci = row % kCin;
                if (k < kOff && ci < a.cin) {
#pragma unroll
                    for (int co = 0; co < 16; ++co)
                        atomicAdd(&a.gw[(co * a.cin + ci) * kOff + k], __uint_as_float(v[co]));
                } else if (k == kOff && ci == 0) {
#pragma unroll
                    for (int co = 0; co < 16; ++co) atomicAdd(&a.gb[co], __uint_as_float(v[co]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kIssuerWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
}

// Channel-major copy of C-channel tiles (k_wgrad_tc's operands): the element (sample m,
// channel c) of a tile moves from the tile-major place ([m/8][c/8][8][8] for 16 channels,
// [m][8] for 8) to [c/8][m/8][8 channels][8 samples].  One block per tile.
template <int kCh>
__global__ void __launch_bounds__(256) k_channel_major(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst)
{
    constexpr int kN = kCh * 128;
    __shared__ uint16_t tile[kN];
    const int64_t t = blockIdx.x;
    for (int i = threadIdx.x; i < kN / 8; i += blockDim.x)
        reinterpret_cast<uint4*>(tile)[i] = reinterpret_cast<const uint4*>(src + t * kN)[i];
    __syncthreads();
    for (int i = threadIdx.x; i < kN; i += blockDim.x) {
        // destination index i = ((c/8) 16 + m/8) 64 + (c%8) 8 + m%8
        const int ms = i & 7, cs = (i >> 3) & 7, mg = (i >> 6) & 15, cg = i >> 10;
        const int m = mg * 8 + ms, c = cg * 8 + cs;
        const int from = kCh == 16 ? ((m >> 3) * 2 + (c >> 3)) * 64 + (m & 7) * 8 + (c & 7) : m * 8 + c;
        dst[t * kN + i] = tile[from];
    }
}

__global__ void k_fill_ones(uint16_t* __restrict__ p, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0x3F80u;   // BF16 1.0
}

int64_t tc_padded(int64_t n) { return (n + kTileM - 1) / kTileM * kTileM; }
size_t r256(size_t x) { return (x + 255) / 256 * 256; }

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int kMode, bool kBitsIn>
t3d_status launch_conv_col(const TcArgs& a, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>(a.n_units, sm_count());
    ProfScope prof(T3D_K_CNN, st);
    k_conv_col<kMode, kBitsIn><<<grid, kTcThreads, kColSmemBytes, st>>>(a);
    T3D_LAUNCH_CHECK("tensor-core convolution");
    return T3D_OK;
}

// Arguments shared by every convolution of a pass over n_samples samples.
TcArgs base_args(int L, int64_t n_samples, int64_t W)
{
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    const int64_t Sp = tc_padded(n_samples);
    a.L = L;
    a.L3 = L * L * L;
    a.Sp = Sp;
    a.n_samples = n_samples;
    a.W = W;
    a.words = words_for(n_samples);
    a.ncx = (L + 1) / 2;
    a.n_units = (Sp / kTileM) * a.ncx * a.ncx;
    return a;
}

t3d_status expand_bits(const TcArgs& a, const uint64_t* s_prev, const uint64_t* s, uint8_t* x0, cudaStream_t st)
{
    ProfScope prof(T3D_K_CNN, st);
    const dim3 grid((unsigned)((a.L3 + 7) / 8), (unsigned)((a.Sp + 255) / 256));
    k_expand_bits<<<grid, 256, 0, st>>>(a.L3, a.Sp, a.W, a.words, s_prev, s, reinterpret_cast<uint4*>(x0));
    T3D_LAUNCH_CHECK("pre-decoder input expansion");
    return T3D_OK;
}

}  // namespace

t3d_status tc_prepare()
{
    static std::mutex mu;
    static bool configured[64] = {};
    int dev = 0;
    T3D_CUDA_CHECK(cudaGetDevice(&dev));
    T3D_REQUIRE(dev >= 0 && dev < 64, "device %d outside the 64 supported", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!configured[dev]) {
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<kTcRelu, true>, attr, kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<kTcRelu, false>, attr, kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<kTcHead, false>, attr, kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<kTcHeadTrain, false>, attr, kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<kTcMask, false>, attr, kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_wgrad_tc<8>, attr, kWgSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_wgrad_tc<kC>, attr, kWgSmemBytes));
        configured[dev] = true;
    }
    return T3D_OK;
}

size_t tc_act_bytes(int L, int64_t n_samples, int channels)
{
    return r256((size_t)L * L * L * (size_t)tc_padded(n_samples) * 2 * (size_t)channels);
}

size_t tc_workspace_bytes(int L, int64_t n_samples)
{
    return tc_act_bytes(L, n_samples, 8) + 2 * tc_act_bytes(L, n_samples, kC);
}

t3d_status launch_forward_tc(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, const uint64_t* s,
                             uint64_t* dec, const Blob* blob, float* logits_out, void* work, cudaStream_t st)
{
    uint8_t* in0 = static_cast<uint8_t*>(work);
    uint8_t* act0 = in0 + tc_act_bytes(L, n_samples, 8);
    uint8_t* act1 = act0 + tc_act_bytes(L, n_samples, kC);
    T3D_TRY(tc_prepare());
    TcArgs a = base_args(L, n_samples, W);
    T3D_TRY(expand_bits(a, s_prev, s, in0, st));
    a.in = in0;
    a.out = act0;
    a.w = &blob->wf[0][0][0][0];
    a.bias = blob->bias[0];
    T3D_TRY((launch_conv_col<kTcRelu, true>(a, st)));
    a.in = act0;
    a.out = act1;
    a.w = &blob->wf[1][0][0][0];
    a.bias = blob->bias[1];
    T3D_TRY((launch_conv_col<kTcRelu, false>(a, st)));
    a.in = act1;
    a.out = nullptr;
    a.w = &blob->wf[2][0][0][0];
    a.bias = blob->bias[2];
    a.w4 = &blob->w4[0][0];
    a.b4 = blob->b4;
    a.dec32 = reinterpret_cast<uint32_t*>(dec);
    a.logits = logits_out;
    T3D_TRY((launch_conv_col<kTcHead, false>(a, st)));
    return T3D_OK;
}

t3d_status tc_train_forward(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, const uint64_t* s,
                            const uint64_t* label, const Blob* blob, uint8_t* x0, uint8_t* y1, uint8_t* y2,
                            uint8_t* g3, float* grad_w4, float* grad_b4, float* loss, cudaStream_t st)
{
    T3D_TRY(tc_prepare());
    TcArgs a = base_args(L, n_samples, W);
    T3D_TRY(expand_bits(a, s_prev, s, x0, st));
    a.in = x0;
    a.out = y1;
    a.w = &blob->wf[0][0][0][0];
    a.bias = blob->bias[0];
    T3D_TRY((launch_conv_col<kTcRelu, true>(a, st)));
    a.in = y1;
    a.out = y2;
    a.w = &blob->wf[1][0][0][0];
    a.bias = blob->bias[1];
    T3D_TRY((launch_conv_col<kTcRelu, false>(a, st)));
    a.in = y2;
    a.out = g3;
    a.w = &blob->wf[2][0][0][0];
    a.bias = blob->bias[2];
    a.w4 = &blob->w4[0][0];
    a.b4 = blob->b4;
    a.label = label;
    a.inv_n = 1.0f / (3.0f * (float)a.L3 * (float)n_samples);
    a.grad_w4 = grad_w4;
    a.grad_b4 = grad_b4;
    a.loss = loss;
    T3D_TRY((launch_conv_col<kTcHeadTrain, false>(a, st)));
    return T3D_OK;
}

t3d_status tc_backward_data(int L, int64_t n_samples, const __nv_bfloat16* wt, const uint8_t* g_in,
                            const uint8_t* mask_act, uint8_t* g_out, cudaStream_t st)
{
    T3D_TRY(tc_prepare());
    TcArgs a = base_args(L, n_samples, words_for(n_samples));
    a.in = g_in;
    a.out = g_out;
    a.w = wt;
    a.mask_act = mask_act;
    return launch_conv_col<kTcMask, false>(a, st);
}

t3d_status tc_fill_ones(uint8_t* tile, cudaStream_t st)
{
    k_fill_ones<<<(2048 + 255) / 256, 256, 0, st>>>(reinterpret_cast<uint16_t*>(tile), 2048);
    T3D_LAUNCH_CHECK("ones tile");
    return T3D_OK;
}

t3d_status tc_weight_grad(int L, int64_t n_samples, int x_ch, int cin_kept, const uint8_t* x, const uint8_t* d,
                          uint8_t* xt, uint8_t* dt, const uint8_t* ones, float* gw, float* gb, cudaStream_t st)
{
    T3D_REQUIRE(x_ch == 8 || x_ch == kC, "weight gradient: %d input channels", x_ch);
    T3D_TRY(tc_prepare());
    const int64_t L3 = (int64_t)L * L * L, n_items = tc_padded(n_samples) / kTileM * L3;
    T3D_REQUIRE(n_items <= 0x7fffffffLL, "weight gradient: %lld (sample tile, site) pairs exceed one grid",
                (long long)n_items);
    ProfScope prof(T3D_K_CNN, st);
    if (x_ch == 8)
        k_channel_major<8><<<(unsigned)n_items, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(x),
                                                              reinterpret_cast<uint16_t*>(xt));
    else
        k_channel_major<kC><<<(unsigned)n_items, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(x),
                                                               reinterpret_cast<uint16_t*>(xt));
    k_channel_major<kC><<<(unsigned)n_items, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(d),
                                                           reinterpret_cast<uint16_t*>(dt));
    T3D_LAUNCH_CHECK("channel-major tiles");
    WgArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = L;
    a.L3 = (int)L3;
    a.n_items = n_items;
    a.xt = xt;
    a.dt = dt;
    a.ones = ones;
    a.cin = cin_kept;
    a.gw = gw;
    a.gb = gb;
    const int grid = (int)std::min<int64_t>(n_items, sm_count());
    if (x_ch == 8)
        k_wgrad_tc<8><<<grid, kTcThreads, kWgSmemBytes, st>>>(a);
    else
        k_wgrad_tc<kC><<<grid, kTcThreads, kWgSmemBytes, st>>>(a);
    T3D_LAUNCH_CHECK("tensor-core weight gradient");
    return T3D_OK;
}

t3d_status tc_set_wait_limit(uint64_t ns)
{
    const unsigned long long v = ns ? (unsigned long long)ns : (unsigned long long)kWaitNs;
    T3D_REQUIRE(v <= kWaitNs, "the wait limit cannot exceed %llu ns", (unsigned long long)kWaitNs);
    T3D_CUDA_CHECK(cudaDeviceSynchronize());
    T3D_CUDA_CHECK(cudaMemcpyToSymbol(g_tc_wait_ns, &v, sizeof(v)));
    return T3D_OK;
}

t3d_status tc_status()
{
    unsigned int flag = 0, zero = 0;
    T3D_CUDA_CHECK(cudaDeviceSynchronize());
    T3D_CUDA_CHECK(cudaMemcpyFromSymbol(&flag, g_tc_error, sizeof(flag)));
    if (flag) {
        T3D_CUDA_CHECK(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(zero)));
        set_error("a tensor-core pre-decoder kernel gave up a bounded wait");
        return T3D_ETIMEOUT;
    }
    return T3D_OK;
}

}  // namespace cnn
}  // namespace t3d
