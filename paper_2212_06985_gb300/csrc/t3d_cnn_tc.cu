// Inference forward pass of the learned pre-decoder on the fifth-generation
// tensor cores (tcgen05 MMA with TMEM accumulators, operands staged in shared
// memory by bulk asynchronous copies).
//
// A 3x3x3 convolution with 16 output channels has a small GEMM N (16), and a
// tcgen05.mma with M = 128, K = 16 takes as long for N = 16 as for N = 128
// (measured on GB300: about 53 cycles from one issuing thread at N = 16, 64 at
// N = 128, 128 at N = 256, the last two at the tensor peak).  So every MMA here
// computes 8 output sites at once:
//   D[sample][(r, co)] += A_i[sample][ci] . B[(r, co)][ci],   M = N = 128, K = 16,
// where A_i is the 128-sample activation tile of one input site i, the 128
// columns of D are 8 consecutive output sites along x (r = 7 - (x - x0)) times 16
// channels, and B stacks, for each of the 8 outputs, the weights of the offset
// that connects it to i (zero where i is not its neighbour).  For a fixed
// (dy, dz) these stacks are strided views of one zero-padded strip of weight
// blocks [0 x 7, W(dx=-1), W(0), W(+1), 0 x 7]: the view for input offset
// a = x_i - x0 starts a blocks further along the strip.  Nine strips (one per
// (dy, dz), sharing their zero padding) take 97 blocks of 512 bytes.
//
// Work unit: one 128-sample tile x one line of 8 output sites (x0..x0+7, y)
// running through all L planes in z.  The CTA streams the unit's input tiles
// plane by plane (input planes z = -1 .. L, each with the 10 x 3 sites
// (x0-1..x0+8, y-1..y+1) around the line, periodic wrap); each input tile is
// loaded into shared memory once and multiplied into the (up to) three output
// planes z-1, z, z+1 it touches, one MMA each.  TMEM holds the accumulators of
// four output planes (4 x 128 columns): while input plane z is multiplied,
// outputs z-1, z, z+1 accumulate and the epilogue drains plane z-2.
//
// Warp roles (192 threads, one CTA per SM):
//   warps 0-3  epilogue: tcgen05.ld of a finished plane (warp w reads TMEM lanes
//              32w..32w+31 = samples), bias + ReLU + BF16 store of the next
//              layer's input, or for the last layer the 16 -> 3 head and the
//              hard decisions;
//   warp 4     producer: one thread issues the bulk copies of input tiles into
//              a ring of shared-memory slots;
//   warp 5     MMA issuer: one thread issues the MMAs and commits their
//              completion to the row's "empty" barrier and to the plane's
//              "accumulators full" barrier (the code takes kIssuers threads
//              owning alternate planes; two were slower than one on GB300).
// Every wait is bounded (one second; toric3d_cnn_debug_wait_limit shortens the
// waits that may give up, so a test can make them run out); a wait that gives
// up sets the device error flag and the CTA winds down (waiting, again bounded
// but always by the full second, for its copies and MMAs in flight, and
// freeing its TMEM) so the context stays usable.
//
// Shared-memory operand layout ("no swizzle", K-major): core matrices of 8 rows
// x 16 bytes stored contiguously.  Hidden activations in global memory use the
// same layout, [site][sample/8][channel/8][8 samples][8 channels] BF16, so a
// tile (site, 128 samples) is one contiguous 4 KiB block: K-direction core
// matrix stride (LBO) 128 B, M-direction stride (SBO) 256 B.  The first
// layer's input (6 of 8 channels used) is stored as [site][sample][8]
// (2 KiB per tile, SBO 128 B); two x-adjacent sites fill one 4 KiB slot as the
// two K chunks of one operand (LBO 2 KiB), see pair_start.  Weight blocks:
// [co/8][ci/8][co%8][ci%8] (512 B, LBO 128 B, SBO 256 B).
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
constexpr int kLine = 8;                            // output sites per MMA (N = 8 x 16)
constexpr int kN = kLine * kC;                      // 128
constexpr int kPlanes = 4;                          // output planes resident in TMEM
constexpr uint32_t kTmemCols = kPlanes * kN;        // 512
constexpr int kRowSlots = kLine + 2;                // input tiles of one row (x0-1 .. x0+8)
constexpr int kGroups = 4;                          // rows in flight; each row has one full / empty barrier
constexpr int kRing = kRowSlots * kGroups;          // 40 shared-memory input slots
constexpr int kSlotBytes = 4096;
constexpr int kStripPad = 7;                        // zero blocks between strips
constexpr int kStripBlocks = kStripPad + 9 * (3 + kStripPad);   // 97
constexpr int kWBytes = kStripBlocks * 512;         // 49,664 B
constexpr int kEpiWarps = 4;
constexpr int kEpiBatch = 4;                        // TMEM loads in flight per epilogue thread
constexpr int kProducerWarp = 4;
constexpr int kIssuerWarp = 5;                      // .. kIssuerWarp + kIssuers - 1
constexpr int kIssuers = 1;                         // two issuers measured slower on GB300
constexpr int kTcThreads = 32 * (kIssuerWarp + kIssuers);
constexpr uint64_t kWaitNs = 1000000000ull;         // bound of every wait

// Dynamic shared memory: ring | weight strips | barriers | misc.
constexpr int kOffW = kRing * kSlotBytes;
constexpr int kOffBar = kOffW + kWBytes;
constexpr int kNumBars = 2 * kGroups + 2 * kPlanes + kIssuers;   // full, empty, acc_full, acc_empty, done
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;        // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

// Block index of W(dx = -1, dy, dz) in the strips; s = (dz + 1) * 3 + (dy + 1).
__host__ __device__ constexpr int strip_start(int s) { return kStripPad + s * (3 + kStripPad); }

// First layer (8 input channels per site): two x-adjacent input sites share
// one K = 16 tile (K chunk 0 = site x, chunk 1 = site x + 1), and the pair
// strip of (dy, dz) holds blocks [W(t) | W(t + 1)] for first-site offsets
// t = -2 .. 1 (W = 0 outside -1..1) between 6 zero blocks; the view for the
// pair starting at input offset xa begins at pair_start(s) + xa - 5.
constexpr int kPairPad = 6;
__host__ __device__ constexpr int pair_start(int s) { return kPairPad + s * (4 + kPairPad); }
static_assert(kPairPad + 9 * (4 + kPairPad) <= kStripBlocks, "pair strips fit the strip area");

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ unsigned int g_tc_error;   // bit 0: a bounded wait gave up
// bound of the waits that may give up (the wind-down drains always use kWaitNs)
__device__ unsigned long long g_tc_wait_ns = kWaitNs;

struct TcArgs {
    int L, L3;
    int64_t Sp;                 // padded samples of the activation buffers (multiple of 128)
    int64_t n_samples;
    int64_t W;                  // row stride of the bit-sliced arrays (words)
    int64_t words;              // words of this pass
    int nbx;                    // line kernel: lines of 8 sites along x
    int ncx;                    // column kernel: 2 x 2 columns per axis (ceil(L / 2))
    int64_t n_units;
    const uint8_t* in;          // input activations
    uint8_t* out;               // hidden layers: output activations
    const __nv_bfloat16* w;     // [27][co][ci]
    const float* bias;          // [16]
    const float* w4;            // head [3][16]
    const float* b4;            // [3]
    uint32_t* dec32;            // head: decision words [word][site][8] 32-bit halves
    float* logits;              // head: optional [3][L^3][n_samples]
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

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Bring a global range toward the L2 ahead of its bulk copy (no completion to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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

// D (+)= A . B^T; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred pa;\n"
        "setp.ne.b32 pa, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n"
        "}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// The same with an instruction descriptor chosen per MMA (N varies).
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
    int x0, y;       // line origin
    int fx;          // line length (clipped at the lattice edge)
};

__device__ __forceinline__ Unit unit_of(const TcArgs& a, int64_t u)
{
    const int64_t lines = (int64_t)a.nbx * a.L;
    const int64_t tile = u / lines;
    const int rem = (int)(u - tile * lines);
    Unit t;
    t.m0 = tile * kTileM;
    t.y = rem / a.nbx;
    t.x0 = (rem % a.nbx) * kLine;
    t.fx = min(kLine, a.L - t.x0);
    return t;
}

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
// for the smallest lattices).  prefetch: bring them to the L2 instead.
__device__ __forceinline__ void copy_row(uint32_t dst, const uint8_t* in, int64_t row, int x0, int n, int L, int L3,
                                         int64_t m0, uint32_t tile_bytes, uint32_t bar, bool prefetch)
{
    int i = 0;
    while (i < n) {
        const int x = wrap(x0 + i, L);
        int k = 1;
        while (i + k < n && x + k < L && wrap(x0 + i + k, L) == x + k) ++k;
        const uint8_t* src = in + tile_off(row + x, m0, L3, tile_bytes);
        if (prefetch)
            bulk_prefetch_l2(src, (uint32_t)k * tile_bytes);
        else
            bulk_load(dst + (uint32_t)i * tile_bytes, src, (uint32_t)k * tile_bytes, bar);
        i += k;
    }
}

// ------------------------------------------------------------------ kernel
template <bool kHead, bool kBitsIn>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t ring = smem_u32(sm);
    const uint32_t wsm = ring + kOffW;
    const uint32_t bars = ring + kOffBar;
    auto full_bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    auto empty_bar = [&](int i) { return bars + 8u * (uint32_t)(kGroups + i); };
    auto accf_bar = [&](int i) { return bars + 8u * (uint32_t)(2 * kGroups + i); };
    auto acce_bar = [&](int i) { return bars + 8u * (uint32_t)(2 * kGroups + kPlanes + i); };
    auto done_bar = [&](int i) { return bars + 8u * (uint32_t)(2 * kGroups + 2 * kPlanes + i); };
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + kOffMisc);   // [0] TMEM base, [1] abort flag
    volatile uint32_t* abort_flag = misc + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // weight strips: zero everything, then W(dx, dy, dz) at block strip_start(s) + dx + 1 in the
    // B-operand layout [co/8][ci/8][co%8][ci%8]; first layer: the pair strips
    for (int i = threadIdx.x; i < kWBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm + kOffW)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < kOff * kC * kC; i += blockDim.x) {
        const int k = i >> 8, co = (i >> 4) & 15, ci = i & 15;
        const int st = k / 3, dx = k % 3 - 1;   // st = (dz + 1) * 3 + (dy + 1)
        const __nv_bfloat16 w = a.w[i];
        const int row = (co >> 3) * 256 + (co & 7) * 16;
        if (kBitsIn) {
            if (ci >= 8) continue;   // no such input channel
            // chunk 0 of the block with t = dx, chunk 1 of the block with t = dx - 1
            *reinterpret_cast<__nv_bfloat16*>(sm + kOffW + (pair_start(st) + dx + 2) * 512 + row + ci * 2) = w;
            *reinterpret_cast<__nv_bfloat16*>(sm + kOffW + (pair_start(st) + dx + 1) * 512 + row + 128 + ci * 2) = w;
        } else {
            const int off = (strip_start(st) + dx + 1) * 512 + row + (ci >> 3) * 128 + (ci & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(sm + kOffW + off) = w;
        }
    }
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        for (int i = 0; i < kGroups; ++i) {
            mbar_init(full_bar(i), 1);
            mbar_init(empty_bar(i), kIssuers);   // one commit per issuer
        }
        for (int i = 0; i < kPlanes; ++i) {
            mbar_init(accf_bar(i), 1);
            mbar_init(acce_bar(i), kEpiWarps);
        }
        for (int i = 0; i < kIssuers; ++i) mbar_init(done_bar(i), 1);
        misc[1] = 0;
        fence_mbar_init();
    }
    if (warp == kIssuerWarp) tmem_alloc(smem_u32(misc), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];

    const int L = a.L;
    const uint32_t in_row = kBitsIn ? 16u : 32u;
    const uint32_t tile_bytes = kTileM * in_row;

    if (warp == kProducerWarp) {
        // one row (fixed input y and z, x = x0-1 .. x0+fx) per slot group, one barrier phase each,
        // copied in runs of x-adjacent tiles (contiguous in the tile-major layout)
        uint32_t gseq = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit t = unit_of(a, u);
            for (int zi = -1; zi <= L && ok; ++zi) {
                const int zw = wrap(zi, L);
                for (int yi = t.y - 1; yi <= t.y + 1; ++yi) {
                    const int g = (int)(gseq % kGroups);
                    const uint32_t use = gseq / kGroups;
                    int good = 1;
                    if (lane == 0 && use > 0) good = wait_bar(empty_bar(g), (use - 1) & 1u, abort_flag) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, good, 0)) {
                        ok = false;
                        break;
                    }
                    const int64_t row = ((int64_t)zw * L + wrap(yi, L)) * L;
                    const int n_tiles = kBitsIn ? 2 * ((t.fx + 3) / 2) : t.fx + 2;
                    if (lane == 0) {
                        // the row's tiles land tile_bytes apart in the slot group, in runs of
                        // consecutive sites
                        mbar_arrive_expect_tx(full_bar(g), (uint32_t)n_tiles * tile_bytes);
                        copy_row(ring + (uint32_t)(g * kRowSlots) * kSlotBytes, a.in, row, t.x0 - 1, n_tiles, L, a.L3,
                                 t.m0, tile_bytes, full_bar(g), false);
                    }
                    ++gseq;
                }
            }
        }
        // copies still in flight land before the CTA exits
        if (lane == 0) {
            const uint32_t last = gseq < (uint32_t)kGroups ? gseq : (uint32_t)kGroups;
            for (uint32_t g = 0; g < last; ++g) {
                // the latest row issued on this group: the largest q < gseq with q % kGroups == g
                const uint32_t q = gseq - 1 - ((gseq - 1 - g) % kGroups);
                wait_bar(full_bar((int)g), (q / kGroups) & 1u, abort_flag, true);
            }
        }
        __syncwarp();
    } else if (warp >= kIssuerWarp && warp < kIssuerWarp + kIssuers) {
        // issuer iss owns the output planes with sequence number q = iss (mod kIssuers): every
        // accumulator is written by one thread, in program order
        const int iss = warp - kIssuerWarp;
        if (lane == 0) {
            uint32_t gseq = 0;
            int64_t qbase = 0;
            bool ok = true;
            // first layer: K chunk 1 is the pair's second site, 2 KiB further
            const uint32_t a_lbo = kBitsIn ? 2048u : 128u, a_sbo = kBitsIn ? 128u : 256u;
            const uint64_t bdesc0 = smem_desc(wsm, 128u, 256u);   // + 32 per 512-byte block
            for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
                const Unit t = unit_of(a, u);
                const bool full = t.fx == kLine;
                for (int zi = -1; zi <= L && ok; ++zi) {
                    // output plane zi + 1 is first written by this input plane
                    if (zi + 1 <= L - 1 && (int)((qbase + zi + 1) % kIssuers) == iss) {
                        const int64_t q = qbase + zi + 1;
                        const uint32_t v = (uint32_t)(q >> 2);
                        if (v > 0 && !wait_bar(acce_bar((int)(q & 3)), (v - 1) & 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    // TMEM column of output plane zi - dz (i = dz + 1), or -1 outside [0, L)
                    int colb[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const int zo = zi - (i - 1);
                        colb[i] = (zo >= 0 && zo < L && (int)((qbase + zo) % kIssuers) == iss)
                                      ? (int)((qbase + zo) & 3) * kN
                                      : -1;
                    }
                    // one tile: input offset xa = x_i - x0 in [-1, 8], dy; the MMA into plane
                    // zi + 1 from the plane's first tile (xa = -1, dy = -1) overwrites D.
                    auto tile_mmas = [&](int xa, int dyi, uint64_t adesc) {
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            if (colb[i] < 0) continue;
                            const int blk = strip_start(i * 3 + dyi) + xa - 6;
                            const uint32_t acc = (i == 0 && dyi == 0 && xa == -1) ? 0u : 1u;
                            mma_bf16(tmem + (uint32_t)colb[i], adesc, bdesc0 + (uint64_t)(32 * blk), acc);
                        }
                    };
                    // the three rows of the plane, each one slot group behind one barrier
                    auto row_mmas = [&](int dyi) {
                        const int g = (int)(gseq % kGroups);
                        // the copies and the MMAs meet through the barrier (both in the async proxy)
                        if (ok && !wait_bar(full_bar(g), (gseq / kGroups) & 1u, abort_flag)) ok = false;
                        if (!ok) return;
                        const uint64_t adesc0 =
                            smem_desc(ring + (uint32_t)(g * kRowSlots) * kSlotBytes, a_lbo, a_sbo);
                        if (kBitsIn) {
                            // pair p: sites x0-1+2p, x0+2p (4 KiB slot p); view pair_start + xa - 5
                            auto pair_mmas = [&](int p) {
                                const int xa = 2 * p - 1;
#pragma unroll
                                for (int i = 0; i < 3; ++i) {
                                    if (colb[i] < 0) continue;
                                    const int blk = pair_start(i * 3 + dyi) + xa - 5;
                                    const uint32_t acc = (i == 0 && dyi == 0 && p == 0) ? 0u : 1u;
                                    mma_bf16(tmem + (uint32_t)colb[i], adesc0 + (uint64_t)(p * (kSlotBytes >> 4)),
                                             bdesc0 + (uint64_t)(32 * blk), acc);
                                }
                            };
                            if (full) {
#pragma unroll
                                for (int p = 0; p < (kLine + 2) / 2; ++p) pair_mmas(p);
                            } else {
                                for (int p = 0; p < (t.fx + 3) / 2; ++p) pair_mmas(p);
                            }
                        } else if (full) {
#pragma unroll
                            for (int xa = -1; xa <= kLine; ++xa)
                                tile_mmas(xa, dyi, adesc0 + (uint64_t)((xa + 1) * (kSlotBytes >> 4)));
                        } else {
                            for (int xa = -1; xa <= t.fx; ++xa)
                                tile_mmas(xa, dyi, adesc0 + (uint64_t)((xa + 1) * (kSlotBytes >> 4)));
                        }
                        mma_commit(empty_bar(g));
                        ++gseq;
                    };
                    row_mmas(0);
                    row_mmas(1);
                    row_mmas(2);
                    if (!ok) break;
                    // output plane zi - 1 has received its last contribution
                    if (zi - 1 >= 0 && zi - 1 <= L - 1 && (int)((qbase + zi - 1) % kIssuers) == iss)
                        mma_commit(accf_bar((int)((qbase + zi - 1) & 3)));
                }
                qbase += L;
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(done_bar(iss));
            wait_bar(done_bar(iss), 0, abort_flag, true);
        }
        __syncwarp();
    } else {
        // epilogue: warp w owns TMEM lanes (= tile rows = samples) 32w .. 32w + 31
        const int r = warp * 32 + lane;
        float bias[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) bias[c] = a.bias[c];
        float w4[kHead ? 3 * kC : 1];
        float b4[3] = {0.0f, 0.0f, 0.0f};
        if (kHead) {
#pragma unroll
            for (int i = 0; i < 3 * kC; ++i) w4[i] = a.w4[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) b4[d] = a.b4[d];
        }
        int64_t q = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit t = unit_of(a, u);
            const int64_t sample = t.m0 + r;
            const bool valid = sample < a.n_samples;
            for (int zo = 0; zo < L; ++zo, ++q) {
                const int s = (int)(q & 3);
                // one lane waits; the warp stays converged for the .sync.aligned TMEM loads
                int got = 1;
                if (lane == 0) got = wait_bar(accf_bar(s), (uint32_t)(q >> 2) & 1u, abort_flag) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // four outputs per batch of TMEM loads, one wait per batch
                for (int ob = 0; ob < t.fx; ob += kEpiBatch) {
                    uint32_t raw[kEpiBatch][16];
#pragma unroll
                    for (int j = 0; j < kEpiBatch; ++j)
                        if (ob + j < t.fx)
                            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) +
                                          (uint32_t)(s * kN + (kLine - 1 - (ob + j)) * kC),
                                      raw[j]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < kEpiBatch; ++j) {
                        if (ob + j >= t.fx) continue;
                        const int64_t site = ((int64_t)zo * L + t.y) * L + (t.x0 + ob + j);
                        float v[16];
#pragma unroll
                        for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(raw[j][c]);
                        if (!kHead) {
                            uint32_t p[8];
#pragma unroll
                            for (int c = 0; c < kC; c += 2)
                                p[c / 2] = pack2(fmaxf(v[c] + bias[c], 0.0f), fmaxf(v[c + 1] + bias[c + 1], 0.0f));
                            uint8_t* dst = a.out + tile_off(site, t.m0, a.L3, 4096) + (r >> 3) * 256 + (r & 7) * 16;
                            *reinterpret_cast<uint4*>(dst) = make_uint4(p[0], p[1], p[2], p[3]);
                            *reinterpret_cast<uint4*>(dst + 128) = make_uint4(p[4], p[5], p[6], p[7]);
                        } else {
                            float z[3] = {b4[0], b4[1], b4[2]};
#pragma unroll
                            for (int c = 0; c < kC; ++c) {
                                const float y = fmaxf(v[c] + bias[c], 0.0f);
#pragma unroll
                                for (int d = 0; d < 3; ++d) z[d] = fmaf(y, w4[d * kC + c], z[d]);
                            }
                            const int64_t wd = (t.m0 + warp * 32) / 64;
                            const int hw = warp & 1;
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                if (a.logits && valid)
                                    a.logits[((int64_t)d * a.L3 + site) * a.n_samples + sample] = z[d];
                                const uint32_t bits = __ballot_sync(0xffffffffu, valid && z[d] > 0.0f);
                                if (lane == 0 && wd < a.words) a.dec32[(wd * a.L3 + site) * 8 + 2 * d + hw] = bits;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce_bar(s));
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
// (108 of 168 per plane; the line kernel: 30%).  A window that would cross
// the ring's end is split in two MMAs.  TMEM columns are zeroed by the
// epilogue after it drains a plane (and once at the start), so every MMA
// accumulates.  The first layer pairs x-adjacent input sites in one K = 16
// operand (chunk c = site 2p - 1 + c of the row) as the line kernel does.
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
    t.fx = 0;
    return t;
}

template <bool kHead, bool kBitsIn>
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
                                 tile_bytes, full_bar(g), false);
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
        float bias[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) bias[c] = a.bias[c];
        float w4[kHead ? 3 * kC : 1];
        float b4[3] = {0.0f, 0.0f, 0.0f};
        if (kHead) {
#pragma unroll
            for (int i = 0; i < 3 * kC; ++i) w4[i] = a.w4[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) b4[d] = a.b4[d];
        }
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
                    float v[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(raw[j][c]);
                    if (!kHead) {
                        uint32_t pk[8];
#pragma unroll
                        for (int c = 0; c < kC; c += 2)
                            pk[c / 2] = pack2(fmaxf(v[c] + bias[c], 0.0f), fmaxf(v[c + 1] + bias[c + 1], 0.0f));
                        uint8_t* dst = a.out + tile_off(site, t.m0, a.L3, 4096) + (r >> 3) * 256 + (r & 7) * 16;
                        *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
                        float z[3] = {b4[0], b4[1], b4[2]};
#pragma unroll
                        for (int c = 0; c < kC; ++c) {
                            const float y = fmaxf(v[c] + bias[c], 0.0f);
#pragma unroll
                            for (int d = 0; d < 3; ++d) z[d] = fmaf(y, w4[d * kC + c], z[d]);
                        }
                        const int64_t wd = (t.m0 + warp * 32) / 64;
                        const int hw = warp & 1;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (a.logits && valid)
                                a.logits[((int64_t)d * a.L3 + site) * a.n_samples + sample] = z[d];
                            const uint32_t bits = __ballot_sync(0xffffffffu, valid && z[d] > 0.0f);
                            if (lane == 0 && wd < a.words) a.dec32[(wd * a.L3 + site) * 8 + 2 * d + hw] = bits;
                        }
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce_bar(s));
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

int64_t tc_padded(int64_t n) { return (n + kTileM - 1) / kTileM * kTileM; }
size_t r256(size_t x) { return (x + 255) / 256 * 256; }

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <bool kHead, bool kBitsIn>
t3d_status launch_conv(const TcArgs& a, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>(a.n_units, sm_count());
    ProfScope prof(T3D_K_CNN, st);
    k_conv_tc<kHead, kBitsIn><<<grid, kTcThreads, kSmemBytes, st>>>(a);
    T3D_LAUNCH_CHECK("tensor-core convolution");
    return T3D_OK;
}

template <bool kHead, bool kBitsIn>
t3d_status launch_conv_col(const TcArgs& a, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>(a.n_units, sm_count());
    ProfScope prof(T3D_K_CNN, st);
    k_conv_col<kHead, kBitsIn><<<grid, kTcThreads, kColSmemBytes, st>>>(a);
    T3D_LAUNCH_CHECK("tensor-core convolution (2 x 2 columns)");
    return T3D_OK;
}

// The line kernel stays selectable (T3D_CNN_LINES=1 in the environment) for comparisons.
bool use_line_kernel()
{
    static const bool lines = [] {
        const char* v = std::getenv("T3D_CNN_LINES");
        return v && v[0] == '1';
    }();
    return lines;
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
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kColSmemBytes));
        T3D_CUDA_CHECK(cudaFuncSetAttribute(k_conv_col<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kColSmemBytes));
        configured[dev] = true;
    }
    return T3D_OK;
}

size_t tc_workspace_bytes(int L, int64_t n_samples)
{
    const size_t sites = (size_t)L * L * L, Sp = (size_t)tc_padded(n_samples);
    return r256(sites * Sp * 16) + 2 * r256(sites * Sp * 32);
}

t3d_status launch_forward_tc(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, const uint64_t* s,
                             uint64_t* dec, const Blob* blob, float* logits_out, void* work, cudaStream_t st)
{
    const int64_t Sp = tc_padded(n_samples), L3 = (int64_t)L * L * L;
    uint8_t* base = static_cast<uint8_t*>(work);
    uint8_t* in0 = base;
    uint8_t* act0 = in0 + r256((size_t)L3 * Sp * 16);
    uint8_t* act1 = act0 + r256((size_t)L3 * Sp * 32);
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = L;
    a.L3 = (int)L3;
    a.Sp = Sp;
    a.n_samples = n_samples;
    a.W = W;
    a.words = words_for(n_samples);
    a.nbx = (L + kLine - 1) / kLine;
    a.ncx = (L + 1) / 2;
    const bool lines = use_line_kernel();
    a.n_units = lines ? (Sp / kTileM) * a.nbx * L : (Sp / kTileM) * a.ncx * a.ncx;
    T3D_TRY(tc_prepare());
    {
        ProfScope prof(T3D_K_CNN, st);
        const dim3 grid((unsigned)((L3 + 7) / 8), (unsigned)((Sp + 255) / 256));
        k_expand_bits<<<grid, 256, 0, st>>>((int)L3, Sp, W, a.words, s_prev, s, reinterpret_cast<uint4*>(in0));
        T3D_LAUNCH_CHECK("pre-decoder input expansion");
    }
    a.in = in0;
    a.out = act0;
    a.w = &blob->wf[0][0][0][0];
    a.bias = blob->bias[0];
    T3D_TRY((lines ? launch_conv<false, true>(a, st) : launch_conv_col<false, true>(a, st)));
    a.in = act0;
    a.out = act1;
    a.w = &blob->wf[1][0][0][0];
    a.bias = blob->bias[1];
    T3D_TRY((lines ? launch_conv<false, false>(a, st) : launch_conv_col<false, false>(a, st)));
    a.in = act1;
    a.out = nullptr;
    a.w = &blob->wf[2][0][0][0];
    a.bias = blob->bias[2];
    a.w4 = &blob->w4[0][0];
    a.b4 = blob->b4;
    a.dec32 = reinterpret_cast<uint32_t*>(dec);
    a.logits = logits_out;
    T3D_TRY((lines ? launch_conv<true, false>(a, st) : launch_conv_col<true, false>(a, st)));
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
