// Product-sum belief propagation on the face Tanner graph of the 3D toric
// code (Sec. 4.1 of arXiv:2212.06985, Eqs. 1-4), FP32, one sample per thread.
//
// Layout: a message buffer is float[words][L^3][3][4][64]; entry
// (w, site, d, k, i) is M_{f->v} into edge v = (d, site) from its k-th face
// (slot order of edge_faces()) for sample 64 w + i -- the same 64 samples as
// one word of the bit-sliced state.  A warp handles one site for 64 samples,
// lane l holding samples 2l and 2l+1 as a float2, so every message access is
// a coalesced 256-byte row.
//
// Check-node arithmetic.  For inputs x_i (variable->check messages) let
// t_i = tanh(|x_i|/2) and d_i = 1 - t_i = 2 e^{-|x_i|} / (1 + e^{-|x_i|}).
// Products of (t, d) pairs are formed as (tA tB, dA + tA dB), which is exact
// algebra with no cancellation, so P = prod t and D = 1 - P are both accurate
// even when P rounds to 1 in FP32.  The output magnitude is
// 2 atanh(P) = log1p(2P / D), and its sign is (-1)^{s_f} times the signs of
// the other inputs.  The measurement-error variable of Sec. 4.1 enters as one
// more constant pair (tq, dq).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "t3d_device.cuh"
#include "t3d_host.hpp"
#include "t3d_bp_math.cuh"
#include "t3d_items.cuh"

namespace t3d {
namespace {

using namespace bpm;

constexpr int kBpThreads = 256;
constexpr int kWord = 64;  // samples per message row (one bit-sliced word)
constexpr float kMsgClamp = 30.0f;
// Message offsets within one word-row block, 3 L^3 * 256 floats, stay below 2^31.
constexpr int kMaxBpL = 128;

// The check node on a lane's two samples at once with the packed two-wide FP32
// instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn): every operation is the scalar
// one of td_of / td_mul / two_atanh (t3d_bp_math.cuh) in the same order and
// rounding, applied to both samples, so the messages are bit for bit those of the
// scalar code; the MUFU approximations and the selects stay per sample.
struct TD2 {
    float2 t, d;
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ TD2 td2_mul(const TD2& A, const TD2& B)
{
    return TD2{__fmul2_rn(A.t, B.t), __ffma2_rn(A.t, B.d, A.d)};
}

__device__ __forceinline__ TD2 td2_of(float2 x)
{
    const float2 a = make_float2(fabsf(x.x), fabsf(x.y));
    const float2 m = __fmul2_rn(make_float2(-a.x, -a.y), f2(kLog2e));
    const float2 E = make_float2(ex2_approx(m.x), ex2_approx(m.y));
    const float2 e1 = __fadd2_rn(f2(1.0f), E);
    const float2 r = make_float2(rcp_approx(e1.x), rcp_approx(e1.y));
    float2 h = __ffma2_rn(a, f2(-1.0f / 24.0f), f2(1.0f / 6.0f));
    h = __ffma2_rn(a, h, f2(-0.5f));
    h = __ffma2_rn(a, h, f2(1.0f));
    const float2 ah = __fmul2_rn(a, h);
    const float2 ome = __fadd2_rn(f2(1.0f), make_float2(-E.x, -E.y));
    const float2 om = make_float2(a.x < 0.1f ? ah.x : ome.x, a.y < 0.1f ? ah.y : ome.y);
    return TD2{__fmul2_rn(om, r), __fmul2_rn(__fadd2_rn(E, E), r)};
}

__device__ __forceinline__ float2 two_atanh2(float2 P, float2 D)
{
    const float2 u = __fmul2_rn(P, P);
    const float2 poly = __ffma2_rn(u, __ffma2_rn(u, f2(1.0f / 5.0f), f2(1.0f / 3.0f)), f2(1.0f));
    const float2 series = __fmul2_rn(__fmul2_rn(f2(2.0f), P), poly);
    const float2 arg = __fmul2_rn(__fadd2_rn(f2(1.0f), P), make_float2(rcp_approx(D.x), rcp_approx(D.y)));
    const float2 logv = __fmul2_rn(f2(kLn2), make_float2(lg2_approx(arg.x), lg2_approx(arg.y)));
    return make_float2(P.x < 0.05f ? series.x : logv.x, P.y < 0.05f ? series.y : logv.y);
}

// Eq. 2 for the four edges of one face on both samples of a lane: y[j] from the other three
// inputs and the measurement-variable pair q; the sign of y[j] is (-1)^{s_f} times the product
// of the other inputs' signs, the XOR of their IEEE sign bits.  Bit for bit the scalar check
// node it replaced (545 -> 424 M warp instructions per iteration at L = 32, 1024 samples; the
// iteration is HBM-bound, 219.7 -> 217.7 ms for 16 iterations of a 25,024-sample chunk).
__device__ __forceinline__ void check_node2(const float2 x[4], bool s_neg0, bool s_neg1, const TD2& q, float2 y[4])
{
    TD2 in[4];
    uint32_t sa0 = s_neg0 ? 0x80000000u : 0u, sa1 = s_neg1 ? 0x80000000u : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        in[j] = td2_of(x[j]);
        sa0 ^= __float_as_uint(x[j].x);
        sa1 ^= __float_as_uint(x[j].y);
    }
    const TD2 pre1 = td2_mul(q, in[0]);
    const TD2 pre2 = td2_mul(pre1, in[1]);
    const TD2 suf2 = in[3];
    const TD2 suf1 = td2_mul(in[2], suf2);
    const TD2 o[4] = {td2_mul(q, td2_mul(in[1], suf1)), td2_mul(pre1, suf1), td2_mul(pre2, suf2),
                      td2_mul(pre2, in[2])};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 v = two_atanh2(o[j].t, o[j].d);
        const float m0 = fminf(v.x, kMsgClamp), m1 = fminf(v.y, kMsgClamp);
        const uint32_t g0 = (sa0 ^ __float_as_uint(x[j].x)) & 0x80000000u;
        const uint32_t g1 = (sa1 ^ __float_as_uint(x[j].y)) & 0x80000000u;
        y[j] = make_float2(__uint_as_float(__float_as_uint(m0) | g0), __uint_as_float(__float_as_uint(m1) | g1));
    }
}

// Work: per item, one warp per (site, word) of the current chunk handles the
// three faces at that site (normals x, y, z) for the word's 64 samples; an
// item's local block lb covers 8 consecutive sites of word lb / site_blocks,
// so sites vary fastest.  With r the site and e_a the unit steps, the faces'
// edges and the slot each face occupies in its edges' face lists are
// (edge_faces order):
//   face n=0: (y,r) slot 2, (y,r+e_z) slot 3, (z,r) slot 2, (z,r+e_y) slot 3
//   face n=1: (x,r) slot 2, (x,r+e_z) slot 3, (z,r) slot 0, (z,r+e_x) slot 1
//   face n=2: (x,r) slot 0, (x,r+e_y) slot 1, (y,r) slot 0, (y,r+e_x) slot 1
struct SiteWarp {
    int64_t w;  // word (64-sample group) within the chunk
    int site;
    int nb[3];  // site + e_x, site + e_y, site + e_z (periodic)
};

constexpr int kWarpsPerBlock = kBpThreads / 32;

__host__ __device__ __forceinline__ int64_t site_blocks(int L3) { return (L3 + kWarpsPerBlock - 1) / kWarpsPerBlock; }

__device__ __forceinline__ bool site_warp(const Lattice& lat, int64_t lb, SiteWarp& sw)
{
    const int64_t sbn = site_blocks(lat.L3);
    sw.w = lb / sbn;
    const int site = (int)((lb - sw.w * sbn) * kWarpsPerBlock + (threadIdx.x >> 5));
    if (site >= lat.L3) return false;
    sw.site = site;
    const Coord r = site_coord(lat, site);
    const int step[3] = {1, lat.L, lat.L2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        sw.nb[a] = site + ((r.x[a] + 1 == lat.L) ? step[a] * (1 - lat.L) : step[a]);
    return true;
}

// Offset of edge (d, site)'s 4x64 message block within a word-row block.
__device__ __forceinline__ int msg_off(int site, int d) { return (site * 3 + d) * (4 * kWord); }

// Where an iteration takes the syndrome from: the caller's bit-sliced words
// (kSynWords), the same and also a per-word copy for later iterations
// (kSynWordsSave: the three faces' words of a site side by side), or that
// copy (kSynSaved), which brings a site's syndrome in one 32-byte load.
enum SynMode { kSynWords = 0, kSynWordsSave = 1, kSynSaved = 2 };

struct __align__(32) Syn3 {
    uint64_t f[4];  // faces 0..2, padding
};

// The two syndrome bits of this lane's samples (2 lane, 2 lane + 1).
__device__ __forceinline__ bool sbit(uint64_t word, int lane, int j) { return (word >> (2 * lane + j)) & 1ULL; }

// One flooding iteration for the three faces of a site: Eq. 3 (variable->check
// inputs, each the prior plus the three messages of its edge other than the
// face's own slot, which is not read) and Eq. 2 (check->variable) into msg_out.
// msg_in == nullptr is the first iteration: every input is the prior l0, so
// every output is (-1)^{s_f} m1 with m1 = 2 atanh(tq tanh(l0/2)^3) computed
// once on the host, and the launch only writes.
template <int kSyn>
__global__ void __launch_bounds__(kBpThreads, 4)
k_bp_step(const __grid_constant__ ItemTable tab, float l0, TD q, float m1)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
    const Lattice lat = d.lat;
    const int64_t W = d.W;
    SiteWarp sw;
    if (!site_warp(lat, lb, sw)) return;
    if (!word_live(d, sw.w)) return;
    const int lane = threadIdx.x & 31;
    Syn3* __restrict__ syn = reinterpret_cast<Syn3*>(d.syn);
    uint64_t s0, s1, s2;
    if (kSyn == kSynSaved) {
        const Syn3 v = syn[sw.w * lat.L3 + sw.site];
        s0 = v.f[0];
        s1 = v.f[1];
        s2 = v.f[2];
    } else {
        s0 = d.s[((int64_t)0 * lat.L3 + sw.site) * W + sw.w];
        s1 = d.s[((int64_t)1 * lat.L3 + sw.site) * W + sw.w];
        s2 = d.s[((int64_t)2 * lat.L3 + sw.site) * W + sw.w];
        if (kSyn == kSynWordsSave && lane == 0) {
            Syn3 v;
            v.f[0] = s0;
            v.f[1] = s1;
            v.f[2] = s2;
            v.f[3] = 0;
            syn[sw.w * lat.L3 + sw.site] = v;
        }
    }
    const int64_t wbase = sw.w * (int64_t)lat.L3 * (3 * 4 * kWord) + 2 * lane;
    const int r = sw.site, rx = sw.nb[0], ry = sw.nb[1], rz = sw.nb[2];
    // message blocks: edges at r (x, y, z) and the six neighbours used
    const int oXr = msg_off(r, 0), oYr = msg_off(r, 1), oZr = msg_off(r, 2);
    const int oXy = msg_off(ry, 0), oXz = msg_off(rz, 0);
    const int oYx = msg_off(rx, 1), oYz = msg_off(rz, 1);
    const int oZx = msg_off(rx, 2), oZy = msg_off(ry, 2);
    if (!d.msg_in) {
        float* o = d.msg_out + wbase;
        auto PUT1 = [&](int off, uint64_t sw) {
            const float a = sbit(sw, lane, 0) ? -m1 : m1, b = sbit(sw, lane, 1) ? -m1 : m1;
            __stcs(reinterpret_cast<float2*>(o + off), make_float2(a, b));
        };
        PUT1(oYr + 2 * kWord, s0);
        PUT1(oYz + 3 * kWord, s0);
        PUT1(oZr + 2 * kWord, s0);
        PUT1(oZy + 3 * kWord, s0);
        PUT1(oXr + 2 * kWord, s1);
        PUT1(oXz + 3 * kWord, s1);
        PUT1(oZr + 0 * kWord, s1);
        PUT1(oZx + 1 * kWord, s1);
        PUT1(oXr + 0 * kWord, s2);
        PUT1(oXy + 1 * kWord, s2);
        PUT1(oYr + 0 * kWord, s2);
        PUT1(oYx + 1 * kWord, s2);
        return;
    }
    // inputs [face][edge] for the lane's two samples, edges in face_edges order
    float2 in[3][4];
    {
        const float* m = d.msg_in + wbase;
        auto M = [&](int o, int k) { return *reinterpret_cast<const float2*>(m + o + k * kWord); };
        const float2 xr0 = M(oXr, 0), xr1 = M(oXr, 1), xr2 = M(oXr, 2), xr3 = M(oXr, 3);
        const float2 yr0 = M(oYr, 0), yr1 = M(oYr, 1), yr2 = M(oYr, 2), yr3 = M(oYr, 3);
        const float2 zr0 = M(oZr, 0), zr1 = M(oZr, 1), zr2 = M(oZr, 2), zr3 = M(oZr, 3);
        const float2 yz0 = M(oYz, 0), yz1 = M(oYz, 1), yz2 = M(oYz, 2);
        const float2 zy0 = M(oZy, 0), zy1 = M(oZy, 1), zy2 = M(oZy, 2);
        const float2 xz0 = M(oXz, 0), xz1 = M(oXz, 1), xz2 = M(oXz, 2);
        const float2 zx0 = M(oZx, 0), zx2 = M(oZx, 2), zx3 = M(oZx, 3);
        const float2 xy0 = M(oXy, 0), xy2 = M(oXy, 2), xy3 = M(oXy, 3);
        const float2 yx0 = M(oYx, 0), yx2 = M(oYx, 2), yx3 = M(oYx, 3);
        const float2 L0 = f2(l0);
        auto A = [](float2 a, float2 b) { return __fadd2_rn(a, b); };
        const float2 xs = A(A(L0, xr1), xr3), ys = A(A(L0, yr1), yr3), zs = A(A(L0, zr1), zr3);
        // face 0: (y,r) excl 2, (y,r+z) excl 3, (z,r) excl 2, (z,r+y) excl 3
        in[0][0] = A(ys, yr0);
        in[0][1] = A(A(A(L0, yz0), yz1), yz2);
        in[0][2] = A(zs, zr0);
        in[0][3] = A(A(A(L0, zy0), zy1), zy2);
        // face 1: (x,r) excl 2, (x,r+z) excl 3, (z,r) excl 0, (z,r+x) excl 1
        in[1][0] = A(xs, xr0);
        in[1][1] = A(A(A(L0, xz0), xz1), xz2);
        in[1][2] = A(zs, zr2);
        in[1][3] = A(A(A(L0, zx0), zx2), zx3);
        // face 2: (x,r) excl 0, (x,r+y) excl 1, (y,r) excl 0, (y,r+x) excl 1
        in[2][0] = A(xs, xr2);
        in[2][1] = A(A(A(L0, xy0), xy2), xy3);
        in[2][2] = A(ys, yr2);
        in[2][3] = A(A(A(L0, yx0), yx2), yx3);
    }
    float* o = d.msg_out + wbase;
    // the new messages are not read again in this launch: store them evict-first
    auto PUT = [&](int off, float2 v) { __stcs(reinterpret_cast<float2*>(o + off), v); };
    const TD2 q2{f2(q.t), f2(q.d)};
    float2 y[4];
    check_node2(in[0], sbit(s0, lane, 0), sbit(s0, lane, 1), q2, y);
    PUT(oYr + 2 * kWord, y[0]);
    PUT(oYz + 3 * kWord, y[1]);
    PUT(oZr + 2 * kWord, y[2]);
    PUT(oZy + 3 * kWord, y[3]);
    check_node2(in[1], sbit(s1, lane, 0), sbit(s1, lane, 1), q2, y);
    PUT(oXr + 2 * kWord, y[0]);
    PUT(oXz + 3 * kWord, y[1]);
    PUT(oZr + 0 * kWord, y[2]);
    PUT(oZx + 1 * kWord, y[3]);
    check_node2(in[2], sbit(s2, lane, 0), sbit(s2, lane, 1), q2, y);
    PUT(oXr + 0 * kWord, y[0]);
    PUT(oXy + 1 * kWord, y[1]);
    PUT(oYr + 0 * kWord, y[2]);
    PUT(oYx + 1 * kWord, y[3]);
    });
}

// 32 ballot bits b_l -> 64-bit word with b_l at bit 2l (the even bits).
__device__ __forceinline__ uint64_t spread_even(uint32_t x)
{
    uint64_t v = x;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFULL;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFULL;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0FULL;
    v = (v | (v << 2)) & 0x3333333333333333ULL;
    v = (v | (v << 1)) & 0x5555555555555555ULL;
    return v;
}

// Eq. 4 posterior and the hard decision, pass 1: for the three edges at a
// site, l = l0 + the four incoming messages and d = [l < 0]; the warp XORs d
// into e at the site (each 64-sample word has exactly one writer) and leaves
// the three decision words in the chunk's syndrome-copy slot of the site,
// which the iterations no longer need.  Every message is read once.
__global__ void __launch_bounds__(kBpThreads)
k_bp_decide(const __grid_constant__ ItemTable tab, float l0)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
    const Lattice lat = d.lat;
    const int64_t W = d.W;
    SiteWarp sw;
    if (!site_warp(lat, lb, sw)) return;
    if (!word_live(d, sw.w)) return;
    const int lane = threadIdx.x & 31;
    const int64_t sample0 = sw.w * kWord + 2 * lane;
    const bool valid0 = sample0 < d.n_samples, valid1 = sample0 + 1 < d.n_samples;
    const int64_t wbase = sw.w * (int64_t)lat.L3 * (3 * 4 * kWord) + 2 * lane;
    const int r = sw.site;
    float2 l[3];
    uint64_t dec[3];
    // all twelve message loads are issued before the first ballot, evict-first (each is read
    // once): 8.40 -> 7.00 ms per 25,024-sample chunk at L = 32, 39.7 GB read against the
    // algorithmic 39.4 GB (83% of the measured HBM bandwidth)
    float2 v[3][4] = {};
    if (d.msg_in) {
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            const float* m = d.msg_in + wbase + msg_off(r, dd);
#pragma unroll
            for (int k = 0; k < 4; ++k) v[dd][k] = __ldcs(reinterpret_cast<const float2*>(m + k * kWord));
        }
    }
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        l[dd] = make_float2(l0, l0);
        if (d.msg_in) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                l[dd].x += v[dd][k].x;
                l[dd].y += v[dd][k].y;
            }
        }
        const uint32_t b0 = __ballot_sync(0xffffffffu, valid0 && l[dd].x < 0.0f);
        const uint32_t b1 = __ballot_sync(0xffffffffu, valid1 && l[dd].y < 0.0f);
        dec[dd] = spread_even(b0) | (spread_even(b1) << 1);
    }
    if (lane < 3) {
        const uint64_t v = lane == 0 ? dec[0] : (lane == 1 ? dec[1] : dec[2]);
        if (v) d.e[((int64_t)lane * lat.L3 + r) * W + sw.w] ^= v;
    }
    if (lane == 0) {
        Syn3 out;
        out.f[0] = dec[0];
        out.f[1] = dec[1];
        out.f[2] = dec[2];
        out.f[3] = 0;
        reinterpret_cast<Syn3*>(d.syn)[sw.w * lat.L3 + r] = out;
    }
    if (d.llr) {
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            float* row = d.llr + ((int64_t)dd * lat.L3 + r) * d.n_samples;
            if (valid0) row[sample0] = l[dd].x;
            if (valid1) row[sample0 + 1] = l[dd].y;
        }
    }
    });
}

// Pass 2: s ^= H d.  One thread per (site, word); a warp covers 32 words of
// one site, so the syndrome rows are read and written coalesced.  Face n at r
// holds the edges listed at the top of this file, so its parity is
//   n=0: d(y,r) ^ d(y,r+e_z) ^ d(z,r) ^ d(z,r+e_y)
//   n=1: d(x,r) ^ d(x,r+e_z) ^ d(z,r) ^ d(z,r+e_x)
//   n=2: d(x,r) ^ d(x,r+e_y) ^ d(y,r) ^ d(y,r+e_x).
constexpr int kSynWordsPerRow = 32;
constexpr int kSynSitesPerBlock = kBpThreads / kSynWordsPerRow;

__host__ __device__ __forceinline__ int64_t syn_blocks(int L3, int64_t words)
{
    return ((L3 + kSynSitesPerBlock - 1) / kSynSitesPerBlock) *
           ((words + kSynWordsPerRow - 1) / kSynWordsPerRow);
}

__global__ void __launch_bounds__(kBpThreads)
k_bp_syndrome(const __grid_constant__ ItemTable tab)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
    const Lattice lat = d.lat;
    const int64_t site_tiles = (lat.L3 + kSynSitesPerBlock - 1) / kSynSitesPerBlock;
    const int64_t word_tile = lb / site_tiles;
    const int r = (int)((lb - word_tile * site_tiles) * kSynSitesPerBlock + (threadIdx.x / kSynWordsPerRow));
    const int64_t w = word_tile * kSynWordsPerRow + (threadIdx.x % kSynWordsPerRow);
    if (r >= lat.L3 || w >= d.words) return;
    if (!word_live(d, w)) return;
    const Coord rc = site_coord(lat, r);
    const int step[3] = {1, lat.L, lat.L2};
    int nb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nb[a] = r + ((rc.x[a] + 1 == lat.L) ? step[a] * (1 - lat.L) : step[a]);
    const Syn3* D = reinterpret_cast<const Syn3*>(d.syn) + w * lat.L3;
    const Syn3 dr = D[r], dx = D[nb[0]], dy = D[nb[1]], dz = D[nb[2]];
    const uint64_t par[3] = {dr.f[1] ^ dz.f[1] ^ dr.f[2] ^ dy.f[2], dr.f[0] ^ dz.f[0] ^ dr.f[2] ^ dx.f[2],
                             dr.f[0] ^ dy.f[0] ^ dr.f[1] ^ dx.f[1]};
#pragma unroll
    for (int n = 0; n < 3; ++n)
        if (par[n]) d.s[((int64_t)n * lat.L3 + r) * d.W + w] ^= par[n];
    });
}

Lattice make_lattice(int L) { return make_lattice_host(L); }

TD meas_pair(double q_meas)
{
    if (!(q_meas > 0.0)) return TD{1.0f, 0.0f};
    double lq = std::log((1.0 - q_meas) / q_meas);
    double E = std::exp(-std::fabs(lq));
    double t = std::tanh(lq / 2.0);
    return TD{(float)t, (float)(2.0 * E / (1.0 + E))};
}

float prior(double p) { return (float)std::log((1.0 - p) / p); }

// First-iteration message magnitude (signed): 2 atanh(tq tanh(l0/2)^3), Eq. 2
// with every input equal to the prior, clamped like every message.
float first_message(double p, double q_meas)
{
    const double l0 = std::log((1.0 - p) / p);
    const double tq = q_meas > 0.0 ? std::tanh(std::log((1.0 - q_meas) / q_meas) / 2.0) : 1.0;
    const double t0 = std::tanh(l0 / 2.0);
    double m = 2.0 * std::atanh(std::max(-1.0 + 1e-15, std::min(1.0 - 1e-15, tq * t0 * t0 * t0)));
    m = std::max(-30.0, std::min(30.0, m));
    return (float)m;
}

int64_t word_floats(int L) { return 3LL * L * L * L * 4 * kWord; }
int64_t word_syn_bytes(int L) { return (int64_t)L * L * L * (int64_t)sizeof(Syn3); }

void set_blocks(ItemTable& tab)
{
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        d.blocks = site_blocks(d.lat.L3) * d.words;
        d.live_wpu = 1;
        d.live_bpu = site_blocks(d.lat.L3);
    }
    finish_table(tab);
}

t3d_status launch_step(ItemTable& tab, int mode, double p, double q_meas, cudaStream_t st)
{
    set_blocks(tab);
    const int64_t blocks = tab.prefix[tab.n];
    const bool live = has_live(tab);
    ProfScope prof(T3D_K_BP_STEP, st);
    if (mode == kSynWordsSave)
        k_bp_step<kSynWordsSave><<<persistent_grid((const void*)k_bp_step<kSynWordsSave>, kBpThreads,
                                                   T3D_K_BP_STEP, blocks, live),
                                   kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas), first_message(p, q_meas));
    else if (mode == kSynSaved)
        k_bp_step<kSynSaved><<<persistent_grid((const void*)k_bp_step<kSynSaved>, kBpThreads, T3D_K_BP_STEP,
                                               blocks, live),
                               kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas), first_message(p, q_meas));
    else
        k_bp_step<kSynWords><<<persistent_grid((const void*)k_bp_step<kSynWords>, kBpThreads, T3D_K_BP_STEP,
                                               blocks, live),
                               kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas), first_message(p, q_meas));
    T3D_LAUNCH_CHECK("bp step");
    return T3D_OK;
}

t3d_status launch_decide(ItemTable& tab, double p, cudaStream_t st)
{
    set_blocks(tab);
    {
        ProfScope prof(T3D_K_BP_DECIDE, st);
        k_bp_decide<<<persistent_grid((const void*)k_bp_decide, kBpThreads, T3D_K_BP_DECIDE, tab.prefix[tab.n], has_live(tab)),
                      kBpThreads, 0, st>>>(tab, prior(p));
        T3D_LAUNCH_CHECK("bp decide");
    }
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        d.blocks = syn_blocks(d.lat.L3, d.words);
        d.live_wpu = kSynWordsPerRow;
        d.live_bpu = (d.lat.L3 + kSynSitesPerBlock - 1) / kSynSitesPerBlock;
    }
    finish_table(tab);
    ProfScope prof(T3D_K_BP_DECIDE, st);
    k_bp_syndrome<<<persistent_grid((const void*)k_bp_syndrome, kBpThreads, T3D_K_BP_DECIDE, tab.prefix[tab.n], has_live(tab)),
                    kBpThreads, 0, st>>>(tab);
    T3D_LAUNCH_CHECK("bp syndrome update");
    return T3D_OK;
}

}  // namespace

size_t bp_bytes_per_word(int L)
{
    return 2 * (size_t)word_floats(L) * sizeof(float) + (size_t)word_syn_bytes(L);
}

// Chunks of chunk_words 64-sample words; an item's buffer holds two
// chunk-sized message buffers followed by the chunk's saved syndrome words.
// The kernels see a chunk's slice of e and s through offset pointers (the row
// stride W stays the whole batch's).
namespace {

int64_t bp_rounds(const ItemTable& items, const int64_t* chunk_words)
{
    int64_t rounds = 0;
    for (int i = 0; i < items.n; ++i) {
        const int64_t W = items.it[i].W;
        rounds = std::max(rounds, (W + chunk_words[i] - 1) / chunk_words[i]);
    }
    return rounds;
}

// Items' round-r chunks (items with no words left are dropped); A and B are
// each chunk's two message buffers.
ItemTable chunk_table(const ItemTable& items, float* const* bufs, const int64_t* chunk_words, int64_t r,
                      float* llr_out, float** A, float** B)
{
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    for (int i = 0; i < items.n; ++i) {
        const ItemDesc& src = items.it[i];
        const int64_t w0 = r * chunk_words[i];
        if (w0 >= src.W) continue;
        const int64_t wc = std::min(chunk_words[i], src.W - w0);
        const int k = tab.n++;
        ItemDesc& d = tab.it[k];
        d = src;
        d.e = src.e + w0;
        d.s = src.s + w0;
        d.w0 = w0;
        d.words = wc;
        d.n_samples = std::min<int64_t>(wc * kWord, src.n_samples - w0 * kWord);
        const int64_t fl = chunk_words[i] * word_floats(src.lat.L);
        A[k] = bufs[i];
        B[k] = bufs[i] + fl;
        d.syn = reinterpret_cast<uint4*>(bufs[i] + 2 * fl);
        d.llr = (llr_out && items.n == 1) ? llr_out + w0 * kWord : nullptr;
    }
    return tab;
}

}  // namespace

t3d_status launch_bp(const ItemTable& items, double p, double q_meas, int iters, float* const* bufs,
                     const int64_t* chunk_words, float* llr_out, cudaStream_t st)
{
    // in round r item i processes words [r*chunk_i, (r+1)*chunk_i)
    const int64_t rounds = bp_rounds(items, chunk_words);
    for (int64_t r = 0; r < rounds; ++r) {
        float* A[kMaxItems];
        float* B[kMaxItems];
        ItemTable tab = chunk_table(items, bufs, chunk_words, r, llr_out, A, B);
        for (int it = 0; it < iters; ++it) {
            for (int k = 0; k < tab.n; ++k) {
                tab.it[k].msg_in = it == 0 ? nullptr : B[k];
                tab.it[k].msg_out = A[k];
            }
            T3D_TRY(launch_step(tab, it == 0 ? kSynWordsSave : kSynSaved, p, q_meas, st));
            for (int k = 0; k < tab.n; ++k) std::swap(A[k], B[k]);
        }
        for (int k = 0; k < tab.n; ++k) tab.it[k].msg_in = iters > 0 ? B[k] : nullptr;
        T3D_TRY(launch_decide(tab, p, st));
    }
    return T3D_OK;
}

t3d_status autotune_bp(const ItemTable& items, double p, double q_meas, float* const* bufs,
                       const int64_t* chunk_words, cudaStream_t st, int* best_cap, float* best_ms)
{
    float* A[kMaxItems];
    float* B[kMaxItems];
    ItemTable tab = chunk_table(items, bufs, chunk_words, 0, nullptr, A, B);
    for (int k = 0; k < tab.n; ++k) {
        tab.it[k].msg_in = nullptr;
        tab.it[k].msg_out = A[k];
    }
    T3D_TRY(launch_step(tab, kSynWordsSave, p, q_meas, st));  // realistic messages in A
    for (int k = 0; k < tab.n; ++k) {
        tab.it[k].msg_in = A[k];
        tab.it[k].msg_out = B[k];
    }
    const int saved = tuned_blocks_per_sm(T3D_K_BP_STEP);
    const int caps[] = {0, 1, 2, 4, 6, 8};
    cudaEvent_t ev[2];
    T3D_CUDA_CHECK(cudaEventCreate(&ev[0]));
    T3D_CUDA_CHECK(cudaEventCreate(&ev[1]));
    *best_cap = 0;
    *best_ms = 1e30f;
    t3d_status status = T3D_OK;
    for (int cap : caps) {
        set_tuned_blocks_per_sm(T3D_K_BP_STEP, cap);
        status = launch_step(tab, kSynSaved, p, q_meas, st);  // warm-up
        if (status != T3D_OK) break;
        cudaEventRecord(ev[0], st);
        for (int rep = 0; rep < 3 && status == T3D_OK; ++rep) status = launch_step(tab, kSynSaved, p, q_meas, st);
        cudaEventRecord(ev[1], st);
        if (status != T3D_OK) break;
        float ms = 0.0f;
        if (cudaEventSynchronize(ev[1]) != cudaSuccess || cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
            set_error("autotune timing failed");
            status = T3D_ECUDA;
            break;
        }
        ms /= 3.0f;
        if (ms < *best_ms) {
            *best_ms = ms;
            *best_cap = cap;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    set_tuned_blocks_per_sm(T3D_K_BP_STEP, status == T3D_OK ? *best_cap : saved);
    return status;
}

}  // namespace t3d

using namespace t3d;

extern "C" size_t toric3d_bp_message_bytes(int L, int64_t n_samples)
{
    if (L < 2 || L > kMaxL || n_samples < 1) return 0;
    return (size_t)words_for(n_samples) * (size_t)word_floats(L) * sizeof(float);
}

extern "C" size_t toric3d_bp_workspace_bytes(int L, int64_t chunk_samples)
{
    if (L < 2 || L > kMaxL || chunk_samples < 1) return 0;
    return (size_t)words_for(chunk_samples) * bp_bytes_per_word(L);
}

static t3d_status bp_common_checks(int L, int64_t n_samples, double p, double q_meas)
{
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(L <= kMaxBpL, "BP supports L <= %d (L=%d)", kMaxBpL, L);
    T3D_REQUIRE(n_samples >= 1 && words_for(n_samples) <= (1LL << 40), "n_samples out of range");
    T3D_REQUIRE(p > 0.0 && p < 1.0, "BP needs 0 < p < 1 (p=%g)", p);
    T3D_REQUIRE(q_meas >= 0.0 && q_meas < 0.5, "BP needs 0 <= q_meas < 0.5 (q=%g)", q_meas);
    return T3D_OK;
}

extern "C" t3d_status toric3d_bp_step(int L, int64_t n_samples, const uint64_t* s, double p,
                                      double q_meas, const float* msg_in, float* msg_out,
                                      t3d_stream stream)
{
    clear_error();
    T3D_TRY(bp_common_checks(L, n_samples, p, q_meas));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(msg_out != nullptr && aligned(msg_out, 16), "msg_out must be 16-byte aligned");
    T3D_REQUIRE(msg_in == nullptr || aligned(msg_in, 16), "msg_in must be 16-byte aligned");
    T3D_REQUIRE(msg_in != msg_out, "msg_in and msg_out must differ");
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = 1;
    ItemDesc& d = tab.it[0];
    d.lat = make_lattice(L);
    d.W = words_for(n_samples);
    d.n_samples = n_samples;
    d.s = const_cast<uint64_t*>(s);
    d.msg_in = const_cast<float*>(msg_in);
    d.msg_out = msg_out;
    d.words = words_for(n_samples);
    return launch_step(tab, kSynWords, p, q_meas, as_stream(stream));
}

extern "C" size_t toric3d_bp_decide_workspace_bytes(int L, int64_t n_samples)
{
    if (L < 2 || L > kMaxL || n_samples < 1) return 0;
    return (size_t)words_for(n_samples) * (size_t)word_syn_bytes(L);
}

extern "C" t3d_status toric3d_bp_decide(int L, int64_t n_samples, const float* msg, double p,
                                        uint64_t* e, uint64_t* s, float* llr_out, void* work,
                                        size_t work_bytes, t3d_stream stream)
{
    clear_error();
    T3D_TRY(bp_common_checks(L, n_samples, p, 0.0));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(msg == nullptr || aligned(msg, 16), "msg must be 16-byte aligned");
    T3D_REQUIRE(llr_out == nullptr || aligned(llr_out, 4), "llr_out must be 4-byte aligned");
    T3D_REQUIRE(work != nullptr && aligned(work, 32), "work must be a 32-byte aligned device pointer");
    T3D_REQUIRE(work_bytes >= toric3d_bp_decide_workspace_bytes(L, n_samples), "workspace too small: %zu < %zu",
                work_bytes, toric3d_bp_decide_workspace_bytes(L, n_samples));
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = 1;
    ItemDesc& d = tab.it[0];
    d.lat = make_lattice(L);
    d.W = words_for(n_samples);
    d.n_samples = n_samples;
    d.e = e;
    d.s = s;
    d.msg_in = const_cast<float*>(msg);
    d.llr = llr_out;
    d.syn = static_cast<uint4*>(work);
    d.words = words_for(n_samples);
    return launch_decide(tab, p, as_stream(stream));
}

extern "C" t3d_status toric3d_bp(int L, int64_t n_samples, uint64_t* e, uint64_t* s, double p,
                                 double q_meas, int iters, void* work, size_t work_bytes,
                                 float* llr_out, t3d_stream stream)
{
    clear_error();
    T3D_TRY(bp_common_checks(L, n_samples, p, q_meas));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(iters >= 0, "iters must be >= 0");
    T3D_REQUIRE(work != nullptr && aligned(work, 16), "work must be a 16-byte aligned device pointer");
    int64_t chunk = (int64_t)(work_bytes / bp_bytes_per_word(L));
    const int64_t G = words_for(n_samples);
    T3D_REQUIRE(chunk >= 1, "workspace too small: %zu bytes, need at least %zu", work_bytes,
                toric3d_bp_workspace_bytes(L, 64));
    chunk = std::min(chunk, G);
    T3D_REQUIRE(llr_out == nullptr || chunk >= G, "llr_out requires a workspace for the whole batch");
    ItemTable items;
    std::memset(&items, 0, sizeof(items));
    items.n = 1;
    items.it[0].lat = make_lattice(L);
    items.it[0].W = words_for(n_samples);
    items.it[0].n_samples = n_samples;
    items.it[0].e = e;
    items.it[0].s = s;
    float* buf = static_cast<float*>(work);
    return launch_bp(items, p, q_meas, iters, &buf, &chunk, llr_out, as_stream(stream));
}
