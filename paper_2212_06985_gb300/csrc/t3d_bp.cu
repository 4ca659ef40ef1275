// Product-sum belief propagation on the face Tanner graph of the 3D toric
// code (Sec. 4.1 of arXiv:2212.06985, Eqs. 1-4), FP32, one sample per thread.
//
// Layout: a message buffer is float[groups][L^3][3][4][32]; entry
// (g, site, d, k, lane) is M_{f->v} into edge v = (d, site) from its k-th face
// (slot order of edge_faces()) for sample 32 g + lane.  A warp handles one
// face for 32 samples, so every message access is a coalesced 128-byte row.
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
#include "t3d_items.cuh"

namespace t3d {
namespace {

constexpr int kBpThreads = 256;
constexpr int kLanes = 32;
constexpr float kMsgClamp = 30.0f;
// Message offsets within one group, 3 L^3 * 128 floats, stay below 2^31.
constexpr int kMaxBpL = 128;

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

// Eq. 2 for the four edges of one face: y[j] from the other three inputs and
// the measurement-variable pair q.  The sign of y[j] is (-1)^{s_f} times the
// product of the other inputs' signs: the XOR of their IEEE sign bits.
__device__ __forceinline__ void check_node(const float x[4], bool s_neg, TD q, float y[4])
{
    TD in[4];
    uint32_t sgn_all = s_neg ? 0x80000000u : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        in[j] = td_of(x[j]);
        sgn_all ^= __float_as_uint(x[j]);
    }
    const TD pre1 = td_mul(q, in[0]);
    const TD pre2 = td_mul(pre1, in[1]);
    const TD suf2 = in[3];
    const TD suf1 = td_mul(in[2], suf2);
    const TD o[4] = {td_mul(q, td_mul(in[1], suf1)), td_mul(pre1, suf1), td_mul(pre2, suf2),
                     td_mul(pre2, in[2])};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float mag = fminf(two_atanh(o[j].t, o[j].d), kMsgClamp);
        const uint32_t sgn = (sgn_all ^ __float_as_uint(x[j])) & 0x80000000u;
        y[j] = __uint_as_float(__float_as_uint(mag) | sgn);
    }
}

// Work: per item, one warp per (site, group) of the current chunk handles the
// three faces at that site (normals x, y, z); an item's local block lb covers
// 8 consecutive sites of group lb / site_blocks, so sites vary fastest.  With r the site and e_a the unit steps, the faces' edges and the
// slot each face occupies in its edges' face lists are (edge_faces order):
//   face n=0: (y,r) slot 2, (y,r+e_z) slot 3, (z,r) slot 2, (z,r+e_y) slot 3
//   face n=1: (x,r) slot 2, (x,r+e_z) slot 3, (z,r) slot 0, (z,r+e_x) slot 1
//   face n=2: (x,r) slot 0, (x,r+e_y) slot 1, (y,r) slot 0, (y,r+e_x) slot 1
struct SiteWarp {
    int64_t g;
    int site;
    int nb[3];  // site + e_x, site + e_y, site + e_z (periodic)
};

constexpr int kWarpsPerBlock = kBpThreads / 32;

__host__ __device__ __forceinline__ int64_t site_blocks(int L3) { return (L3 + kWarpsPerBlock - 1) / kWarpsPerBlock; }

__device__ __forceinline__ bool site_warp(const Lattice& lat, int64_t lb, SiteWarp& sw)
{
    const int64_t sbn = site_blocks(lat.L3);
    sw.g = lb / sbn;
    const int site = (int)((lb - sw.g * sbn) * kWarpsPerBlock + (threadIdx.x >> 5));
    if (site >= lat.L3) return false;
    sw.site = site;
    const Coord r = site_coord(lat, site);
    const int step[3] = {1, lat.L, lat.L2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        sw.nb[a] = site + ((r.x[a] + 1 == lat.L) ? step[a] * (1 - lat.L) : step[a]);
    return true;
}

// Offset of edge (d, site)'s 4x32 message block within a group.
__device__ __forceinline__ int msg_off(int site, int d) { return (site * 3 + d) * (4 * kLanes); }

// The 32-sample half word of face (n, site)'s syndrome for group g.
__device__ __forceinline__ uint32_t syndrome_half(const uint64_t* s, const Lattice& lat, int64_t W,
                                                  int n, int site, int64_t g)
{
    const uint64_t w = s[((int64_t)n * lat.L3 + site) * W + (g >> 1)];
    return (uint32_t)(w >> ((g & 1) * 32));
}

// Where an iteration takes the syndrome from: the caller's bit-sliced words
// (kSynWords), the same and also a per-group copy for later iterations
// (kSynWordsSave: uint4 per site and group, faces 0..2 in .x .y .z), or that
// copy (kSynSaved), which puts the three faces' bits in one 16-byte load.
enum SynMode { kSynWords = 0, kSynWordsSave = 1, kSynSaved = 2 };

// One flooding iteration for the three faces of a site: Eq. 3 (variable->check
// inputs, each the prior plus the three messages of its edge other than the
// face's own slot, which is not read) and Eq. 2 (check->variable) into msg_out.
// msg_in == nullptr is the first iteration: every input is the prior l0.
template <int kSyn>
__global__ void __launch_bounds__(kBpThreads, 6)
k_bp_step(const __grid_constant__ ItemTable tab, float l0, TD q)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
    const Lattice lat = d.lat;
    const int64_t W = d.W;
    const uint64_t* __restrict__ s = d.s;
    uint4* __restrict__ syn = d.syn;
    const float* __restrict__ msg_in = d.msg_in;
    float* __restrict__ msg_out = d.msg_out;
    SiteWarp sw;
    if (!site_warp(lat, lb, sw)) return;
    const int lane = threadIdx.x & 31;
    uint4 sh;
    if (kSyn == kSynSaved) {
        sh = syn[sw.g * lat.L3 + sw.site];
    } else {
        sh.x = syndrome_half(s, lat, W, 0, sw.site, sw.g);
        sh.y = syndrome_half(s, lat, W, 1, sw.site, sw.g);
        sh.z = syndrome_half(s, lat, W, 2, sw.site, sw.g);
        sh.w = 0;
        if (kSyn == kSynWordsSave && lane == 0) syn[sw.g * lat.L3 + sw.site] = sh;
    }
    const int64_t gbase = sw.g * (int64_t)lat.L3 * (3 * 4 * kLanes) + lane;
    const int r = sw.site, rx = sw.nb[0], ry = sw.nb[1], rz = sw.nb[2];
    // message blocks: edges at r (x, y, z) and the six neighbours used
    const int oXr = msg_off(r, 0), oYr = msg_off(r, 1), oZr = msg_off(r, 2);
    const int oXy = msg_off(ry, 0), oXz = msg_off(rz, 0);
    const int oYx = msg_off(rx, 1), oYz = msg_off(rz, 1);
    const int oZx = msg_off(rx, 2), oZy = msg_off(ry, 2);
    // inputs x[face][edge] in face_edges order
    float in0[4], in1[4], in2[4];
    if (msg_in) {
        const float* m = msg_in + gbase;
#define MSG(o, k) m[(o) + (k) * kLanes]
        const float xr0 = MSG(oXr, 0), xr1 = MSG(oXr, 1), xr2 = MSG(oXr, 2), xr3 = MSG(oXr, 3);
        const float yr0 = MSG(oYr, 0), yr1 = MSG(oYr, 1), yr2 = MSG(oYr, 2), yr3 = MSG(oYr, 3);
        const float zr0 = MSG(oZr, 0), zr1 = MSG(oZr, 1), zr2 = MSG(oZr, 2), zr3 = MSG(oZr, 3);
        const float xs = l0 + xr1 + xr3, ys = l0 + yr1 + yr3, zs = l0 + zr1 + zr3;
        // face 0: (y,r) excl 2, (y,r+z) excl 3, (z,r) excl 2, (z,r+y) excl 3
        in0[0] = ys + yr0;
        in0[1] = l0 + MSG(oYz, 0) + MSG(oYz, 1) + MSG(oYz, 2);
        in0[2] = zs + zr0;
        in0[3] = l0 + MSG(oZy, 0) + MSG(oZy, 1) + MSG(oZy, 2);
        // face 1: (x,r) excl 2, (x,r+z) excl 3, (z,r) excl 0, (z,r+x) excl 1
        in1[0] = xs + xr0;
        in1[1] = l0 + MSG(oXz, 0) + MSG(oXz, 1) + MSG(oXz, 2);
        in1[2] = zs + zr2;
        in1[3] = l0 + MSG(oZx, 0) + MSG(oZx, 2) + MSG(oZx, 3);
        // face 2: (x,r) excl 0, (x,r+y) excl 1, (y,r) excl 0, (y,r+x) excl 1
        in2[0] = xs + xr2;
        in2[1] = l0 + MSG(oXy, 0) + MSG(oXy, 2) + MSG(oXy, 3);
        in2[2] = ys + yr2;
        in2[3] = l0 + MSG(oYx, 0) + MSG(oYx, 2) + MSG(oYx, 3);
#undef MSG
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) in0[j] = in1[j] = in2[j] = l0;
    }
    float y[4];
    float* o = msg_out + gbase;
    // the new messages are not read again in this launch: store them evict-first
#define PUT(off, v) __stcs(o + (off), (v))
    check_node(in0, (sh.x >> lane) & 1u, q, y);
    PUT(oYr + 2 * kLanes, y[0]);
    PUT(oYz + 3 * kLanes, y[1]);
    PUT(oZr + 2 * kLanes, y[2]);
    PUT(oZy + 3 * kLanes, y[3]);
    check_node(in1, (sh.y >> lane) & 1u, q, y);
    PUT(oXr + 2 * kLanes, y[0]);
    PUT(oXz + 3 * kLanes, y[1]);
    PUT(oZr + 0 * kLanes, y[2]);
    PUT(oZx + 1 * kLanes, y[3]);
    check_node(in2, (sh.z >> lane) & 1u, q, y);
    PUT(oXr + 0 * kLanes, y[0]);
    PUT(oXy + 1 * kLanes, y[1]);
    PUT(oYr + 0 * kLanes, y[2]);
    PUT(oYx + 1 * kLanes, y[3]);
#undef PUT
    });
}

// Eq. 4 posterior and the hard decision for the three edges at a site (the
// edges this site's faces own): l = l0 + the four incoming messages, d = [l < 0].
// The warp XORs d into e at r and, for each face at r, the parity of its four
// edges' decisions into s (each 32-sample half word has exactly one writer).
__global__ void __launch_bounds__(kBpThreads)
k_bp_decide(const __grid_constant__ ItemTable tab, float l0)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
    const Lattice lat = d.lat;
    const int64_t W = d.W;
    const int64_t n_samples = d.n_samples;
    const float* __restrict__ msg = d.msg_in;
    uint32_t* __restrict__ e32 = reinterpret_cast<uint32_t*>(d.e);
    uint32_t* __restrict__ s32 = reinterpret_cast<uint32_t*>(d.s);
    float* __restrict__ llr_out = d.llr;
    SiteWarp sw;
    if (!site_warp(lat, lb, sw)) return;
    const int lane = threadIdx.x & 31;
    const int64_t sample = sw.g * kLanes + lane;
    const bool valid = sample < n_samples;
    const int64_t gbase = sw.g * (int64_t)lat.L3 * (3 * 4 * kLanes) + lane;
    auto post = [&](int site, int d) {
        float l = l0;
        if (msg) {
            const float* m = msg + gbase + msg_off(site, d);
            l += m[0];
            l += m[kLanes];
            l += m[2 * kLanes];
            l += m[3 * kLanes];
        }
        return l;
    };
    const int r = sw.site;
    float lr[3];
    unsigned dr[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lr[d] = post(r, d);
        dr[d] = __ballot_sync(0xffffffffu, valid && lr[d] < 0.0f);
    }
    const unsigned dXy = __ballot_sync(0xffffffffu, valid && post(sw.nb[1], 0) < 0.0f);
    const unsigned dXz = __ballot_sync(0xffffffffu, valid && post(sw.nb[2], 0) < 0.0f);
    const unsigned dYx = __ballot_sync(0xffffffffu, valid && post(sw.nb[0], 1) < 0.0f);
    const unsigned dYz = __ballot_sync(0xffffffffu, valid && post(sw.nb[2], 1) < 0.0f);
    const unsigned dZx = __ballot_sync(0xffffffffu, valid && post(sw.nb[0], 2) < 0.0f);
    const unsigned dZy = __ballot_sync(0xffffffffu, valid && post(sw.nb[1], 2) < 0.0f);
    const unsigned par[3] = {dr[1] ^ dYz ^ dr[2] ^ dZy, dr[0] ^ dXz ^ dr[2] ^ dZx,
                             dr[0] ^ dXy ^ dr[1] ^ dYx};
    const int64_t half = 2 * (sw.g >> 1) + (sw.g & 1);
    if (lane < 3) {
        const int64_t idx = 2 * ((int64_t)lane * lat.L3 + r) * W + half;
        if (par[lane]) s32[idx] ^= par[lane];
        if (dr[lane]) e32[idx] ^= dr[lane];
    }
    if (llr_out && valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) llr_out[((int64_t)d * lat.L3 + r) * n_samples + sample] = lr[d];
    }
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

int64_t group_floats(int L) { return 3LL * L * L * L * 4 * kLanes; }
int64_t group_syn(int L) { return (int64_t)L * L * L; }  // uint4 per site

void set_blocks(ItemTable& tab)
{
    for (int i = 0; i < tab.n; ++i) tab.it[i].blocks = site_blocks(tab.it[i].lat.L3) * tab.it[i].groups;
    finish_table(tab);
}

t3d_status launch_step(ItemTable& tab, int mode, double p, double q_meas, cudaStream_t st)
{
    set_blocks(tab);
    const int64_t blocks = tab.prefix[tab.n];
    ProfScope prof(T3D_K_BP_STEP, st);
    if (mode == kSynWordsSave)
        k_bp_step<kSynWordsSave><<<persistent_grid((const void*)k_bp_step<kSynWordsSave>, kBpThreads,
                                                   T3D_K_BP_STEP, blocks),
                                   kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas));
    else if (mode == kSynSaved)
        k_bp_step<kSynSaved><<<persistent_grid((const void*)k_bp_step<kSynSaved>, kBpThreads, T3D_K_BP_STEP,
                                               blocks),
                               kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas));
    else
        k_bp_step<kSynWords><<<persistent_grid((const void*)k_bp_step<kSynWords>, kBpThreads, T3D_K_BP_STEP,
                                               blocks),
                               kBpThreads, 0, st>>>(tab, prior(p), meas_pair(q_meas));
    T3D_LAUNCH_CHECK("bp step");
    return T3D_OK;
}

t3d_status launch_decide(ItemTable& tab, double p, cudaStream_t st)
{
    set_blocks(tab);
    ProfScope prof(T3D_K_BP_DECIDE, st);
    k_bp_decide<<<persistent_grid((const void*)k_bp_decide, kBpThreads, T3D_K_BP_DECIDE, tab.prefix[tab.n]),
                  kBpThreads, 0, st>>>(tab, prior(p));
    T3D_LAUNCH_CHECK("bp decide");
    return T3D_OK;
}

}  // namespace

size_t bp_bytes_per_group(int L)
{
    return 2 * (size_t)group_floats(L) * sizeof(float) + (size_t)group_syn(L) * sizeof(uint4);
}

// Chunks of chunk_groups groups; buf holds two chunk-sized message buffers
// followed by the chunk's saved syndrome words.
// The s/e words of chunk c start at group c*chunk_groups, so the kernels see
// the chunk's slice of the arrays through offset pointers and a local group
// count (groups are aligned to 64-sample words when chunk_groups is even).
namespace {

// Items' round-r chunks (items with no groups left are dropped); A and B are
// each chunk's two message buffers.
int64_t bp_rounds(const ItemTable& items, const int64_t* chunk_groups)
{
    int64_t rounds = 0;
    for (int i = 0; i < items.n; ++i) {
        const int64_t G = groups_for(items.it[i].n_samples);
        rounds = std::max(rounds, (G + chunk_groups[i] - 1) / chunk_groups[i]);
    }
    return rounds;
}

ItemTable chunk_table(const ItemTable& items, float* const* bufs, const int64_t* chunk_groups, int64_t r,
                      float* llr_out, float** A, float** B)
{
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    for (int i = 0; i < items.n; ++i) {
        const ItemDesc& src = items.it[i];
        const int64_t G = groups_for(src.n_samples);
        const int64_t g0 = r * chunk_groups[i];
        if (g0 >= G) continue;
        const int64_t gc = std::min(chunk_groups[i], G - g0);
        const int64_t w0 = g0 / 2;  // chunks start on 64-sample words (even g0)
        const int k = tab.n++;
        ItemDesc& d = tab.it[k];
        d = src;
        d.e = src.e + w0;
        d.s = src.s + w0;
        d.g0 = g0;
        d.groups = gc;
        d.n_samples = std::min<int64_t>(gc * kLanes, src.n_samples - g0 * kLanes);
        const int64_t fl = chunk_groups[i] * group_floats(src.lat.L);
        A[k] = bufs[i];
        B[k] = bufs[i] + fl;
        d.syn = reinterpret_cast<uint4*>(bufs[i] + 2 * fl);
        d.llr = (llr_out && items.n == 1) ? llr_out + g0 * kLanes : nullptr;
    }
    return tab;
}

}  // namespace

t3d_status launch_bp(const ItemTable& items, double p, double q_meas, int iters, float* const* bufs,
                     const int64_t* chunk_groups, float* llr_out, cudaStream_t st)
{
    // in round r item i processes groups [r*chunk_i, (r+1)*chunk_i)
    const int64_t rounds = bp_rounds(items, chunk_groups);
    for (int64_t r = 0; r < rounds; ++r) {
        float* A[kMaxItems];
        float* B[kMaxItems];
        ItemTable tab = chunk_table(items, bufs, chunk_groups, r, llr_out, A, B);
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
                       const int64_t* chunk_groups, cudaStream_t st, int* best_cap, float* best_ms)
{
    float* A[kMaxItems];
    float* B[kMaxItems];
    ItemTable tab = chunk_table(items, bufs, chunk_groups, 0, nullptr, A, B);
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
    return (size_t)groups_for(n_samples) * (size_t)group_floats(L) * sizeof(float);
}

extern "C" size_t toric3d_bp_workspace_bytes(int L, int64_t chunk_samples)
{
    if (L < 2 || L > kMaxL || chunk_samples < 1) return 0;
    int64_t g = groups_for(chunk_samples);
    g += g & 1;  // chunks hold whole 64-sample words
    return (size_t)g * bp_bytes_per_group(L);
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
    d.groups = groups_for(n_samples);
    return launch_step(tab, kSynWords, p, q_meas, as_stream(stream));
}

extern "C" t3d_status toric3d_bp_decide(int L, int64_t n_samples, const float* msg, double p,
                                        uint64_t* e, uint64_t* s, float* llr_out,
                                        t3d_stream stream)
{
    clear_error();
    T3D_TRY(bp_common_checks(L, n_samples, p, 0.0));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(msg == nullptr || aligned(msg, 16), "msg must be 16-byte aligned");
    T3D_REQUIRE(llr_out == nullptr || aligned(llr_out, 4), "llr_out must be 4-byte aligned");
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
    d.groups = groups_for(n_samples);
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
    int64_t chunk = (int64_t)(work_bytes / bp_bytes_per_group(L));
    const int64_t G = groups_for(n_samples);
    if (chunk < G) chunk &= ~1LL;  // partial chunks must cover whole 64-sample words
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
