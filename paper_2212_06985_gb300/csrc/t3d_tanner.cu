// The decoders on a generic Tanner graph (Sec. 5 asks whether they carry
// over to other LDPC codes): phenomenological noise, noisy syndrome
// measurement, the parallel flip and p-flip rules stated per variable
// (Sec. 3.1: flip on a strict majority of unsatisfied checks; Sec. 3.2: a
// coin decides ties) and product-sum BP with one prior per variable
// (Sec. 4.1, Eqs. 1-4).
//
// Bit-sliced state as on the toric code: e uint64[n][W], s uint64[m][W], 64
// samples per word.  A bit-sliced kernel thread owns (index, word); blocks
// are 32 words x 8 indices.  The rule kernel keeps a vertical (bit-sliced)
// counter of unsatisfied checks per variable and compares it with the
// degree's majority and tie values; one thread decides four consecutive
// variables, which share their coins (word v mod 4 of the coin stream keyed
// v / 4: two Philox blocks).  BP messages are FP32 on the Tanner edges in CSR
// order, samples innermost ([edge][S]), double-buffered; an iteration is a
// variable pass (totals T_v = prior_v + sum of incoming messages) and a
// check pass (inputs T_v - M_{c->v}), four samples per thread, with the
// check node specialised for degrees up to 8 and a loop beyond.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "t3d_bp_math.cuh"
#include "t3d_device.cuh"
#include "t3d_host.hpp"

namespace t3d {
namespace tg {
namespace {

using bpm::check_node;
using bpm::comp;
using bpm::ld4;
using bpm::st4;

constexpr int kMaxDeg = 32;          // largest variable and check degree accepted
constexpr int kCounterBits = 6;      // counts 0..32
constexpr int kThreads = 256;

struct G {
    int64_t n, m;
    const int32_t* cptr;
    const int32_t* cvar;
    const int32_t* vptr;
    const int32_t* vedge;
    const int32_t* vcheck;
};

G view(const t3d_tanner& g) { return G{g.n_vars, g.n_checks, g.cptr, g.cvar, g.vptr, g.vedge, g.vcheck}; }

// (index, word) of a bit-sliced thread: blocks of tx words x ty indices, 256 threads,
// tx = min(32, W rounded up to a power of two) so that few word lanes idle.
__device__ __forceinline__ bool index_word(int64_t count, int64_t W, int64_t& i, int64_t& w)
{
    i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    w = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    return i < count && w < W;
}

dim3 bs_block(int64_t W)
{
    unsigned tx = 1;
    while (tx < 32 && tx < W) tx *= 2;
    return dim3(tx, kThreads / tx);
}

dim3 bs_grid(int64_t count, int64_t W)
{
    const dim3 b = bs_block(W);
    return dim3((unsigned)((count + b.y - 1) / b.y), (unsigned)((W + b.x - 1) / b.x));
}

__global__ void k_tg_noise(const G g, int64_t W, uint64_t* __restrict__ e, uint64_t thr, uint64_t seed,
                           uint64_t group0, uint32_t cycle)
{
    int64_t v, w;
    if (!index_word(g.n, W, v, w)) return;
    const uint64_t flips = bernoulli_word(thr, seed, kStreamQubit, (uint64_t)v, cycle, 0, group0 + w);
    if (flips) e[v * W + w] ^= flips;
}

// s_c = XOR of its variables, then ^= Bernoulli(q) keyed by the check index.
__global__ void k_tg_syndrome(const G g, int64_t W, const uint64_t* __restrict__ e, uint64_t* __restrict__ s,
                              uint64_t thr, uint64_t seed, uint64_t group0, uint32_t cycle)
{
    int64_t c, w;
    if (!index_word(g.m, W, c, w)) return;
    uint64_t acc = 0;
    for (int32_t t = g.cptr[c]; t < g.cptr[c + 1]; ++t) acc ^= e[(int64_t)g.cvar[t] * W + w];
    s[c * W + w] = acc ^ bernoulli_word(thr, seed, kStreamMeas, (uint64_t)c, cycle, 0, group0 + w);
}

// Lanes where the bit-sliced counter u (cnt[0] least significant) is > K and == K.
__device__ __forceinline__ void compare_const(const uint64_t (&cnt)[kCounterBits], int K, uint64_t& gt, uint64_t& eq)
{
    gt = 0;
    eq = ~0ULL;
#pragma unroll
    for (int b = kCounterBits - 1; b >= 0; --b) {
        if ((K >> b) & 1) {
            eq &= cnt[b];
        } else {
            gt |= eq & cnt[b];
            eq &= ~cnt[b];
        }
    }
}

// One rule application's decisions for variables 4q .. 4q+3 of word w: flip words
// into f, e ^= f.  Majority: u > deg - u; tie (p-flip only): u == deg - u.
__global__ void k_tg_decide(const G g, int64_t W, uint64_t* __restrict__ e, const uint64_t* __restrict__ s,
                            uint64_t* __restrict__ f, int probabilistic, uint64_t seed, uint64_t group0,
                            uint32_t cycle, uint32_t sweep)
{
    int64_t q, w;
    if (!index_word((g.n + 3) / 4, W, q, w)) return;
    U64x4 coins;
    if (probabilistic) coins = coin_words(seed, (uint64_t)q, cycle, sweep, group0 + w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t v = 4 * q + k;
        if (v >= g.n) continue;
        const int32_t t0 = g.vptr[v], deg = g.vptr[v + 1] - t0;
        uint64_t cnt[kCounterBits] = {0, 0, 0, 0, 0, 0};
        for (int32_t j = 0; j < deg; ++j) {
            uint64_t carry = s[(int64_t)g.vcheck[t0 + j] * W + w];
#pragma unroll
            for (int b = 0; b < kCounterBits; ++b) {
                const uint64_t nb = cnt[b] ^ carry;
                carry &= cnt[b];
                cnt[b] = nb;
            }
        }
        // 2u > deg  <=>  u > floor(deg / 2) for either parity of deg; a tie
        // (2u == deg) exists only for even deg and is u == deg / 2
        uint64_t gt, eq;
        compare_const(cnt, deg / 2, gt, eq);
        uint64_t flip = gt;
        if (probabilistic && deg > 0 && !(deg & 1)) flip |= eq & coins.v[k];
        f[v * W + w] = flip;
        if (flip) e[v * W + w] ^= flip;
    }
}

// s_c ^= XOR of the flip words of its variables (nw words; row strides sW and fW).
__global__ void k_tg_apply(const G g, int64_t nw, uint64_t* __restrict__ s, int64_t sW, const uint64_t* __restrict__ f,
                           int64_t fW)
{
    int64_t c, w;
    if (!index_word(g.m, nw, c, w)) return;
    uint64_t acc = 0;
    for (int32_t t = g.cptr[c]; t < g.cptr[c + 1]; ++t) acc ^= f[(int64_t)g.cvar[t] * fW + w];
    if (acc) s[c * sW + w] ^= acc;
}

// ------------------------------------------------------------------ BP
struct BpArgs {
    G g;
    int64_t S;            // padded samples of the chunk (multiple of 64)
    int64_t W;            // row stride of the bit-sliced arrays
    const uint64_t* s;    // chunk's first word at column 0
    const float* prior;   // [n]
    float* T;             // [n][S]
    const float* in;      // [E][S]
    float* out;           // [E][S]
};

__device__ __forceinline__ int64_t quad_sample() { return ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * 4; }


// T_v = prior_v + sum of the messages into v (Eq. 3 / Eq. 4 without the leave-one-out).
__global__ void __launch_bounds__(kThreads) k_tg_totals(const BpArgs a)
{
    const int64_t smp = quad_sample(), v = blockIdx.x;
    if (smp >= a.S) return;
    const float p = a.prior[v];
    float4 t = make_float4(p, p, p, p);
    for (int32_t k = a.g.vptr[v]; k < a.g.vptr[v + 1]; ++k) {
        const float4 m = ld4(a.in, a.g.vedge[k], a.S, smp);
        t = make_float4(t.x + m.x, t.y + m.y, t.z + m.z, t.w + m.w);
    }
    st4(a.T, v, a.S, smp, t);
}

__device__ __forceinline__ uint32_t syn_bits4(const BpArgs& a, int64_t c, int64_t smp)
{
    return (uint32_t)(a.s[c * a.W + (smp >> 6)] >> (smp & 63)) & 0xFu;
}


template <int K>
__device__ __forceinline__ void check_quad(const BpArgs& a, int64_t c, int32_t t0, int64_t smp)
{
    float4 x4[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 T = ld4(a.T, a.g.cvar[t0 + k], a.S, smp), M = ld4(a.in, t0 + k, a.S, smp);
        x4[k] = make_float4(T.x - M.x, T.y - M.y, T.z - M.z, T.w - M.w);
    }
    const uint32_t syn = syn_bits4(a, c, smp);
    float o4[K][4];
#pragma unroll
    for (int cpt = 0; cpt < 4; ++cpt) {
        float x[K], o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] = comp(x4[k], cpt);
        check_node<K>(x, (syn >> cpt) & 1u, o);
#pragma unroll
        for (int k = 0; k < K; ++k) o4[k][cpt] = o[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) st4(a.out, t0 + k, a.S, smp, make_float4(o4[k][0], o4[k][1], o4[k][2], o4[k][3]));
}

// Degrees above 8: the same arithmetic one sample at a time, prefix pairs in a local array.
__device__ void check_loop(const BpArgs& a, int64_t c, int32_t t0, int deg, int64_t smp)
{
    const uint32_t syn4 = syn_bits4(a, c, smp);
    for (int cpt = 0; cpt < 4; ++cpt) {
        const int64_t sm = smp + cpt;
        bpm::TD pre[kMaxDeg];
        uint32_t sgn_all = ((syn4 >> cpt) & 1u) ? 0x80000000u : 0u;
        bpm::TD run{1.0f, 0.0f};
        for (int k = 0; k < deg; ++k) {
            const float x = a.T[(int64_t)a.g.cvar[t0 + k] * a.S + sm] - a.in[(int64_t)(t0 + k) * a.S + sm];
            sgn_all ^= __float_as_uint(x);
            pre[k] = run;
            run = bpm::td_mul(run, bpm::td_of(x));
        }
        bpm::TD suf{1.0f, 0.0f};
        for (int k = deg - 1; k >= 0; --k) {
            const float x = a.T[(int64_t)a.g.cvar[t0 + k] * a.S + sm] - a.in[(int64_t)(t0 + k) * a.S + sm];
            const bpm::TD o = bpm::td_mul(pre[k], suf);
            const float mag = fminf(bpm::two_atanh(o.t, o.d), bpm::kCheckClamp);
            const uint32_t sgn = (sgn_all ^ __float_as_uint(x)) & 0x80000000u;
            a.out[(int64_t)(t0 + k) * a.S + sm] = __uint_as_float(__float_as_uint(mag) | sgn);
            suf = bpm::td_mul(bpm::td_of(x), suf);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_tg_checks(const BpArgs a)
{
    const int64_t smp = quad_sample(), c = blockIdx.x;
    if (smp >= a.S) return;
    const int32_t t0 = a.g.cptr[c];
    const int deg = a.g.cptr[c + 1] - t0;
    switch (deg) {
        case 0: break;
        case 1: check_quad<1>(a, c, t0, smp); break;
        case 2: check_quad<2>(a, c, t0, smp); break;
        case 3: check_quad<3>(a, c, t0, smp); break;
        case 4: check_quad<4>(a, c, t0, smp); break;
        case 5: check_quad<5>(a, c, t0, smp); break;
        case 6: check_quad<6>(a, c, t0, smp); break;
        case 7: check_quad<7>(a, c, t0, smp); break;
        case 8: check_quad<8>(a, c, t0, smp); break;
        default: check_loop(a, c, t0, deg, smp); break;
    }
}

// Posterior decision of variable v for 32 samples per ballot: d = [T_v < 0] into the
// decision words (as e's layout), e ^= d; optional posteriors.
__global__ void __launch_bounds__(kThreads) k_tg_decide_bp(const BpArgs a, int64_t n_valid, uint64_t* __restrict__ e,
                                                            uint64_t* __restrict__ d, int64_t dW,
                                                            float* __restrict__ llr, int64_t llr_stride)
{
    const int64_t smp = (int64_t)blockIdx.y * kThreads + threadIdx.x, v = blockIdx.x;
    if (smp >= a.S) return;   // S is a multiple of 64: whole warps
    const float l = a.T[v * a.S + smp];
    const bool valid = smp < n_valid;
    const uint32_t bits = __ballot_sync(0xffffffffu, valid && l < 0.0f);
    if ((threadIdx.x & 31) == 0) {
        const int64_t word = smp >> 6, half = (smp >> 5) & 1;
        reinterpret_cast<uint32_t*>(d + v * dW + word)[half] = bits;
        if (bits) reinterpret_cast<uint32_t*>(e + v * a.W + word)[half] ^= bits;
    }
    if (llr && valid) llr[v * llr_stride + smp] = l;
}

unsigned quad_threads(int64_t S) { return (unsigned)std::min<int64_t>(kThreads, (S / 4 + 31) / 32 * 32); }

unsigned quad_blocks(int64_t S) { return (unsigned)((S / 4 + quad_threads(S) - 1) / quad_threads(S)); }

t3d_status launch_bp_iteration(BpArgs& a, const float* in, float* out, cudaStream_t st)
{
    a.in = in;
    a.out = out;
    ProfScope prof(T3D_K_BP_STEP, st);
    k_tg_totals<<<dim3((unsigned)a.g.n, quad_blocks(a.S)), quad_threads(a.S), 0, st>>>(a);
    T3D_LAUNCH_CHECK("Tanner BP totals");
    k_tg_checks<<<dim3((unsigned)a.g.m, quad_blocks(a.S)), quad_threads(a.S), 0, st>>>(a);
    T3D_LAUNCH_CHECK("Tanner BP checks");
    return T3D_OK;
}

size_t bp_bytes_per_word(const t3d_tanner& g)
{
    // T [n][64] + two message sets [E][64] (FP32) + decision words [n]
    return 64 * sizeof(float) * (size_t)(g.n_vars + 2 * g.n_edges) + 8 * (size_t)g.n_vars + 4 * 256;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

t3d_status check_graph(const t3d_tanner* g)
{
    T3D_REQUIRE(g != nullptr && g->cptr && g->cvar && g->vptr && g->vedge && g->vcheck,
                "graph is NULL or not prepared (toric3d_tanner_prepare)");
    T3D_REQUIRE(g->n_vars >= 1 && g->n_checks >= 1 && g->n_vars < (1LL << 31) && g->n_checks < (1LL << 31),
                "graph sizes out of range");
    return T3D_OK;
}

t3d_status check_samples(int64_t n_samples, int64_t words_limit)
{
    T3D_REQUIRE(n_samples >= 1 && words_for(n_samples) <= words_limit, "n_samples out of range");
    return T3D_OK;
}

}  // namespace
}  // namespace tg
}  // namespace t3d

using namespace t3d;
using namespace t3d::tg;

extern "C" size_t toric3d_tanner_bytes(int64_t n_vars, int64_t n_checks, int64_t n_edges)
{
    if (n_vars < 1 || n_checks < 1 || n_edges < 0) return 0;
    return round256(4 * (size_t)(n_checks + 1)) + round256(4 * (size_t)n_edges) + round256(4 * (size_t)(n_vars + 1)) +
           2 * round256(4 * (size_t)n_edges);
}

extern "C" t3d_status toric3d_tanner_prepare(int64_t n_vars, int64_t n_checks, const int32_t* cptr,
                                             const int32_t* cvar, void* blob, size_t blob_bytes, t3d_tanner* out)
{
    clear_error();
    T3D_REQUIRE(out != nullptr && cptr != nullptr, "cptr and out must not be NULL");
    T3D_REQUIRE(n_vars >= 1 && n_checks >= 1 && n_vars < (1LL << 31) && n_checks < (1LL << 31),
                "need 1 <= n_vars, n_checks < 2^31");
    T3D_REQUIRE(cptr[0] == 0, "cptr[0] must be 0");
    for (int64_t c = 0; c < n_checks; ++c) {
        T3D_REQUIRE(cptr[c + 1] >= cptr[c], "cptr must be non-decreasing (check %lld)", (long long)c);
        T3D_REQUIRE(cptr[c + 1] - cptr[c] <= kMaxDeg, "check %lld has degree %d > %d", (long long)c,
                    cptr[c + 1] - cptr[c], kMaxDeg);
    }
    const int64_t E = cptr[n_checks];
    T3D_REQUIRE(E >= 1 && E < (1LL << 31), "the graph needs 1 .. 2^31 - 1 edges");
    T3D_REQUIRE(cvar != nullptr, "cvar must not be NULL");
    T3D_REQUIRE(blob != nullptr && aligned(blob, 256), "blob must be a 256-byte aligned device pointer");
    T3D_REQUIRE(blob_bytes >= toric3d_tanner_bytes(n_vars, n_checks, E), "blob too small: %zu < %zu bytes",
                blob_bytes, toric3d_tanner_bytes(n_vars, n_checks, E));
    std::vector<int32_t> deg(n_vars + 1, 0);
    int32_t max_cdeg = 0;
    for (int64_t c = 0; c < n_checks; ++c) {
        max_cdeg = std::max(max_cdeg, cptr[c + 1] - cptr[c]);
        for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) {
            T3D_REQUIRE(cvar[t] >= 0 && cvar[t] < n_vars, "cvar[%d] = %d out of range", t, cvar[t]);
            for (int32_t u = cptr[c]; u < t; ++u)
                T3D_REQUIRE(cvar[u] != cvar[t], "check %lld lists variable %d twice", (long long)c, cvar[t]);
            deg[cvar[t] + 1]++;
        }
    }
    int32_t max_vdeg = 0;
    for (int64_t v = 0; v < n_vars; ++v) {
        max_vdeg = std::max(max_vdeg, deg[v + 1]);
        T3D_REQUIRE(deg[v + 1] <= kMaxDeg, "variable %lld has degree %d > %d", (long long)v, deg[v + 1], kMaxDeg);
        deg[v + 1] += deg[v];
    }
    // variable-major lists of (Tanner edge, check), checks ascending within a variable
    std::vector<int32_t> vptr(deg), vedge(E), vcheck(E), fill(deg.begin(), deg.end() - 1);
    for (int64_t c = 0; c < n_checks; ++c)
        for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) {
            const int32_t k = fill[cvar[t]]++;
            vedge[k] = t;
            vcheck[k] = (int32_t)c;
        }
    char* base = static_cast<char*>(blob);
    auto put = [&](const int32_t* src, size_t count) -> const int32_t* {
        char* dst = base;
        base += round256(4 * count);
        if (count && cudaMemcpy(dst, src, 4 * count, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return reinterpret_cast<const int32_t*>(dst);
    };
    t3d_tanner g;
    std::memset(&g, 0, sizeof(g));
    g.n_vars = n_vars;
    g.n_checks = n_checks;
    g.n_edges = E;
    g.max_var_degree = max_vdeg;
    g.max_check_degree = max_cdeg;
    g.cptr = put(cptr, n_checks + 1);
    g.cvar = put(cvar, E);
    g.vptr = put(vptr.data(), n_vars + 1);
    g.vedge = put(vedge.data(), E);
    g.vcheck = put(vcheck.data(), E);
    T3D_REQUIRE(g.cptr && g.cvar && g.vptr && g.vedge && g.vcheck, "copy of the graph to the device failed: %s",
                cudaGetErrorString(cudaGetLastError()));
    *out = g;
    return T3D_OK;
}

extern "C" t3d_status toric3d_tanner_noise(const t3d_tanner* g, int64_t n_samples, uint64_t* e, double p,
                                           uint64_t seed, uint64_t sample0, uint32_t cycle, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_graph(g));
    T3D_TRY(check_samples(n_samples, 65535LL * 32));
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(p >= 0.0 && p <= 1.0, "p must lie in [0, 1]");
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    const int64_t W = words_for(n_samples);
    cudaStream_t st = as_stream(stream);
    ProfScope prof(T3D_K_NOISE, st);
    k_tg_noise<<<bs_grid(g->n_vars, W), bs_block(W), 0, st>>>(view(*g), W, e, prob_threshold(p), seed, sample0 / 64,
                                                            cycle);
    T3D_LAUNCH_CHECK("Tanner noise");
    return T3D_OK;
}

extern "C" t3d_status toric3d_tanner_syndrome(const t3d_tanner* g, int64_t n_samples, const uint64_t* e,
                                              uint64_t* s, double q, uint64_t seed, uint64_t sample0, uint32_t cycle,
                                              t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_graph(g));
    T3D_TRY(check_samples(n_samples, 65535LL * 32));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(disjoint(e, (size_t)g->n_vars * words_for(n_samples) * 8, s, (size_t)g->n_checks * words_for(n_samples) * 8),
                "e and s must not overlap");
    T3D_REQUIRE(q >= 0.0 && q <= 1.0, "q must lie in [0, 1]");
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    const int64_t W = words_for(n_samples);
    cudaStream_t st = as_stream(stream);
    ProfScope prof(T3D_K_SYNDROME, st);
    k_tg_syndrome<<<bs_grid(g->n_checks, W), bs_block(W), 0, st>>>(view(*g), W, e, s, prob_threshold(q), seed,
                                                                 sample0 / 64, cycle);
    T3D_LAUNCH_CHECK("Tanner syndrome");
    return T3D_OK;
}

extern "C" size_t toric3d_tanner_flip_workspace_bytes(const t3d_tanner* g, int64_t n_samples)
{
    if (g == nullptr || n_samples < 1) return 0;
    return (size_t)g->n_vars * (size_t)words_for(n_samples) * 8;
}

extern "C" t3d_status toric3d_tanner_pflip(const t3d_tanner* g, int64_t n_samples, uint64_t* e, uint64_t* s,
                                           const char* schedule, int n_apply, uint32_t sweep0, uint64_t seed,
                                           uint64_t sample0, uint32_t cycle, void* work, size_t work_bytes,
                                           t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_graph(g));
    T3D_TRY(check_samples(n_samples, 65535LL * 32));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(disjoint(e, (size_t)g->n_vars * words_for(n_samples) * 8, s, (size_t)g->n_checks * words_for(n_samples) * 8),
                "e and s must not overlap");
    T3D_REQUIRE(n_apply >= 0, "n_apply must be >= 0");
    T3D_REQUIRE((uint64_t)sweep0 + (uint64_t)n_apply <= kMaxSweep, "sweep indices must stay below 2^22");
    const size_t slen = schedule ? strnlen(schedule, 64) : 0;
    T3D_REQUIRE(n_apply == 0 || (slen >= 1 && slen < 64), "n_apply > 0 needs a schedule of 1..63 letters");
    for (size_t i = 0; i < slen; ++i)
        T3D_REQUIRE(schedule[i] == 'F' || schedule[i] == 'P', "schedule may hold only 'F' and 'P'");
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    T3D_REQUIRE(work != nullptr && aligned(work, 8) && work_bytes >= toric3d_tanner_flip_workspace_bytes(g, n_samples),
                "work: >= %zu bytes, 8-byte aligned", toric3d_tanner_flip_workspace_bytes(g, n_samples));
    const int64_t W = words_for(n_samples);
    cudaStream_t st = as_stream(stream);
    uint64_t* f = static_cast<uint64_t*>(work);
    const G gv = view(*g);
    for (int k = 0; k < n_apply; ++k) {
        const bool prob = schedule[k % slen] == 'P';
        ProfScope prof(prob ? T3D_K_PFLIP : T3D_K_FLIP, st);
        k_tg_decide<<<bs_grid((g->n_vars + 3) / 4, W), bs_block(W), 0, st>>>(gv, W, e, s, f, prob ? 1 : 0, seed,
                                                                           sample0 / 64, cycle, sweep0 + k);
        T3D_LAUNCH_CHECK("Tanner rule decisions");
        k_tg_apply<<<bs_grid(g->n_checks, W), bs_block(W), 0, st>>>(gv, W, s, W, f, W);
        T3D_LAUNCH_CHECK("Tanner rule syndrome update");
    }
    return T3D_OK;
}

extern "C" size_t toric3d_tanner_bp_message_bytes(const t3d_tanner* g, int64_t n_samples)
{
    if (g == nullptr || n_samples < 1) return 0;
    return (size_t)g->n_edges * 64 * (size_t)words_for(n_samples) * sizeof(float);
}

extern "C" size_t toric3d_tanner_bp_workspace_bytes(const t3d_tanner* g, int64_t chunk_samples)
{
    if (g == nullptr || chunk_samples < 1) return 0;
    return (size_t)words_for(chunk_samples) * bp_bytes_per_word(*g);
}

extern "C" t3d_status toric3d_tanner_bp_step(const t3d_tanner* g, int64_t n_samples, const uint64_t* s,
                                             const float* prior, const float* msg_in, float* msg_out, void* work,
                                             size_t work_bytes, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_graph(g));
    T3D_TRY(check_samples(n_samples, 65535LL * kThreads / 64));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(prior != nullptr && aligned(prior, 4), "prior must be a device float array");
    T3D_REQUIRE(msg_in != nullptr && msg_out != nullptr && aligned(msg_in, 16) && aligned(msg_out, 16),
                "msg_in and msg_out must be 16-byte aligned device pointers");
    const size_t mb = toric3d_tanner_bp_message_bytes(g, n_samples);
    const char *ib = reinterpret_cast<const char*>(msg_in), *ob = reinterpret_cast<const char*>(msg_out);
    T3D_REQUIRE(ib + mb <= ob || ob + mb <= ib, "msg_in and msg_out must not overlap");
    const int64_t S = 64 * words_for(n_samples);
    T3D_REQUIRE(work != nullptr && aligned(work, 16) && work_bytes >= (size_t)g->n_vars * S * sizeof(float),
                "work: >= %zu bytes, 16-byte aligned", (size_t)g->n_vars * S * sizeof(float));
    BpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = view(*g);
    a.S = S;
    a.W = words_for(n_samples);
    a.s = s;
    a.prior = prior;
    a.T = static_cast<float*>(work);
    return launch_bp_iteration(a, msg_in, msg_out, as_stream(stream));
}

extern "C" t3d_status toric3d_tanner_bp(const t3d_tanner* g, int64_t n_samples, uint64_t* e, uint64_t* s,
                                        const float* prior, int iters, void* work, size_t work_bytes,
                                        float* llr_out, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_graph(g));
    T3D_TRY(check_samples(n_samples, 65535LL * 32));
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(disjoint(e, (size_t)g->n_vars * words_for(n_samples) * 8, s, (size_t)g->n_checks * words_for(n_samples) * 8),
                "e and s must not overlap");
    T3D_REQUIRE(prior != nullptr && aligned(prior, 4), "prior must be a device float array");
    T3D_REQUIRE(iters >= 0, "negative iteration count");
    T3D_REQUIRE(work != nullptr && aligned(work, 256), "work must be a 256-byte aligned device pointer");
    const int64_t words = words_for(n_samples), W = words;
    const int64_t chunk = std::min<int64_t>({words, (int64_t)(work_bytes / bp_bytes_per_word(*g)),
                                             65535LL * kThreads / 64});
    T3D_REQUIRE(chunk >= 1, "workspace too small: %zu bytes < %zu per 64-sample word", work_bytes,
                bp_bytes_per_word(*g));
    T3D_REQUIRE(llr_out == nullptr || chunk == words, "llr_out needs a workspace for all samples at once");
    cudaStream_t st = as_stream(stream);
    const G gv = view(*g);
    for (int64_t w0 = 0; w0 < words; w0 += chunk) {
        const int64_t cw = std::min(chunk, words - w0), S = 64 * cw;
        char* base = static_cast<char*>(work);
        auto take = [&](size_t bytes) {
            char* p = base;
            base += round256(bytes);
            return p;
        };
        float* T = reinterpret_cast<float*>(take((size_t)g->n_vars * S * 4));
        float* M[2] = {reinterpret_cast<float*>(take((size_t)g->n_edges * S * 4)),
                       reinterpret_cast<float*>(take((size_t)g->n_edges * S * 4))};
        uint64_t* d = reinterpret_cast<uint64_t*>(take((size_t)g->n_vars * cw * 8));
        T3D_CUDA_CHECK(cudaMemsetAsync(M[0], 0, (size_t)g->n_edges * S * 4, st));
        BpArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = gv;
        a.S = S;
        a.W = W;
        a.s = s + w0;
        a.prior = prior;
        a.T = T;
        for (int it = 0; it < iters; ++it) T3D_TRY(launch_bp_iteration(a, M[it & 1], M[(it + 1) & 1], st));
        a.in = M[iters & 1];
        ProfScope prof(T3D_K_BP_DECIDE, st);
        k_tg_totals<<<dim3((unsigned)g->n_vars, quad_blocks(S)), quad_threads(S), 0, st>>>(a);
        T3D_LAUNCH_CHECK("Tanner BP posteriors");
        k_tg_decide_bp<<<dim3((unsigned)g->n_vars, (unsigned)((S + kThreads - 1) / kThreads)), kThreads, 0, st>>>(
            a, std::min<int64_t>(S, n_samples - 64 * w0), e + w0, d, cw, llr_out, n_samples);
        T3D_LAUNCH_CHECK("Tanner BP decisions");
        k_tg_apply<<<bs_grid(g->n_checks, cw), bs_block(cw), 0, st>>>(gv, cw, s + w0, W, d, cw);
        T3D_LAUNCH_CHECK("Tanner BP syndrome update");
    }
    return T3D_OK;
}
