// Bit-sliced kernels (64 samples per uint64_t word, word index innermost):
// phenomenological noise, noisy syndrome measurement, synchronous flip /
// p-flip applications, logical readout, and layout conversion.
//
// Each thread owns one (site, word) pair; a warp covers 32 consecutive words
// of one site, so every global access is a coalesced 256-byte row and the
// periodic neighbours of a site sit at fixed word strides of the same row.
#include <cuda_runtime.h>

#include <cstring>

#include "t3d_device.cuh"
#include "t3d_host.hpp"

namespace t3d {
namespace {

constexpr int kThreads = 256;

struct SiteWordGrid {
    dim3 grid, block;
};

// x = words (coalesced), y = sites.
SiteWordGrid site_word_grid(int64_t n_sites, int64_t words)
{
    int tx = 32;
    while (tx > 1 && tx / 2 >= words) tx /= 2;
    int ty = kThreads / tx;
    SiteWordGrid g;
    g.block = dim3(tx, ty, 1);
    g.grid = dim3((unsigned)((n_sites + ty - 1) / ty), (unsigned)((words + tx - 1) / tx), 1);
    return g;
}

__device__ __forceinline__ bool site_word(int64_t n_sites, int64_t W, int& site, int64_t& w)
{
    w = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    site = (int)(blockIdx.x * blockDim.y + threadIdx.y);
    return w < W && site < n_sites;
}

// e ^= Bernoulli(p) for every edge (Sec. 3.1 phenomenological qubit noise).
__global__ void k_noise(Lattice lat, int64_t W, uint64_t* __restrict__ e, uint64_t thr,
                        uint64_t seed, uint64_t group0, uint32_t cycle)
{
    int v;
    int64_t w;
    if (!site_word(3LL * lat.L3, W, v, w)) return;
    uint64_t flips = bernoulli_word(thr, seed, kStreamQubit, (uint64_t)v, cycle, 0, group0 + w);
    if (flips) e[(int64_t)v * W + w] ^= flips;
}

// s_f = XOR of the face's four edges, then ^= Bernoulli(q) (Sec. 2, Sec. 3.1).
__global__ void k_syndrome(Lattice lat, int64_t W, const uint64_t* __restrict__ e,
                           uint64_t* __restrict__ s, uint64_t thr, uint64_t seed,
                           uint64_t group0, uint32_t cycle)
{
    int f;
    int64_t w;
    if (!site_word(3LL * lat.L3, W, f, w)) return;
    int n = f / lat.L3, site = f - n * lat.L3;
    FaceEdges fe = face_edges(lat, n, site_coord(lat, site));
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc ^= e[((int64_t)fe.dir[j] * lat.L3 + fe.site[j]) * W + w];
    acc ^= bernoulli_word(thr, seed, kStreamMeas, (uint64_t)f, cycle, 0, group0 + w);
    s[(int64_t)f * W + w] = acc;
}

// Periodic neighbour offsets of a site: step[a] and the +1 / -1 moves along
// each axis expressed as index deltas.
struct Moves {
    int plus[3];
    int minus[3];
};

__device__ __forceinline__ Moves site_moves(const Lattice& lat, int site)
{
    const Coord r = site_coord(lat, site);
    const int step[3] = {1, lat.L, lat.L2};
    Moves m;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.plus[a] = (r.x[a] + 1 == lat.L) ? step[a] * (1 - lat.L) : step[a];
        m.minus[a] = (r.x[a] == 0) ? step[a] * (lat.L - 1) : -step[a];
    }
    return m;
}

// One synchronous flip (or p-flip) application for the three faces at a site.
// The thread of site r decides the nine edges its faces touch -- (x,r), (y,r),
// (z,r), (x,r+e_y), (x,r+e_z), (y,r+e_x), (y,r+e_z), (z,r+e_x), (z,r+e_y) --
// each from its four faces in the old snapshot s_in, writes s_out at its three
// faces (old value XOR its four edges' flips) and applies the flips of the
// three edges at r to e.  Edge (a, r') lies on the faces with normal 3-a-c at
// r' and r' - e_c for the two axes c != a.
template <bool kProbabilistic>
__global__ void k_sweep(Lattice lat, int64_t W, uint64_t* __restrict__ e,
                        const uint64_t* __restrict__ s_in, uint64_t* __restrict__ s_out,
                        uint64_t seed, uint64_t group0, uint32_t cycle, uint32_t sweep)
{
    int r;
    int64_t w;
    if (!site_word(lat.L3, W, r, w)) return;
    const Moves mv = site_moves(lat, r);
    const int rx = r + mv.plus[0], ry = r + mv.plus[1], rz = r + mv.plus[2];
    const int64_t L3 = lat.L3;
    auto S = [&](int n, int site) { return s_in[((int64_t)n * L3 + site) * W + w]; };
    const uint64_t s0 = S(0, r), s1 = S(1, r), s2 = S(2, r);
    const uint64_t group = group0 + (uint64_t)w;
    auto decide = [&](uint64_t a, uint64_t b, uint64_t c, uint64_t d, int dir, int site) {
        uint64_t fl = at_least_three(a, b, c, d);
        if (kProbabilistic) {
            const uint64_t two = exactly_two(a, b, c, d);
            if (two) fl |= two & coin_word(seed, (uint64_t)dir * L3 + site, cycle, sweep, group);
        }
        return fl;
    };
    const uint64_t fx0 = decide(s2, S(2, r + mv.minus[1]), s1, S(1, r + mv.minus[2]), 0, r);
    const uint64_t fy0 = decide(s2, S(2, r + mv.minus[0]), s0, S(0, r + mv.minus[2]), 1, r);
    const uint64_t fz0 = decide(s1, S(1, r + mv.minus[0]), s0, S(0, r + mv.minus[1]), 2, r);
    const uint64_t fxy = decide(S(2, ry), s2, S(1, ry), S(1, ry + mv.minus[2]), 0, ry);
    const uint64_t fxz = decide(S(2, rz), S(2, rz + mv.minus[1]), S(1, rz), s1, 0, rz);
    const uint64_t fyx = decide(S(2, rx), s2, S(0, rx), S(0, rx + mv.minus[2]), 1, rx);
    const uint64_t fyz = decide(S(2, rz), S(2, rz + mv.minus[0]), S(0, rz), s0, 1, rz);
    const uint64_t fzx = decide(S(1, rx), s1, S(0, rx), S(0, rx + mv.minus[1]), 2, rx);
    const uint64_t fzy = decide(S(1, ry), S(1, ry + mv.minus[0]), S(0, ry), s0, 2, ry);
    s_out[((int64_t)0 * L3 + r) * W + w] = s0 ^ fy0 ^ fyz ^ fz0 ^ fzy;
    s_out[((int64_t)1 * L3 + r) * W + w] = s1 ^ fx0 ^ fxz ^ fz0 ^ fzx;
    s_out[((int64_t)2 * L3 + r) * W + w] = s2 ^ fx0 ^ fxy ^ fy0 ^ fyx;
    if (fx0) e[((int64_t)0 * L3 + r) * W + w] ^= fx0;
    if (fy0) e[((int64_t)1 * L3 + r) * W + w] ^= fy0;
    if (fz0) e[((int64_t)2 * L3 + r) * W + w] ^= fz0;
}

// Logical readout.  Block (32, 8): threadIdx.x = word of a 32-word tile,
// threadIdx.y splits the L^2 lines of each axis.  Line parities are summed
// per lane in a bit-sliced counter, partial counters are added in shared
// memory, and a lane fails axis d iff 2 c_d >= L^2.
constexpr int kCountBits = 17;  // L^2 <= 65536
constexpr int kLineSplit = 8;

__device__ __forceinline__ void counter_add_bit(uint64_t (&c)[kCountBits], uint64_t bit)
{
#pragma unroll
    for (int b = 0; b < kCountBits; ++b) {
        uint64_t carry = c[b] & bit;
        c[b] ^= bit;
        bit = carry;
    }
}

__global__ void __launch_bounds__(32 * kLineSplit)
k_logical(Lattice lat, int64_t W, int64_t n_samples, const uint64_t* __restrict__ e,
          uint8_t* __restrict__ mask, unsigned long long* __restrict__ counts8)
{
    __shared__ uint64_t part[kLineSplit][kCountBits][32];
    __shared__ uint64_t fail[3][32];
    __shared__ unsigned int hist[8];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t w = (int64_t)blockIdx.x * 32 + tx;
    if (tx < 8 && ty == 0) hist[tx] = 0;
    const int L = lat.L, L2 = lat.L2;
    for (int d = 0; d < 3; ++d) {
        const int u_axis = (d == 0) ? 1 : 0;
        const int v_axis = (d == 2) ? 1 : 2;
        uint64_t cnt[kCountBits];
#pragma unroll
        for (int b = 0; b < kCountBits; ++b) cnt[b] = 0;
        if (w < W) {
            for (int line = ty; line < L2; line += kLineSplit) {
                Coord r;
                r.x[u_axis] = line % L;
                r.x[v_axis] = line / L;
                uint64_t par = 0;
                for (int t = 0; t < L; ++t) {
                    r.x[d] = t;
                    par ^= e[((int64_t)d * lat.L3 + site_index(lat, r)) * W + w];
                }
                counter_add_bit(cnt, par);
            }
        }
#pragma unroll
        for (int b = 0; b < kCountBits; ++b) part[ty][b][tx] = cnt[b];
        __syncthreads();
        if (ty == 0) {
            uint64_t tot[kCountBits];
#pragma unroll
            for (int b = 0; b < kCountBits; ++b) tot[b] = part[0][b][tx];
            for (int k = 1; k < kLineSplit; ++k) {
                uint64_t carry = 0;
#pragma unroll
                for (int b = 0; b < kCountBits; ++b) {
                    uint64_t x = part[k][b][tx];
                    uint64_t sum = tot[b] ^ x ^ carry;
                    carry = (tot[b] & x) | (carry & (tot[b] ^ x));
                    tot[b] = sum;
                }
            }
            // lanes with count >= ceil(L^2 / 2)
            const unsigned need = (unsigned)(L2 + 1) / 2;
            uint64_t gt = 0, eq = ~0ULL;
#pragma unroll
            for (int b = kCountBits - 1; b >= 0; --b) {
                if ((need >> b) & 1u) {
                    eq &= tot[b];
                } else {
                    gt |= eq & tot[b];
                    eq &= ~tot[b];
                }
            }
            fail[d][tx] = gt | eq;
        }
        __syncthreads();
    }
    if (w < W) {
        for (int j = ty * 8; j < ty * 8 + 8; ++j) {
            int64_t sample = w * 64 + j;
            if (sample >= n_samples) break;
            unsigned m = (unsigned)((fail[0][tx] >> j) & 1ULL) |
                         ((unsigned)((fail[1][tx] >> j) & 1ULL) << 1) |
                         ((unsigned)((fail[2][tx] >> j) & 1ULL) << 2);
            if (mask) mask[sample] = (uint8_t)m;
            if (counts8) atomicAdd(&hist[m], 1u);
        }
    }
    __syncthreads();
    if (counts8 && ty == 0 && tx < 8 && hist[tx]) atomicAdd(&counts8[tx], (unsigned long long)hist[tx]);
}

__global__ void k_pack(int64_t n_bits, int64_t n_samples, int64_t W, const uint8_t* __restrict__ bits,
                       uint64_t* __restrict__ words)
{
    int64_t w = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (w >= W || i >= n_bits) return;
    uint64_t acc = 0;
    for (int j = 0; j < 64; ++j) {
        int64_t sample = w * 64 + j;
        if (sample >= n_samples) break;
        acc |= (uint64_t)(bits[sample * n_bits + i] & 1) << j;
    }
    words[i * W + w] = acc;
}

__global__ void k_unpack(int64_t n_bits, int64_t n_samples, int64_t W, const uint64_t* __restrict__ words,
                         uint8_t* __restrict__ bits)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t sample = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (i >= n_bits || sample >= n_samples) return;
    bits[sample * n_bits + i] = (uint8_t)((words[i * W + sample / 64] >> (sample % 64)) & 1ULL);
}

Lattice make_lattice(int L) { return make_lattice_host(L); }

}  // namespace

// ----------------------------------------------------------------- launchers
t3d_status launch_noise(int L, int64_t words, uint64_t* e, uint64_t thr, uint64_t seed,
                        uint64_t group0, uint32_t cycle, cudaStream_t st)
{
    if (thr == 0) return T3D_OK;
    auto g = site_word_grid(3LL * L * L * L, words);
    ProfScope prof(T3D_K_NOISE, st);
    k_noise<<<g.grid, g.block, 0, st>>>(make_lattice(L), words, e, thr, seed, group0, cycle);
    T3D_LAUNCH_CHECK("noise");
    return T3D_OK;
}

t3d_status launch_syndrome(int L, int64_t words, const uint64_t* e, uint64_t* s, uint64_t thr,
                           uint64_t seed, uint64_t group0, uint32_t cycle, cudaStream_t st)
{
    auto g = site_word_grid(3LL * L * L * L, words);
    ProfScope prof(T3D_K_SYNDROME, st);
    k_syndrome<<<g.grid, g.block, 0, st>>>(make_lattice(L), words, e, s, thr, seed, group0, cycle);
    T3D_LAUNCH_CHECK("syndrome");
    return T3D_OK;
}

t3d_status launch_sweeps(int L, int64_t words, uint64_t* e, uint64_t* s, uint64_t* tmp,
                         const char* schedule, int slen, int n_apply, uint32_t sweep0,
                         uint64_t seed, uint64_t group0, uint32_t cycle, cudaStream_t st)
{
    auto g = site_word_grid((int64_t)L * L * L, words);
    Lattice lat = make_lattice(L);
    uint64_t* bufs[2] = {s, tmp};
    for (int k = 0; k < n_apply; ++k) {
        const uint64_t* in = bufs[k & 1];
        uint64_t* out = bufs[(k + 1) & 1];
        const bool pk = schedule[k % slen] == 'P';
        ProfScope prof(pk ? T3D_K_PFLIP : T3D_K_FLIP, st);
        if (pk)
            k_sweep<true><<<g.grid, g.block, 0, st>>>(lat, words, e, in, out, seed, group0, cycle,
                                                       sweep0 + (uint32_t)k);
        else
            k_sweep<false><<<g.grid, g.block, 0, st>>>(lat, words, e, in, out, seed, group0, cycle,
                                                        sweep0 + (uint32_t)k);
        T3D_LAUNCH_CHECK("flip sweep");
    }
    if (n_apply & 1)
        T3D_CUDA_CHECK(cudaMemcpyAsync(s, tmp, (size_t)3 * L * L * L * words * sizeof(uint64_t),
                                       cudaMemcpyDeviceToDevice, st));
    return T3D_OK;
}

t3d_status launch_logical(int L, int64_t n_samples, const uint64_t* e, uint8_t* mask,
                          int64_t* counts8, cudaStream_t st)
{
    int64_t W = words_for(n_samples);
    if (counts8) T3D_CUDA_CHECK(cudaMemsetAsync(counts8, 0, 8 * sizeof(int64_t), st));
    dim3 block(32, kLineSplit);
    dim3 grid((unsigned)((W + 31) / 32));
    ProfScope prof(T3D_K_LOGICAL, st);
    k_logical<<<grid, block, 0, st>>>(make_lattice(L), W, n_samples, e, mask,
                                      reinterpret_cast<unsigned long long*>(counts8));
    T3D_LAUNCH_CHECK("logical");
    return T3D_OK;
}

}  // namespace t3d

using namespace t3d;

// ----------------------------------------------------------------- C ABI
extern "C" t3d_status toric3d_noise(int L, int64_t words, uint64_t* e, double p, uint64_t seed,
                                    uint64_t sample0, uint32_t cycle, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(p >= 0.0 && p <= 1.0, "p=%g outside [0,1]", p);
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    return launch_noise(L, words, e, prob_threshold(p), seed, sample0 / 64, cycle, as_stream(stream));
}

extern "C" t3d_status toric3d_syndrome(int L, int64_t words, const uint64_t* e, uint64_t* s,
                                       double q, uint64_t seed, uint64_t sample0, uint32_t cycle,
                                       t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE((const void*)e != (const void*)s, "e and s must not overlap");
    T3D_REQUIRE(q >= 0.0 && q <= 1.0, "q=%g outside [0,1]", q);
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    return launch_syndrome(L, words, e, s, prob_threshold(q), seed, sample0 / 64, cycle,
                           as_stream(stream));
}

extern "C" size_t toric3d_flip_workspace_bytes(int L, int64_t words)
{
    if (L < 2 || L > kMaxL || words < 1) return 0;
    return (size_t)3 * L * L * L * (size_t)words * sizeof(uint64_t);
}

static t3d_status sweeps_common(int L, int64_t words, uint64_t* e, uint64_t* s, const char* schedule,
                                int n_apply, uint32_t sweep0, uint64_t seed, uint64_t sample0,
                                uint32_t cycle, void* work, size_t work_bytes, t3d_stream stream)
{
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(n_apply >= 0, "negative number of applications");
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    if (n_apply == 0) return T3D_OK;
    T3D_REQUIRE(schedule != nullptr, "schedule is NULL");
    size_t slen = strnlen(schedule, 64);
    T3D_REQUIRE(slen >= 1 && slen <= 63, "schedule length must be 1..63");
    for (size_t i = 0; i < slen; ++i)
        T3D_REQUIRE(schedule[i] == 'F' || schedule[i] == 'P', "schedule may hold only 'F' and 'P'");
    T3D_REQUIRE(work != nullptr && aligned(work, 16), "work must be a 16-byte aligned device pointer");
    T3D_REQUIRE(work_bytes >= toric3d_flip_workspace_bytes(L, words), "workspace too small: %zu < %zu",
                work_bytes, toric3d_flip_workspace_bytes(L, words));
    return launch_sweeps(L, words, e, s, static_cast<uint64_t*>(work), schedule, (int)slen, n_apply,
                         sweep0, seed, sample0 / 64, cycle, as_stream(stream));
}

extern "C" t3d_status toric3d_flip(int L, int64_t words, uint64_t* e, uint64_t* s, int sweeps,
                                   void* work, size_t work_bytes, t3d_stream stream)
{
    clear_error();
    return sweeps_common(L, words, e, s, "F", sweeps, 0, 0, 0, 0, work, work_bytes, stream);
}

extern "C" t3d_status toric3d_pflip(int L, int64_t words, uint64_t* e, uint64_t* s,
                                    const char* schedule, int n_apply, uint32_t sweep0,
                                    uint64_t seed, uint64_t sample0, uint32_t cycle, void* work,
                                    size_t work_bytes, t3d_stream stream)
{
    clear_error();
    return sweeps_common(L, words, e, s, schedule, n_apply, sweep0, seed, sample0, cycle, work,
                         work_bytes, stream);
}

extern "C" t3d_status toric3d_logical(int L, int64_t n_samples, const uint64_t* e, uint8_t* mask,
                                      int64_t* counts8, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(n_samples >= 1 && words_for(n_samples) <= 65535LL * 32, "n_samples out of range");
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(counts8 == nullptr || aligned(counts8, 8), "counts8 must be 8-byte aligned");
    return launch_logical(L, n_samples, e, mask, counts8, as_stream(stream));
}

extern "C" t3d_status toric3d_pack(int64_t n_bits, int64_t n_samples, const uint8_t* bits,
                                   uint64_t* words, t3d_stream stream)
{
    clear_error();
    T3D_REQUIRE(n_bits >= 1 && n_samples >= 1, "empty input");
    T3D_REQUIRE(bits != nullptr, "bits is NULL");
    T3D_TRY(check_words(words, "words"));
    int64_t W = words_for(n_samples);
    T3D_REQUIRE(W <= 65535LL * 32, "n_samples out of range");
    auto g = site_word_grid(n_bits, W);
    ProfScope prof(T3D_K_LAYOUT, as_stream(stream));
    k_pack<<<g.grid, g.block, 0, as_stream(stream)>>>(n_bits, n_samples, W, bits, words);
    T3D_LAUNCH_CHECK("pack");
    return T3D_OK;
}

extern "C" t3d_status toric3d_unpack(int64_t n_bits, int64_t n_samples, const uint64_t* words,
                                     uint8_t* bits, t3d_stream stream)
{
    clear_error();
    T3D_REQUIRE(n_bits >= 1 && n_samples >= 1, "empty input");
    T3D_REQUIRE(bits != nullptr, "bits is NULL");
    T3D_TRY(check_words(words, "words"));
    int64_t W = words_for(n_samples);
    dim3 block(256);
    unsigned gy = (unsigned)std::min<int64_t>(n_samples, 65535);
    unsigned gz = (unsigned)((n_samples + gy - 1) / gy);
    dim3 grid((unsigned)((n_bits + 255) / 256), gy, gz);
    ProfScope prof(T3D_K_LAYOUT, as_stream(stream));
    k_unpack<<<grid, block, 0, as_stream(stream)>>>(n_bits, n_samples, W, words, bits);
    T3D_LAUNCH_CHECK("unpack");
    return T3D_OK;
}
