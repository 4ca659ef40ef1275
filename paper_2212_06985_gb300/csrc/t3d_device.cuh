// Device-side building blocks shared by the toric3d kernels: lattice index
// arithmetic for the periodic L^3 cubic lattice (Sec. 2 of arXiv:2212.06985,
// primal picture: qubits on edges, Z checks on faces), the Philox4x32-10
// counter-based generator and the bit-sliced Bernoulli comparator.
#pragma once

#include <cstdint>

namespace t3d {

// ----------------------------------------------------------------- lattice
// site = (z*L + y)*L + x; edge (d, site) = d*L^3 + site; face (n, site) = n*L^3 + site.
struct Lattice {
    int L;
    int L2;
    int L3;
    uint32_t magic;  // floor(2^32 / L) + 1: n / L == __umulhi(n, magic) for 0 <= n < 2^32 / L
};

inline Lattice make_lattice_host(int L)
{
    return Lattice{L, L * L, L * L * L, (uint32_t)((1ULL << 32) / (uint64_t)L + 1)};
}

// Exact n / L for 0 <= n < 2^24 (at most 256^3 sites): with magic = 2^32/L + eps,
// 0 < eps <= 1, n*magic/2^32 = n/L + n*eps/2^32 exceeds n/L by less than 1/L.
__device__ __forceinline__ int div_L(const Lattice& lat, int n)
{
    return (int)__umulhi((uint32_t)n, lat.magic);
}

struct Coord {
    int x[3];
};

__device__ __forceinline__ Coord site_coord(const Lattice& lat, int site)
{
    Coord r;
    int t = div_L(lat, site);
    r.x[0] = site - t * lat.L;
    int z = div_L(lat, t);
    r.x[1] = t - z * lat.L;
    r.x[2] = z;
    return r;
}

__device__ __forceinline__ int site_index(const Lattice& lat, const Coord& r)
{
    return (r.x[2] * lat.L + r.x[1]) * lat.L + r.x[0];
}

// r shifted by +1 or -1 along `axis`, periodic.
__device__ __forceinline__ Coord shifted(const Lattice& lat, Coord r, int axis, int delta)
{
    int v = r.x[axis] + delta;
    v = (v < 0) ? v + lat.L : (v >= lat.L ? v - lat.L : v);
    r.x[axis] = v;
    return r;
}

// The two in-plane axes a < b of a face with normal n.
__device__ __forceinline__ void plane_axes(int n, int& a, int& b)
{
    a = (n == 0) ? 1 : 0;
    b = (n == 2) ? 1 : 2;
}

// The four faces holding edge (a, r), in slot order k = 0..3: for the two
// other axes c0 < c1, slot 2i is the face with normal 3-a-ci at r and slot
// 2i+1 the same face at r - e_ci.
__device__ __forceinline__ void edge_faces(const Lattice& lat, int a, const Coord& r, int out[4])
{
    int c0 = (a == 0) ? 1 : 0;
    int c1 = (a == 2) ? 1 : 2;
    int m0 = 3 - a - c0, m1 = 3 - a - c1;
    out[0] = m0 * lat.L3 + site_index(lat, r);
    out[1] = m0 * lat.L3 + site_index(lat, shifted(lat, r, c0, -1));
    out[2] = m1 * lat.L3 + site_index(lat, r);
    out[3] = m1 * lat.L3 + site_index(lat, shifted(lat, r, c1, -1));
}

// The four edges of face (n, r) and, for each, the slot that face occupies in
// the edge's face list:  (a, r) slot 2(b-1);  (a, r+e_b) slot 2(b-1)+1;
// (b, r) slot 2a;  (b, r+e_a) slot 2a+1.
struct FaceEdges {
    int dir[4];
    int site[4];
    int slot[4];
};

__device__ __forceinline__ FaceEdges face_edges(const Lattice& lat, int n, const Coord& r)
{
    int a, b;
    plane_axes(n, a, b);
    FaceEdges fe;
    int s0 = site_index(lat, r);
    fe.dir[0] = a; fe.site[0] = s0;                                   fe.slot[0] = 2 * (b - 1);
    fe.dir[1] = a; fe.site[1] = site_index(lat, shifted(lat, r, b, 1)); fe.slot[1] = 2 * (b - 1) + 1;
    fe.dir[2] = b; fe.site[2] = s0;                                   fe.slot[2] = 2 * a;
    fe.dir[3] = b; fe.site[3] = site_index(lat, shifted(lat, r, a, 1)); fe.slot[3] = 2 * a + 1;
    return fe;
}

// Face (n, r) owns edge ((n+1) mod 3, r) for in-place updates of e; this is a
// bijection between faces and edges.  Returns the index 0..3 of that edge in
// face_edges(): edge 0 = (a, r) when n != 1, edge 2 = (b, r) when n == 1.
__device__ __forceinline__ int owned_edge_slot(int n) { return (n == 1) ? 2 : 0; }

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): 10 rounds of two 32x32->64 multiplies and a word permutation, with
// a Weyl key schedule.  Each product is taken as its high and low 32-bit
// halves (__umulhi and a plain multiply), which measured 16-18% fewer
// instructions in the noise and measurement kernels than one 64-bit product.
struct U32x4 {
    uint32_t v[4];
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t h0 = __umulhi(M0, c0), l0 = M0 * c0;
        const uint32_t h1 = __umulhi(M1, c2), l1 = M1 * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0;
        const uint32_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    U32x4 r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

enum : uint32_t { kStreamQubit = 0, kStreamMeas = 1, kStreamCoin = 2 };
constexpr uint32_t kMaxSweep = 1u << 22;   // sweep indices fit the counter's 22 bits

// Block b of the random stream at (seed, stream, site, cycle, sweep, group): its
// two 64-bit words are words 2b (outputs 0, 1) and 2b + 1 (outputs 2, 3).
struct Words2 {
    uint64_t w[2];
};

__device__ __forceinline__ Words2 stream_words(uint64_t seed, uint32_t stream, uint64_t site, uint32_t cycle,
                                               uint32_t sweep, uint64_t group, uint32_t block)
{
    const U32x4 o = philox4x32_10((uint32_t)group, (uint32_t)site, cycle, (stream << 30) | (sweep << 8) | block,
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    Words2 r;
    r.w[0] = (uint64_t)o.v[0] | ((uint64_t)o.v[1] << 32);
    r.w[1] = (uint64_t)o.v[2] | ((uint64_t)o.v[3] << 32);
    return r;
}

// 64 Bernoulli(P / 2^32) bits, one per sample of word `group` (P = thr): lane j is set iff
// U_j < P for a 32-bit uniform U_j.  The six high bits of every lane (bit 31-i of U_j = bit j
// of stream word i, i = 0..5, blocks 0..2) are compared with P's, most significant first and
// bit-sliced over the 64 lanes; that decides every lane but the ties (six high bits equal to
// P's: one lane in 64 on average).  The k-th tied lane in lane order takes U's low 26 bits
// from the high 26 bits of output k % 4 of block 3 + k/4.  A word costs three blocks plus
// one per four ties -- about four for a warp of words, where comparing all 32 bits
// bit-sliced until every lane was decided cost a warp about six (the slowest of its words).
__device__ __forceinline__ uint64_t bernoulli_word(uint64_t thr, uint64_t seed, uint32_t stream,
                                                   uint64_t site, uint32_t cycle, uint32_t sweep,
                                                   uint64_t group)
{
    if (thr == 0) return 0;
    if (thr >= (1ULL << 32)) return ~0ULL;
    uint64_t lt = 0, eq = ~0ULL;
    // unrolled: each block's two threshold bits sit at compile-time positions
#pragma unroll
    for (uint32_t blk = 0; blk < 3; ++blk) {
        const Words2 w = stream_words(seed, stream, site, cycle, sweep, group, blk);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int bit = 31 - (int)(2 * blk + i);
            if ((thr >> bit) & 1ULL) {
                lt |= eq & ~w.w[i];
                eq &= w.w[i];
            } else {
                eq &= ~w.w[i];
            }
        }
    }
    const uint32_t low = (uint32_t)thr & ((1u << 26) - 1);
    for (uint32_t blk = 3; eq != 0; ++blk) {   // at most 16 blocks: four ties each
        const U32x4 o = philox4x32_10((uint32_t)group, (uint32_t)site, cycle, (stream << 30) | (sweep << 8) | blk,
                                      (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t b = eq & (0 - eq);   // the lowest tied lane left (0 once none is)
            if ((o.v[i] >> 6) < low) lt |= b;
            eq ^= b;
        }
    }
    return lt;
}

// p-flip coin words for 64 samples of up to four variables keyed by one site:
// stream-2 word d is the coin word of the site's d-th variable (d-edge of a
// lattice site; variable 4 site + d of a generic code).
struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 coin_words(uint64_t seed, uint64_t site, uint32_t cycle, uint32_t sweep,
                                            uint64_t group)
{
    const Words2 a = stream_words(seed, kStreamCoin, site, cycle, sweep, group, 0);
    const Words2 b = stream_words(seed, kStreamCoin, site, cycle, sweep, group, 1);
    U64x4 r;
    r.v[0] = a.w[0]; r.v[1] = a.w[1]; r.v[2] = b.w[0]; r.v[3] = b.w[1];
    return r;
}

// ----------------------------------------------------------------- majority logic
// For four bit-sliced checks: lanes with >= 3 set, and lanes with exactly 2 set.
__device__ __forceinline__ uint64_t at_least_three(uint64_t a, uint64_t b, uint64_t c, uint64_t d)
{
    return (a & b & (c | d)) | (c & d & (a | b));
}

__device__ __forceinline__ uint64_t exactly_two(uint64_t a, uint64_t b, uint64_t c, uint64_t d)
{
    return (a & b & ~(c | d)) | (c & d & ~(a | b)) | ((a ^ b) & (c ^ d));
}

// XOR v into a bit-sliced word that only this thread updates during the launch, as a
// reduction the memory system carries out (the result is not returned): the thread neither
// loads the word nor waits for it, and a word with no flipped lane (v = 0) is not touched,
// so after the first applications of a cycle, where few words change, most of the
// word array is neither read nor written.
__device__ __forceinline__ void xor_into(uint64_t* w, uint64_t v)
{
    static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "64-bit words");
    if (v) atomicXor(reinterpret_cast<unsigned long long*>(w), (unsigned long long)v);
}

}  // namespace t3d
