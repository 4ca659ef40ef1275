// Bit-sliced kernels (64 samples per uint64_t word, word index innermost):
// phenomenological noise, noisy syndrome measurement, synchronous flip /
// p-flip applications, logical readout, and layout conversion.
//
// Each thread owns one (site, word) pair; a warp covers up to 32 consecutive
// words of one site, so every global access is a coalesced row and the
// periodic neighbours of a site sit at fixed word strides of the same row.
// The run kernels take an item table (t3d_items.cuh) and walk the blocks of
// every item in a persistent grid-stride loop, so lattices of different size
// share one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "t3d_device.cuh"
#include "t3d_host.hpp"
#include "t3d_items.cuh"

namespace t3d {
namespace {

constexpr int kThreads = 256;

struct SiteWordGrid {
    dim3 grid, block;
};

// Words per block row: 32, or the next power of two >= words for tiny batches.
int row_words(int64_t words)
{
    int tx = 32;
    while (tx > 1 && tx / 2 >= words) tx /= 2;
    return tx;
}

// x = words (coalesced), y = sites (layout conversion kernels).
SiteWordGrid site_word_grid(int64_t n_sites, int64_t words)
{
    int tx = row_words(words);
    int ty = kThreads / tx;
    SiteWordGrid g;
    g.block = dim3(tx, ty, 1);
    g.grid = dim3((unsigned)((n_sites + ty - 1) / ty), (unsigned)((words + tx - 1) / tx), 1);
    return g;
}

// Blocks an item needs for a (sites x words) tiling with rows of tx words.
int64_t tile_blocks(int64_t n_sites, int64_t W, int tx)
{
    const int ty = kThreads / tx;
    return ((n_sites + ty - 1) / ty) * ((W + tx - 1) / tx);
}

// The same for the kernels that split a block index with 32-bit arithmetic
// (tile_site_word): T3D_EINVAL if the item needs 2^32 blocks or more (a state
// array of at least 2^32 x 256 words, far beyond device memory).
t3d_status tile_blocks_checked(const ItemDesc& d, int64_t n_sites, int64_t W, int tx, int64_t* blocks)
{
    *blocks = tile_blocks(n_sites, W, tx);
    T3D_REQUIRE(n_sites < (1LL << 31) && *blocks < (1LL << 32),
                "lattice L = %d with %lld words needs too many thread blocks", d.lat.L, (long long)W);
    return T3D_OK;
}

// Local block lb of an item -> this thread's (site, word); sites vary fastest
// across blocks so neighbouring sites run together.  tx and ty = kThreads / tx
// are powers of two (shifts), and one 32-bit division splits lb: every launcher
// checks that an item's blocks stay below 2^32 (tile_blocks_checked).  The
// 64-bit divisions this replaces were a quarter of the noise kernel's
// instructions.
__device__ __forceinline__ bool tile_site_word(const ItemDesc& d, int64_t lb, int n_sites,
                                               int& site, int64_t& w)
{
    const int tx = d.tx, lx = __ffs(tx) - 1, ly = __ffs(kThreads) - 1 - lx;
    const uint32_t site_tiles = ((uint32_t)n_sites + (1u << ly) - 1) >> ly;
    const uint32_t word_tile = (uint32_t)lb / site_tiles;
    const uint32_t site_tile = (uint32_t)lb - word_tile * site_tiles;
    const int t = threadIdx.x;
    w = (int64_t)word_tile * tx + (t & (tx - 1));
    site = (int)(site_tile << ly) + (t >> lx);
    return w < (d.nw ? d.nw : d.W) && site < n_sites;
}


// e ^= Bernoulli(p) for every edge (Sec. 3.1 phenomenological qubit noise).
__global__ void __launch_bounds__(kThreads)
k_noise(const __grid_constant__ ItemTable tab, uint64_t thr, uint64_t seed, uint32_t cycle)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        int v;
        int64_t w;
        if (!tile_site_word(d, lb, 3 * d.lat.L3, v, w)) return;
        const uint64_t flips =
            bernoulli_word(thr, seed, kStreamQubit, (uint64_t)v, cycle, 0, d.group0 + w);
        if (flips) d.e[(int64_t)v * d.W + w] ^= flips;
    });
}

// s_f = XOR of the face's four edges, then ^= Bernoulli(q) (Sec. 2, Sec. 3.1).
__global__ void __launch_bounds__(kThreads)
k_syndrome(const __grid_constant__ ItemTable tab, uint64_t thr, uint64_t seed, uint32_t cycle)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        const Lattice lat = d.lat;
        int f;
        int64_t w;
        if (!tile_site_word(d, lb, 3 * lat.L3, f, w)) return;
        const int n = (f >= lat.L3) + (f >= 2 * lat.L3), site = f - n * lat.L3;
        // face (n, r) spans the axes a < b other than n; its edges are the a-edges at r and
        // r + e_b and the b-edges at r and r + e_a (periodic site deltas by selects, no
        // per-thread arrays)
        const Coord r = site_coord(lat, site);
        const int L = lat.L;
        const int dx = r.x[0] + 1 == L ? 1 - L : 1, dy = r.x[1] + 1 == L ? L - lat.L2 : L,
                  dz = r.x[2] + 1 == L ? lat.L2 - lat.L3 : lat.L2;
        const int a = n == 0 ? 1 : 0, b = n == 2 ? 1 : 2;
        const int da = a == 0 ? dx : dy, db = b == 1 ? dy : dz;
        const uint64_t* __restrict__ pa = d.e + ((int64_t)a * lat.L3 + site) * d.W + w;
        const uint64_t* __restrict__ pb = d.e + ((int64_t)b * lat.L3 + site) * d.W + w;
        uint64_t acc = pa[0] ^ pa[(int64_t)db * d.W] ^ pb[0] ^ pb[(int64_t)da * d.W];
        acc ^= bernoulli_word(thr, seed, kStreamMeas, (uint64_t)f, cycle, 0, d.group0 + w);
        d.s[(int64_t)f * d.W + w] = acc;
    });
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

// Flip until clear (ItemDesc::stop): whether application d.stop_k runs -- the first
// always does, a later one only if the previous one left an unsatisfied check in the
// item.  The decision is the same for every thread of the launch.  The thread of local
// block 0 also clears the flag slot the next application writes and counts the
// applications after the first that run.
__device__ __forceinline__ bool stop_run(const ItemDesc& d, int64_t lb)
{
    if (!d.stop) return true;
    const int k = d.stop_k;
    const bool run = k == 0 || *(volatile uint32_t*)&d.stop[(k + 2) % 3] != 0;
    if (lb == 0 && threadIdx.x == 0) {
        d.stop[(k + 1) % 3] = 0;
        if (run && k > 0) d.stop[3] += 1u;
    }
    return run;
}

// Flip until clear, per thread: note an unsatisfied check left in the output (nz) and, in
// the first application, one found in the input (nzin).  The flag is read before the
// atomic so that a launch makes few atomics once the flag is up.
__device__ __forceinline__ void stop_note(const ItemDesc& d, uint64_t nz, uint64_t nzin)
{
    uint32_t* out = &d.stop[d.stop_k % 3];
    if (nz && *(volatile uint32_t*)out == 0) atomicOr(out, 1u);
    if (d.stop_k == 0 && nzin && *(volatile uint32_t*)&d.stop[4] == 0) atomicOr(&d.stop[4], 1u);
}

// The same for a whole block (every thread of the block calls it).
__device__ __forceinline__ void stop_note_block(const ItemDesc& d, uint64_t nz, uint64_t nzin)
{
    const int out = __syncthreads_or(nz != 0);
    const int in = d.stop_k == 0 ? __syncthreads_or(nzin != 0) : 0;
    if (threadIdx.x == 0) {
        if (out) atomicOr(&d.stop[d.stop_k % 3], 1u);
        if (in) atomicOr(&d.stop[4], 1u);
    }
}

// One synchronous flip application for the three faces at a site, reading the
// item's s and writing its tmp (64 registers: four blocks per SM).  The thread
// of site r decides the nine edges its faces touch -- (x,r), (y,r),
// (z,r), (x,r+e_y), (x,r+e_z), (y,r+e_x), (y,r+e_z), (z,r+e_x), (z,r+e_y) --
// each from its four faces in the old snapshot s_in, writes s_out at its three
// faces (old value XOR its four edges' flips) and applies the flips of the
// three edges at r to e (as XOR reductions: e is touched only where an edge flips).  Edge (a, r') lies on the faces with normal 3-a-c at
// r' and r' - e_c for the two axes c != a.
__global__ void __launch_bounds__(kThreads, 4)
k_flip(const __grid_constant__ ItemTable tab)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        if (!stop_run(d, lb)) return;   // the item's syndrome has cleared
        const Lattice lat = d.lat;
        int r;
        int64_t w;
        if (!tile_site_word(d, lb, lat.L3, r, w)) return;
        const uint64_t* __restrict__ s_in = d.s;
        uint64_t* __restrict__ s_out = d.tmp;
        uint64_t* __restrict__ e = d.e;
        const int64_t W = d.W;
        if (!word_live(d, w)) return;
        // row pointers of the three faces at r and the element offsets of the six neighbour
        // sites (periodic wrap folded in): every neighbour load is one add away
        const Moves mv = site_moves(lat, r);
        const int64_t L3W = (int64_t)lat.L3 * W;
        const uint64_t* __restrict__ p0 = s_in + (int64_t)r * W + w;
        const uint64_t* __restrict__ p1 = p0 + L3W;
        const uint64_t* __restrict__ p2 = p1 + L3W;
        const int64_t mx = (int64_t)mv.minus[0] * W, my = (int64_t)mv.minus[1] * W, mz = (int64_t)mv.minus[2] * W;
        const int64_t px = (int64_t)mv.plus[0] * W, py = (int64_t)mv.plus[1] * W, pz = (int64_t)mv.plus[2] * W;
        const uint64_t s0 = p0[0], s1 = p1[0], s2 = p2[0];
        // the nine edges whose flips touch this site's faces: the three at r and two each at
        // r + e_x, r + e_y, r + e_z; their four checks each
        const uint64_t q[9][4] = {
            {s2, p2[my], s1, p1[mz]},                 // x-edge at r
            {s2, p2[mx], s0, p0[mz]},                 // y-edge at r
            {s1, p1[mx], s0, p0[my]},                 // z-edge at r
            {p2[py], s2, p1[py], p1[py + mz]},        // x-edge at r + e_y
            {p2[pz], p2[pz + my], p1[pz], s1},        // x-edge at r + e_z
            {p2[px], s2, p0[px], p0[px + mz]},        // y-edge at r + e_x
            {p2[pz], p2[pz + mx], p0[pz], s0},        // y-edge at r + e_z
            {p1[px], s1, p0[px], p0[px + my]},        // z-edge at r + e_x
            {p1[py], p1[py + mx], p0[py], s0}};       // z-edge at r + e_y
        uint64_t f[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = at_least_three(q[k][0], q[k][1], q[k][2], q[k][3]);
        const uint64_t fx0 = f[0], fy0 = f[1], fz0 = f[2], fxy = f[3], fxz = f[4], fyx = f[5], fyz = f[6],
                       fzx = f[7], fzy = f[8];
        uint64_t* __restrict__ q0 = s_out + (int64_t)r * W + w;
        const uint64_t n0 = s0 ^ fy0 ^ fyz ^ fz0 ^ fzy, n1 = s1 ^ fx0 ^ fxz ^ fz0 ^ fzx,
                       n2 = s2 ^ fx0 ^ fxy ^ fy0 ^ fyx;
        q0[0] = n0;
        q0[L3W] = n1;
        q0[2 * L3W] = n2;
        if (d.stop) stop_note(d, n0 | n1 | n2, s0 | s1 | s2);
        uint64_t* __restrict__ e0 = e + (int64_t)r * W + w;
        xor_into(e0, fx0);
        xor_into(e0 + L3W, fy0);
        xor_into(e0 + 2 * L3W, fz0);
    });
}

// The same flip application with the syndrome staged through shared memory.
// A block owns one z-plane of one tile of Wt words (d.tx) and sweeps y from 0
// to L-1; thread (x, wl) handles site (x, y, z), word wl of the tile.  The
// lines its nine edges' checks come from -- plane z at y-1, y, y+1, plane z-1
// at y and y+1 (faces 0, 1), plane z+1 at y-1 and y -- sit in rings of
// shared-memory face-lines (L x Wt words each, the periodic x-halo being the
// line itself), so each step loads three new lines of plane z, z-1 and z+1
// (8 face-lines) instead of 24 scattered words per thread.  The loads of the
// next step's lines are issued before the current step computes (software
// pipelining across the y sweep).  The error words are never loaded: the
// flips go to e as XOR reductions, only where an edge flips, so after a cycle's
// first application nearly all of e is neither read nor written (one
// application alone 1.14 -> 0.94 ms at L = 32, 10^5 samples, against
// prefetching e with the face-lines).  A block has L x Wt threads (the launch
// takes the largest tile of the batch).  When every lattice of the batch has
// L >= 32 a tile may have up to 1024 threads, so that Wt = 32 at L = 32 and a
// warp reads one 256-byte run of a row: a copy with this kernel's row pattern
// moved 2.95 TB/s with 64-byte runs (4 rows per warp, Wt = 8) and 4.97 TB/s
// with 256-byte runs, and one application at L = 32, 10^5 samples took
// 0.89 ms (0.91 with Wt = 8; inside the FFPFF cycle 0.71 of the HBM peak
// against 0.57).  Smaller lattices keep tiles of at most 256 threads (at L = 16
// and 24 the 512- and 768-thread tiles, fewer blocks per SM, measured 0.121
// and 0.380 ms against 0.104 and 0.368).  64 registers; the rings are dynamic
// shared memory, kTileSlots face-lines of blockDim.x words.
constexpr int kFlipThreads = 1024;              // largest tile: L x Wt threads, all L >= 32
constexpr int kFlipThreadsSmall = 256;          // largest tile when a lattice has L < 32
constexpr int kTileSlots = 9 + 4 + 6;           // plane z: 3 lines x 3 faces; z-1: 2 x 2; z+1: 2 x 3

__device__ __forceinline__ int ring3(int y) { return (y + 3) % 3; }
__device__ __forceinline__ int ring2(int y) { return (y + 2) & 1; }

__global__ void __launch_bounds__(kFlipThreads, 1)
k_flip_tiled(const __grid_constant__ ItemTable tab)
{
    extern __shared__ uint64_t sm[];   // kTileSlots face-lines of tw words
    const int tw = blockDim.x;
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        if (!stop_run(d, lb)) return;   // the item's syndrome has cleared (uniform over the launch)
        __syncthreads();   // the previous block's last step may still read the rings
        const Lattice lat = d.lat;
        const int L = lat.L, Wt = d.tx;
        uint64_t nz = 0, nzin = 0;   // flip until clear: unsatisfied checks written / read
        const int64_t W = d.W, nw = d.nw ? d.nw : d.W, L3W = (int64_t)lat.L3 * W;
        const int z = (int)(lb % L);
        const int64_t w = (lb / L) * Wt + (threadIdx.x & (Wt - 1));
        const int x = threadIdx.x / Wt, wl = threadIdx.x & (Wt - 1);
        const bool act = x < L && w < nw && word_live(d, w);
        const int zm = z == 0 ? L - 1 : z - 1, zp = z + 1 == L ? 0 : z + 1;
        const int xm = x == 0 ? L - 1 : x - 1, xp = x + 1 == L ? 0 : x + 1;
        const int me = x * Wt + wl;
        // element offsets: a y-row of one face-plane is L W words, a z-plane L^2 W; this
        // thread's column (x, w) of plane zz starts at zz L^2 W + x W + w, and row yy (one
        // periodic wrap at most: -1 <= yy <= L) adds yy L W
        const int64_t rowW = (int64_t)L * W, planeW = (int64_t)L * rowW, col = (int64_t)x * W + w;
        const int64_t cz = (int64_t)z * planeW + col, czp = (int64_t)zp * planeW + col,
                      czm = (int64_t)zm * planeW + col;
        auto row = [&](int yy) { return (int64_t)(yy < 0 ? yy + L : (yy >= L ? yy - L : yy)) * rowW; };
        // this thread's word of face n at (x, yy, zz), given the plane's column offset
        auto gword = [&](const uint64_t* base, int n, int yy, int64_t cplane) {
            return base[(int64_t)n * L3W + cplane + row(yy)];
        };
        auto put = [&](int slot, uint64_t v) { sm[slot * tw + me] = v; };
        auto P0 = [&](int yy, int n, int xx) { return sm[(ring3(yy) * 3 + n) * tw + xx * Wt + wl]; };
        auto Pm = [&](int yy, int n, int xx) { return sm[(9 + ring2(yy) * 2 + n) * tw + xx * Wt + wl]; };
        auto Pp = [&](int yy, int n, int xx) { return sm[(13 + ring2(yy) * 3 + n) * tw + xx * Wt + wl]; };
        // the eight face-line words entering at step yy (plane z at yy+1, plane z+1 at yy,
        // plane z-1 at yy+1 faces 0, 1)
        uint64_t nx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        auto fetch = [&](int yy) {
            if (!act) return;
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                nx[n] = gword(d.s, n, yy + 1, cz);
                nx[3 + n] = gword(d.s, n, yy, czp);
            }
            nx[6] = gword(d.s, 0, yy + 1, czm);
            nx[7] = gword(d.s, 1, yy + 1, czm);
        };
        auto stash = [&](int yy) {
            if (!act) return;
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                put(ring3(yy + 1) * 3 + n, nx[n]);
                put(13 + ring2(yy) * 3 + n, nx[3 + n]);
            }
            put(9 + ring2(yy + 1) * 2 + 0, nx[6]);
            put(9 + ring2(yy + 1) * 2 + 1, nx[7]);
        };
        // fill: plane z lines -1 and 0, plane z-1 line 0, plane z+1 line -1
        if (act) {
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                put(ring3(-1) * 3 + n, gword(d.s, n, -1, cz));
                put(ring3(0) * 3 + n, gword(d.s, n, 0, cz));
                put(13 + ring2(-1) * 3 + n, gword(d.s, n, -1, czp));
            }
            put(9 + ring2(0) * 2 + 0, gword(d.s, 0, 0, czm));
            put(9 + ring2(0) * 2 + 1, gword(d.s, 1, 0, czm));
        }
        fetch(0);
        for (int y = 0; y < L; ++y) {
            stash(y);
            __syncthreads();
            if (y + 1 < L) fetch(y + 1);   // in flight while this step computes
            if (act) {
                const uint64_t s0 = P0(y, 0, x), s1 = P0(y, 1, x), s2 = P0(y, 2, x);
                const int64_t own = cz + (int64_t)y * rowW;
                uint64_t* __restrict__ q0 = d.tmp + own;
                {
                    const uint64_t q[9][4] = {
                        {s2, P0(y - 1, 2, x), s1, Pm(y, 1, x)},                       // x-edge at r
                        {s2, P0(y, 2, xm), s0, Pm(y, 0, x)},                          // y-edge at r
                        {s1, P0(y, 1, xm), s0, P0(y - 1, 0, x)},                      // z-edge at r
                        {P0(y + 1, 2, x), s2, P0(y + 1, 1, x), Pm(y + 1, 1, x)},      // x-edge at r + e_y
                        {Pp(y, 2, x), Pp(y - 1, 2, x), Pp(y, 1, x), s1},              // x-edge at r + e_z
                        {P0(y, 2, xp), s2, P0(y, 0, xp), Pm(y, 0, xp)},               // y-edge at r + e_x
                        {Pp(y, 2, x), Pp(y, 2, xm), Pp(y, 0, x), s0},                 // y-edge at r + e_z
                        {P0(y, 1, xp), s1, P0(y, 0, xp), P0(y - 1, 0, xp)},           // z-edge at r + e_x
                        {P0(y + 1, 1, x), P0(y + 1, 1, xm), P0(y + 1, 0, x), s0}};    // z-edge at r + e_y
                    uint64_t f[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) f[k] = at_least_three(q[k][0], q[k][1], q[k][2], q[k][3]);
                    const uint64_t n0 = s0 ^ f[1] ^ f[6] ^ f[2] ^ f[8], n1 = s1 ^ f[0] ^ f[4] ^ f[2] ^ f[7],
                                   n2 = s2 ^ f[0] ^ f[3] ^ f[1] ^ f[5];
                    q0[0] = n0;
                    q0[L3W] = n1;
                    q0[2 * L3W] = n2;
                    nz |= n0 | n1 | n2;
                    nzin |= s0 | s1 | s2;
                    uint64_t* __restrict__ e0 = d.e + own;   // this thread alone updates its site's edges
                    xor_into(e0, f[0]);
                    xor_into(e0 + L3W, f[1]);
                    xor_into(e0 + 2 * L3W, f[2]);
                }
            }
            __syncthreads();
        }
        if (d.stop) stop_note_block(d, nz, nzin);
    });
}

// Words per tile row of k_flip_tiled: L x Wt <= max_threads, Wt a power of two <= 32
// and no wider than the batch.
int tiled_words(int L, int64_t nw, int max_threads)
{
    int wt = 32;
    while (wt > 1 && (L * wt > max_threads || wt / 2 >= nw)) wt /= 2;
    return wt;
}

// p-flip in two passes, so that each (site, word) draws one Philox block.
// The first pass is bound by the Philox arithmetic; at 40 registers six blocks
// per SM keep the integer pipes busier (2.45 -> 2.27 ms per application at
// L = 32, 10^5 samples), and computing the coin block while the syndrome and
// error words load hides their latency (2.27 -> 2.04 ms).
// Pass 1: the thread of site r decides its own three edges from their checks
// (s at r, r - e_x, r - e_y, r - e_z), with the coin of the site's block for
// the lanes with exactly two unsatisfied checks, writes the flip words to
// d.tmp [3L^3][W] and applies them to e.
__global__ void __launch_bounds__(kThreads, 6)
k_pflip_decide(const __grid_constant__ ItemTable tab, uint64_t seed, uint32_t cycle, uint32_t sweep)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        const Lattice lat = d.lat;
        int r;
        int64_t w;
        if (!tile_site_word(d, lb, lat.L3, r, w)) return;
        if (!word_live(d, w)) return;
        const int64_t W = d.W;
        const Moves mv = site_moves(lat, r);
        const int64_t L3W = (int64_t)lat.L3 * W;
        const uint64_t* __restrict__ p0 = d.s + (int64_t)r * W + w;
        const uint64_t* __restrict__ p1 = p0 + L3W;
        const uint64_t* __restrict__ p2 = p1 + L3W;
        const int64_t mx = (int64_t)mv.minus[0] * W, my = (int64_t)mv.minus[1] * W, mz = (int64_t)mv.minus[2] * W;
        // the syndrome words are requested first; the coin block does not depend on them, so
        // its arithmetic runs while they are in flight (nearly every site-word has a lane with
        // a tie, so computing it unconditionally costs nothing); the flips reach e as XOR
        // reductions (e is not loaded: one p-flip application 1.80 -> 1.74 ms at L = 32,
        // 10^5 samples)
        const uint64_t s0 = p0[0], s1 = p1[0], s2 = p2[0];
        const uint64_t q[3][4] = {{s2, p2[my], s1, p1[mz]},    // x-edge at r
                                  {s2, p2[mx], s0, p0[mz]},    // y-edge at r
                                  {s1, p1[mx], s0, p0[my]}};   // z-edge at r
        uint64_t* __restrict__ e0 = d.e + (int64_t)r * W + w;
        const U64x4 c = coin_words(seed, (uint64_t)r, cycle, sweep, word_group(d, w));
        uint64_t f[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            f[k] = at_least_three(q[k][0], q[k][1], q[k][2], q[k][3]) |
                   (exactly_two(q[k][0], q[k][1], q[k][2], q[k][3]) & c.v[k]);
        uint64_t* __restrict__ fo = d.tmp + (int64_t)r * W + w;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fo[k * L3W] = f[k];
            xor_into(e0 + k * L3W, f[k]);
        }
    });
}

// Pass 2: every face of site r XORs in the flips of its four edges (in place:
// each thread updates only its own faces and reads only flip words; the update
// is a XOR reduction, so a face none of whose edges flipped -- most of them -- is
// neither read nor written: the FFPFF cycle at L = 32, 10^5 samples 14.40 ->
// 14.20 ms).
__global__ void __launch_bounds__(kThreads, 6)
k_pflip_apply(const __grid_constant__ ItemTable tab)
{
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        const Lattice lat = d.lat;
        int r;
        int64_t w;
        if (!tile_site_word(d, lb, lat.L3, r, w)) return;
        if (!word_live(d, w)) return;
        const int64_t W = d.W;
        const Moves mv = site_moves(lat, r);
        const int64_t L3W = (int64_t)lat.L3 * W;
        const uint64_t* __restrict__ fx = d.tmp + (int64_t)r * W + w;   // x-edge flips
        const uint64_t* __restrict__ fy = fx + L3W;
        const uint64_t* __restrict__ fz = fy + L3W;
        const int64_t px = (int64_t)mv.plus[0] * W, py = (int64_t)mv.plus[1] * W, pz = (int64_t)mv.plus[2] * W;
        const uint64_t fx0 = fx[0], fy0 = fy[0], fz0 = fz[0];
        uint64_t* __restrict__ q0 = d.s + (int64_t)r * W + w;
        xor_into(q0, fy0 ^ fy[pz] ^ fz0 ^ fz[py]);         // normal x: y-edges at r, r + e_z; z-edges at r, r + e_y
        xor_into(q0 + L3W, fx0 ^ fx[pz] ^ fz0 ^ fz[px]);   // normal y
        xor_into(q0 + 2 * L3W, fx0 ^ fx[py] ^ fy0 ^ fy[px]);   // normal z
    });
}

// Logical readout.  A block takes a tile of kLogWords words and splits the L^2
// lines of each axis over kLogSplit thread rows (thread = row x word, so a warp
// reads 64-byte runs of four lines at once); each thread sums its lines'
// parities in a bit-sliced counter, the rows' counters are added in shared
// memory by a tree of bit-sliced additions, and a lane fails axis d iff
// 2 c_d >= L^2.  Eight-word tiles give about 200 blocks at 10^5 samples (the
// 32-word tiles before gave 49 for 152 SMs: 1.9 ms for the 1.2 GB of e at L = 32).
constexpr int kCountBits = 17;  // L^2 <= 65536
constexpr int kLineSplit = 8;   // the fallback gate's face split
constexpr int kLogWords = 8;
constexpr int kLogSplit = 32;

__device__ __forceinline__ void counter_add_bit(uint64_t (&c)[kCountBits], uint64_t bit)
{
#pragma unroll
    for (int b = 0; b < kCountBits; ++b) {
        uint64_t carry = c[b] & bit;
        c[b] ^= bit;
        bit = carry;
    }
}

__global__ void __launch_bounds__(kLogWords * kLogSplit)
k_logical(const __grid_constant__ ItemTable tab)
{
    __shared__ uint64_t part[kLogSplit][kCountBits][kLogWords];
    __shared__ uint64_t fail[3][kLogWords];
    __shared__ unsigned int hist[8];
    const int tx = threadIdx.x % kLogWords, ty = threadIdx.x / kLogWords;
    // block-uniform loop: every thread reaches every barrier
    for_each_item_block(tab, [&](const ItemDesc& d, int64_t lb) {
        const Lattice lat = d.lat;
        const int64_t W = d.W;
        const int64_t w = lb * kLogWords + tx;
        if (threadIdx.x < 8) hist[threadIdx.x] = 0;
        const int L = lat.L, L2 = lat.L2;
        for (int dd = 0; dd < 3; ++dd) {
            const int u_axis = (dd == 0) ? 1 : 0;
            const int v_axis = (dd == 2) ? 1 : 2;
            uint64_t cnt[kCountBits];
#pragma unroll
            for (int b = 0; b < kCountBits; ++b) cnt[b] = 0;
            if (w < W) {
                // step between consecutive sites of a line along axis dd
                const int64_t step = (dd == 0 ? 1 : (dd == 1 ? L : L2)) * W;
                for (int line = ty; line < L2; line += kLogSplit) {
                    Coord r;
                    r.x[u_axis] = line % L;
                    r.x[v_axis] = line / L;
                    r.x[dd] = 0;
                    const uint64_t* __restrict__ p = d.e + ((int64_t)dd * lat.L3 + site_index(lat, r)) * W + w;
                    uint64_t par = 0;
#pragma unroll 8
                    for (int t = 0; t < L; ++t) par ^= __ldcs(p + t * step);
                    counter_add_bit(cnt, par);
                }
            }
#pragma unroll
            for (int b = 0; b < kCountBits; ++b) part[ty][b][tx] = cnt[b];
            __syncthreads();
            for (int half = kLogSplit / 2; half > 0; half >>= 1) {
                if (ty < half) {
                    uint64_t carry = 0;
#pragma unroll
                    for (int b = 0; b < kCountBits; ++b) {
                        const uint64_t x = part[ty][b][tx], y = part[ty + half][b][tx];
                        part[ty][b][tx] = x ^ y ^ carry;
                        carry = (x & y) | (carry & (x ^ y));
                    }
                }
                __syncthreads();
            }
            if (ty == 0) {
                // lanes with count >= ceil(L^2 / 2)
                const unsigned need = (unsigned)(L2 + 1) / 2;
                uint64_t gt = 0, eq = ~0ULL;
#pragma unroll
                for (int b = kCountBits - 1; b >= 0; --b) {
                    const uint64_t tb = part[0][b][tx];
                    if ((need >> b) & 1u) {
                        eq &= tb;
                    } else {
                        gt |= eq & tb;
                        eq &= ~tb;
                    }
                }
                fail[dd][tx] = gt | eq;
            }
            __syncthreads();
        }
        if (w < W) {
            constexpr int per = 64 / kLogSplit;   // samples of the word per thread row
            for (int j = ty * per; j < ty * per + per; ++j) {
                const int64_t sample = w * 64 + j;
                if (sample >= d.n_samples) break;
                const unsigned m = (unsigned)((fail[0][tx] >> j) & 1ULL) |
                                   ((unsigned)((fail[1][tx] >> j) & 1ULL) << 1) |
                                   ((unsigned)((fail[2][tx] >> j) & 1ULL) << 2);
                if (d.mask) d.mask[sample] = (uint8_t)m;
                if (d.counts8) atomicAdd(&hist[m], 1u);
            }
        }
        __syncthreads();
        if (d.counts8 && threadIdx.x < 8 && hist[threadIdx.x])
            atomicAdd(&d.counts8[threadIdx.x], (unsigned long long)hist[threadIdx.x]);
        __syncthreads();
    });
}

// Fallback gate: flag every word in which some sample's syndrome has more
// than max_weight unsatisfied checks.  Two passes.  k_gate_count: block
// (32, 8) over a 32-word tile and one of Y face ranges (blockIdx.y);
// threadIdx.y splits the range further; per-lane counts are bit-sliced and
// the block's partial count goes to part[y][bit][w].  k_gate_decide: one
// thread per word adds the Y partials and compares.
constexpr int kWeightBits = 23;  // 3 L^3 <= 3 * 128^3 < 2^23

__device__ __forceinline__ void add_sliced(uint64_t (&tot)[kWeightBits], const uint64_t* x, int64_t stride)
{
    uint64_t carry = 0;
#pragma unroll
    for (int b = 0; b < kWeightBits; ++b) {
        const uint64_t v = x[b * stride];
        const uint64_t sum = tot[b] ^ v ^ carry;
        carry = (tot[b] & v) | (carry & (tot[b] ^ v));
        tot[b] = sum;
    }
}

__global__ void __launch_bounds__(256)
k_gate_count(Lattice lat, int64_t W, const uint64_t* __restrict__ s, int64_t faces_per_y,
             uint64_t* __restrict__ part)
{
    __shared__ uint64_t red[kLineSplit][kWeightBits][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * 32 + tx;
    const int64_t f0 = (int64_t)blockIdx.y * faces_per_y;
    const int64_t f1 = min(f0 + faces_per_y, (int64_t)3 * lat.L3);
    uint64_t cnt[kWeightBits];
#pragma unroll
    for (int b = 0; b < kWeightBits; ++b) cnt[b] = 0;
    if (w < W) {
        for (int64_t f = f0 + ty; f < f1; f += kLineSplit) {
            uint64_t bit = __ldcs(&s[f * W + w]);
#pragma unroll
            for (int b = 0; b < kWeightBits; ++b) {
                const uint64_t carry = cnt[b] & bit;
                cnt[b] ^= bit;
                bit = carry;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < kWeightBits; ++b) red[ty][b][tx] = cnt[b];
    __syncthreads();
    if (ty == 0 && w < W) {
        uint64_t tot[kWeightBits];
#pragma unroll
        for (int b = 0; b < kWeightBits; ++b) tot[b] = red[0][b][tx];
        for (int k = 1; k < kLineSplit; ++k) add_sliced(tot, &red[k][0][tx], 32);
        uint64_t* out = part + (int64_t)blockIdx.y * kWeightBits * W + w;
#pragma unroll
        for (int b = 0; b < kWeightBits; ++b) out[b * W] = tot[b];
    }
}

__global__ void k_gate_decide(int64_t W, int Y, const uint64_t* __restrict__ part, uint32_t max_weight,
                              uint8_t* __restrict__ gate, unsigned long long* __restrict__ n_flagged)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    uint64_t tot[kWeightBits];
#pragma unroll
    for (int b = 0; b < kWeightBits; ++b) tot[b] = part[b * W + w];
    for (int y = 1; y < Y; ++y) add_sliced(tot, part + (int64_t)y * kWeightBits * W + w, W);
    // lanes with count > max_weight, i.e. count >= max_weight + 1 (MSB-first comparison)
    const uint64_t need = (uint64_t)max_weight + 1;
    uint64_t gt = 0, eq = ~0ULL;
#pragma unroll
    for (int b = kWeightBits - 1; b >= 0; --b) {
        if ((need >> b) & 1u) {
            eq &= tot[b];
        } else {
            gt |= eq & tot[b];
            eq &= ~tot[b];
        }
    }
    const bool flag = (need >> kWeightBits) == 0 && (gt | eq) != 0;
    gate[w] = flag ? 1 : 0;
    if (flag && n_flagged) atomicAdd(n_flagged, 1ULL);
}

// Flip until clear, after the last application: if the item's syndrome cleared (the last
// application left no unsatisfied check, or did not run), its s is all zero -- the
// applications that did not run left stale words in the ping-pong buffers, so s is
// written as zero here -- and the number of applications that ran goes to *sweeps_done:
// the first if its input had an unsatisfied check, and every later one that ran.
__global__ void k_flip_finish(const __grid_constant__ ItemDesc d, int n_apply, int32_t* __restrict__ sweeps_done)
{
    const uint32_t* st = d.stop;
    if (blockIdx.x == 0 && threadIdx.x == 0 && sweeps_done) *sweeps_done = (int32_t)(st[4] + st[3]);
    if (st[(n_apply - 1) % 3] != 0) return;
    const int64_t n = (int64_t)3 * d.lat.L3 * d.W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d.s[i] = 0;
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

}  // namespace

// ----------------------------------------------------------------- launchers
t3d_status launch_noise(ItemTable& tab, uint64_t thr, uint64_t seed, uint32_t cycle, cudaStream_t st)
{
    if (thr == 0) return T3D_OK;
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        const int64_t nw = d.nw ? d.nw : d.W;
        d.tx = row_words(nw);
        T3D_TRY(tile_blocks_checked(d, 3LL * d.lat.L3, nw, d.tx, &d.blocks));
    }
    finish_table(tab);
    ProfScope prof(T3D_K_NOISE, st);
    k_noise<<<persistent_grid((const void*)k_noise, kThreads, T3D_K_NOISE, tab.prefix[tab.n], has_live(tab)), kThreads,
              0, st>>>(tab, thr, seed, cycle);
    T3D_LAUNCH_CHECK("noise");
    return T3D_OK;
}

t3d_status launch_syndrome(ItemTable& tab, uint64_t thr, uint64_t seed, uint32_t cycle, cudaStream_t st)
{
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        const int64_t nw = d.nw ? d.nw : d.W;
        d.tx = row_words(nw);
        T3D_TRY(tile_blocks_checked(d, 3LL * d.lat.L3, nw, d.tx, &d.blocks));
    }
    finish_table(tab);
    ProfScope prof(T3D_K_SYNDROME, st);
    k_syndrome<<<persistent_grid((const void*)k_syndrome, kThreads, T3D_K_SYNDROME, tab.prefix[tab.n], has_live(tab)),
                 kThreads, 0, st>>>(tab, thr, seed, cycle);
    T3D_LAUNCH_CHECK("syndrome");
    return T3D_OK;
}

t3d_status launch_sweeps(ItemTable& tab, const char* schedule, int slen, int n_apply, uint32_t sweep0,
                         uint64_t seed, uint32_t cycle, cudaStream_t st)
{
    if (n_apply <= 0) return T3D_OK;
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        const int64_t nw = d.nw ? d.nw : d.W;
        d.tx = row_words(nw);
        T3D_TRY(tile_blocks_checked(d, d.lat.L3, nw, d.tx, &d.blocks));
        d.live_wpu = d.tx;
        d.live_bpu = tile_blocks(d.lat.L3, d.tx, d.tx);   // site tiles of one word row
    }
    finish_table(tab);
    // the shared-memory flip when every face-line of the batch fits a tile row of at
    // least 16 words (1024-thread tiles: all L >= 32, so L <= 64) or 8 words (256-thread
    // tiles: L <= 32); the block takes the batch's largest tile.  Above that k_flip
    // (L = 48: 1.78 ms tiled against 1.82 untiled, L = 64: 1.05 against 1.08).
    bool wide = true;
    for (int i = 0; i < tab.n; ++i) wide = wide && tab.it[i].lat.L >= 32;
    const int max_threads = wide ? kFlipThreads : kFlipThreadsSmall;
    bool tiled = true;
    int tile_threads = 32;
    ItemTable tt = tab;
    for (int i = 0; i < tt.n; ++i) {
        ItemDesc& d = tt.it[i];
        const int64_t nw = d.nw ? d.nw : d.W;
        tiled = tiled && d.lat.L * (wide ? 16 : 8) <= max_threads;
        d.tx = tiled_words(d.lat.L, nw, max_threads);
        d.blocks = (int64_t)d.lat.L * ((nw + d.tx - 1) / d.tx);
        d.live_wpu = d.tx;
        d.live_bpu = d.lat.L;   // one z-plane per block, word tiles outermost
        tile_threads = std::max(tile_threads, (d.lat.L * d.tx + 31) / 32 * 32);
    }
    finish_table(tt);
    const size_t tile_smem = (size_t)kTileSlots * tile_threads * sizeof(uint64_t);
    if (tiled) T3D_TRY(allow_dynamic_smem((const void*)k_flip_tiled, tile_smem));
    ItemTable t = tab;  // flip: s and tmp swap roles; p-flip: tmp holds the flip words, s updated in place
    int swaps = 0;
    for (int k = 0; k < n_apply; ++k) {
        const bool pk = schedule[k % slen] == 'P';
        for (int i = 0; i < t.n; ++i) t.it[i].stop_k = k;
        for (int i = 0; i < tt.n; ++i) tt.it[i].stop_k = k;
        ProfScope prof(pk ? T3D_K_PFLIP : T3D_K_FLIP, st);
        if (pk) {
            k_pflip_decide<<<persistent_grid((const void*)k_pflip_decide, kThreads, T3D_K_PFLIP, t.prefix[t.n], has_live(t)),
                             kThreads, 0, st>>>(t, seed, cycle, sweep0 + (uint32_t)k);
            T3D_LAUNCH_CHECK("p-flip decisions");
            k_pflip_apply<<<persistent_grid((const void*)k_pflip_apply, kThreads, T3D_K_PFLIP, t.prefix[t.n], has_live(t)),
                            kThreads, 0, st>>>(t);
            T3D_LAUNCH_CHECK("p-flip syndrome update");
        } else {
            if (tiled) {
                k_flip_tiled<<<persistent_grid((const void*)k_flip_tiled, tile_threads, T3D_K_FLIP, tt.prefix[tt.n],
                                               has_live(tt), tile_smem),
                               tile_threads, tile_smem, st>>>(tt);
            } else {
                k_flip<<<persistent_grid((const void*)k_flip, kThreads, T3D_K_FLIP, t.prefix[t.n], has_live(t)), kThreads, 0,
                         st>>>(t);
            }
            T3D_LAUNCH_CHECK("flip sweep");
            for (int i = 0; i < t.n; ++i) std::swap(t.it[i].s, t.it[i].tmp);
            for (int i = 0; i < tt.n; ++i) std::swap(tt.it[i].s, tt.it[i].tmp);
            ++swaps;
        }
    }
    if (swaps & 1) {
        for (int i = 0; i < tab.n; ++i) {
            const ItemDesc& d = tab.it[i];
            const size_t pitch = (size_t)d.W * sizeof(uint64_t);
            const size_t width = (size_t)(d.nw ? d.nw : d.W) * sizeof(uint64_t);
            T3D_CUDA_CHECK(cudaMemcpy2DAsync(d.s, pitch, d.tmp, pitch, width, (size_t)3 * d.lat.L3,
                                             cudaMemcpyDeviceToDevice, st));
        }
    }
    return T3D_OK;
}

t3d_status launch_flip_until_clear(ItemTable& tab, int max_sweeps, int32_t* sweeps_done, cudaStream_t st)
{
    if (max_sweeps <= 0) {
        if (sweeps_done) T3D_CUDA_CHECK(cudaMemsetAsync(sweeps_done, 0, sizeof(int32_t), st));
        return T3D_OK;
    }
    for (int i = 0; i < tab.n; ++i) {
        T3D_REQUIRE(tab.it[i].stop != nullptr, "flip until clear: item %d has no flag words", i);
        T3D_CUDA_CHECK(cudaMemsetAsync(tab.it[i].stop, 0, kStopWords * sizeof(uint32_t), st));
    }
    T3D_TRY(launch_sweeps(tab, "F", 1, max_sweeps, 0, 0, 0, st));
    ProfScope prof(T3D_K_FLIP, st);
    for (int i = 0; i < tab.n; ++i) {
        const ItemDesc& d = tab.it[i];
        const int64_t n = (int64_t)3 * d.lat.L3 * d.W;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
        k_flip_finish<<<grid, 256, 0, st>>>(d, max_sweeps, i == 0 ? sweeps_done : nullptr);
        T3D_LAUNCH_CHECK("flip until clear: finish");
    }
    return T3D_OK;
}

t3d_status launch_logical(ItemTable& tab, cudaStream_t st)
{
    for (int i = 0; i < tab.n; ++i) {
        ItemDesc& d = tab.it[i];
        d.blocks = (d.W + kLogWords - 1) / kLogWords;
        if (d.counts8) T3D_CUDA_CHECK(cudaMemsetAsync(d.counts8, 0, 8 * sizeof(int64_t), st));
    }
    finish_table(tab);
    ProfScope prof(T3D_K_LOGICAL, st);
    k_logical<<<persistent_grid((const void*)k_logical, kLogWords * kLogSplit, T3D_K_LOGICAL, tab.prefix[tab.n],
                                has_live(tab)),
                kLogWords * kLogSplit, 0, st>>>(tab);
    T3D_LAUNCH_CHECK("logical");
    return T3D_OK;
}

// The fallback gate splits the faces over Y block rows so that a launch has about four
// blocks per SM of a GB300 (152 SMs).  The split only shapes the grid and the scratch size
// (the counts are exact for any Y), and it is computed without a device so that workspace
// sizes can be asked for on the host alone.
constexpr int kGateGridSms = 152;

int gate_splits(int L, int64_t W)
{
    const int64_t faces = 3LL * L * L * L;
    const int64_t tiles = (W + 31) / 32;
    int64_t y = (4 * kGateGridSms + tiles - 1) / tiles;     // about four blocks per SM
    y = std::min<int64_t>(y, (faces + 8 * 64 - 1) / (8 * 64));  // at least 64 faces per warp
    return (int)std::max<int64_t>(1, std::min<int64_t>(y, 64));
}

size_t gate_scratch_bytes(int L, int64_t W)
{
    return (size_t)gate_splits(L, W) * kWeightBits * (size_t)W * sizeof(uint64_t);
}

t3d_status launch_gate(const Lattice& lat, int64_t W, const uint64_t* s, uint32_t max_weight, uint8_t* gate,
                       unsigned long long* n_flagged, uint64_t* scratch, cudaStream_t st)
{
    ProfScope prof(T3D_K_LOGICAL, st);
    const int Y = gate_splits(lat.L, W);
    const int64_t faces = 3LL * lat.L3;
    const int64_t per_y = (faces + Y - 1) / Y;
    k_gate_count<<<dim3((unsigned)((W + 31) / 32), (unsigned)Y), 256, 0, st>>>(lat, W, s, per_y, scratch);
    T3D_LAUNCH_CHECK("fallback gate count");
    k_gate_decide<<<(unsigned)((W + 255) / 256), 256, 0, st>>>(W, Y, scratch, max_weight, gate, n_flagged);
    T3D_LAUNCH_CHECK("fallback gate decide");
    return T3D_OK;
}

namespace {

// Fallback compaction.  k_compact_words: one block lists the flagged words of
// gate[0..W) in increasing order (wsrc) and their count (*live), by a block
// prefix sum over 1024 flags at a time.
constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads)
k_compact_words(const uint8_t* __restrict__ gate, int64_t W, uint32_t* __restrict__ wsrc, int64_t* __restrict__ live)
{
    __shared__ int warp_base[kCompactThreads / 32];
    __shared__ int total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t base = 0;
    for (int64_t c0 = 0; c0 < W; c0 += kCompactThreads) {
        const int64_t w = c0 + threadIdx.x;
        const bool f = w < W && gate[w] != 0;
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_base[warp] = __popc(b);
        __syncthreads();
        if (warp == 0) {
            const int v = warp_base[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            warp_base[lane] = incl - v;
            if (lane == 31) total = incl;
        }
        __syncthreads();
        if (f) wsrc[base + warp_base[warp] + __popc(b & ((1u << lane) - 1u))] = (uint32_t)w;
        base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *live = base;
}

// Copy the live word columns between the batch arrays (row stride W) and their
// compacted copies: gather a[r][wsrc[k]] -> c[r][k], or scatter back.  A warp
// takes one row and strides over the live columns.
__global__ void __launch_bounds__(kThreads)
k_move_words(int64_t rows, int64_t W, const int64_t* __restrict__ live, const uint32_t* __restrict__ wsrc,
             uint64_t* a0, uint64_t* c0, uint64_t* a1, uint64_t* c1, bool gather)
{
    const int64_t n = *live;
    if (n == 0) return;
    const int lane = threadIdx.x & 31;
    for (int64_t r = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); r < rows;
         r += (int64_t)gridDim.x * (kThreads / 32)) {
        for (int64_t k = lane; k < n; k += 32) {
            const int64_t ia = r * W + wsrc[k], ic = r * W + k;
            if (gather) {
                c0[ic] = a0[ia];
                c1[ic] = a1[ia];
            } else {
                a0[ia] = c0[ic];
                a1[ia] = c1[ic];
            }
        }
    }
}

}  // namespace

t3d_status launch_compact_words(const uint8_t* gate, int64_t W, uint32_t* wsrc, int64_t* live, cudaStream_t st)
{
    ProfScope prof(T3D_K_LOGICAL, st);
    k_compact_words<<<1, kCompactThreads, 0, st>>>(gate, W, wsrc, live);
    T3D_LAUNCH_CHECK("fallback word compaction");
    return T3D_OK;
}

t3d_status launch_move_words(const Lattice& lat, int64_t W, const int64_t* live, const uint32_t* wsrc, uint64_t* e,
                             uint64_t* e_c, uint64_t* s, uint64_t* s_c, bool gather, cudaStream_t st)
{
    const int64_t rows = 3LL * lat.L3;
    const int64_t blocks = std::min<int64_t>((rows + kThreads / 32 - 1) / (kThreads / 32), 152LL * 8);
    ProfScope prof(T3D_K_LOGICAL, st);
    k_move_words<<<(unsigned)blocks, kThreads, 0, st>>>(rows, W, live, wsrc, e, e_c, s, s_c, gather);
    T3D_LAUNCH_CHECK("fallback word gather / scatter");
    return T3D_OK;
}

namespace {

// A one-item table for the single-lattice entry points.
ItemTable single_item(int L, int64_t words, int64_t n_samples, uint64_t group0, uint64_t* e, uint64_t* s,
                      uint64_t* tmp)
{
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = 1;
    ItemDesc& d = tab.it[0];
    d.lat = make_lattice_host(L);
    d.W = words;
    d.n_samples = n_samples;
    d.group0 = group0;
    d.e = e;
    d.s = s;
    d.tmp = tmp;
    return tab;
}

}  // namespace
}  // namespace t3d

using namespace t3d;

// ----------------------------------------------------------------- C ABI
extern "C" size_t toric3d_gate_workspace_bytes(int L, int64_t words)
{
    if (L < 2 || L > 1024 || words < 1) return 0;
    return gate_scratch_bytes(L, words);
}

extern "C" t3d_status toric3d_gate(int L, int64_t words, const uint64_t* s, uint32_t max_weight, uint8_t* gate,
                                   int64_t* n_flagged, void* work, size_t work_bytes, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(gate != nullptr, "gate is NULL");
    T3D_REQUIRE(n_flagged == nullptr || aligned(n_flagged, 8), "n_flagged must be 8-byte aligned");
    T3D_TRY(check_words(static_cast<const uint64_t*>(work), "work"));
    T3D_REQUIRE(work_bytes >= gate_scratch_bytes(L, words), "workspace %zu bytes < %zu needed", work_bytes,
                gate_scratch_bytes(L, words));
    return launch_gate(make_lattice_host(L), words, s, max_weight, gate,
                       reinterpret_cast<unsigned long long*>(n_flagged), static_cast<uint64_t*>(work),
                       as_stream(stream));
}

extern "C" t3d_status toric3d_noise(int L, int64_t words, uint64_t* e, double p, uint64_t seed,
                                    uint64_t sample0, uint32_t cycle, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(p >= 0.0 && p <= 1.0, "p=%g outside [0,1]", p);
    T3D_REQUIRE(sample0 % 64 == 0, "sample0 must be a multiple of 64");
    ItemTable tab = single_item(L, words, words * 64, sample0 / 64, e, nullptr, nullptr);
    return launch_noise(tab, prob_threshold(p), seed, cycle, as_stream(stream));
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
    ItemTable tab = single_item(L, words, words * 64, sample0 / 64, const_cast<uint64_t*>(e), s, nullptr);
    return launch_syndrome(tab, prob_threshold(q), seed, cycle, as_stream(stream));
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
    T3D_REQUIRE((uint64_t)sweep0 + (uint64_t)n_apply <= kMaxSweep, "sweep indices must stay below 2^22");
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
    ItemTable tab = single_item(L, words, words * 64, sample0 / 64, e, s, static_cast<uint64_t*>(work));
    return launch_sweeps(tab, schedule, (int)slen, n_apply, sweep0, seed, cycle, as_stream(stream));
}

extern "C" t3d_status toric3d_flip(int L, int64_t words, uint64_t* e, uint64_t* s, int sweeps,
                                   void* work, size_t work_bytes, t3d_stream stream)
{
    clear_error();
    return sweeps_common(L, words, e, s, "F", sweeps, 0, 0, 0, 0, work, work_bytes, stream);
}

extern "C" size_t toric3d_flip_until_clear_workspace_bytes(int L, int64_t words)
{
    const size_t b = toric3d_flip_workspace_bytes(L, words);
    return b ? (b + 255) / 256 * 256 + 256 : 0;
}

extern "C" t3d_status toric3d_flip_until_clear(int L, int64_t words, uint64_t* e, uint64_t* s, int max_sweeps,
                                               int32_t* sweeps_done, void* work, size_t work_bytes,
                                               t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(max_sweeps >= 0 && (uint64_t)max_sweeps <= kMaxSweep, "max_sweeps must be in [0, 2^22]");
    T3D_REQUIRE(sweeps_done == nullptr || aligned(sweeps_done, 4), "sweeps_done must be 4-byte aligned");
    T3D_REQUIRE(work != nullptr && aligned(work, 16), "work must be a 16-byte aligned device pointer");
    const size_t need = toric3d_flip_until_clear_workspace_bytes(L, words);
    T3D_REQUIRE(work_bytes >= need, "workspace too small: %zu < %zu", work_bytes, need);
    ItemTable tab = single_item(L, words, words * 64, 0, e, s, static_cast<uint64_t*>(work));
    tab.it[0].stop = reinterpret_cast<uint32_t*>(static_cast<char*>(work) + need - 256);
    return launch_flip_until_clear(tab, max_sweeps, sweeps_done, as_stream(stream));
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
    ItemTable tab = single_item(L, words_for(n_samples), n_samples, 0, const_cast<uint64_t*>(e), nullptr,
                                nullptr);
    tab.it[0].mask = mask;
    tab.it[0].counts8 = reinterpret_cast<unsigned long long*>(counts8);
    return launch_logical(tab, as_stream(stream));
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
