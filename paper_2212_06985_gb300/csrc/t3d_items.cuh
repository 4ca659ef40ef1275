// Work items for persistent multi-lattice launches.
//
// A batch holds up to kMaxItems independent ensembles, each with its own
// lattice size L, sample count and buffers.  Every kernel of a run is launched
// once per step for the whole batch: the item table travels by value in the
// kernel parameters, each item needs `blocks` thread blocks of work, and a
// persistent grid (a multiple of the SM count) walks the concatenated block
// ranges with a grid-stride loop, so uneven lattices share one launch and no
// SM idles at the tail of a small item.
#pragma once

#include <cstdint>

#include "t3d_device.cuh"

namespace t3d {

constexpr int kMaxItems = 8;

struct ItemDesc {
    Lattice lat;
    int64_t W;            // 64-bit words per bit-sliced row (row stride)
    int64_t nw;           // bit-sliced kernels: words to process from the row start (0 = W)
    int64_t n_samples;
    uint64_t group0;      // global index of the item's first 64-sample word
    uint64_t* e;          // bit-sliced error state [3L^3][W]
    uint64_t* s;          // bit-sliced syndrome [3L^3][W]
    uint64_t* tmp;        // ping-pong syndrome for synchronous applications
    float* msg_in;        // BP messages of the current chunk (nullptr: priors)
    float* msg_out;
    uint4* syn;           // BP per-word syndrome copy of the current chunk
    float* llr;           // optional posteriors [3L^3][n_samples]
    uint8_t* mask;
    unsigned long long* counts8;
    int64_t w0;           // BP: first 64-sample word of the current chunk
    int64_t words;        // BP: words in the current chunk
    // Compacted word columns (the learned decoder's fallback): when live is set, only the
    // words w0 + w < *live hold data and the others are skipped; word w of the arrays is
    // word wsrc[w] of the batch (its random numbers are keyed by group0 + wsrc[w]).  A
    // launch over a single such item walks only the blocks that hold live words: local
    // block lb covers words [(lb / live_bpu) * live_wpu, + live_wpu) of the launch.
    const int64_t* live;  // device, nullable
    const uint32_t* wsrc; // device, nullable
    int64_t live_bpu;     // blocks per unit of live_wpu words (set by each launcher)
    int live_wpu;
    // Flip until clear (nullable): stop[0..2] a ring of "an unsatisfied check is left" flags of
    // the applications (application k writes slot k % 3), stop[3] the applications after the
    // first that ran, stop[4] whether the first application's input had an unsatisfied check.
    // Application k runs only if application k - 1 left an unsatisfied check in the item.
    uint32_t* stop;
    int stop_k;           // index of the application being launched
    int tx;               // bit-sliced kernels: words per thread-block row (power of 2)
    int64_t blocks;       // thread blocks this item needs in the current launch
};

struct ItemTable {
    int n;
    int64_t prefix[kMaxItems + 1];   // prefix[i] = first block of item i
    ItemDesc it[kMaxItems];
};

// Item owning global block b of the concatenated ranges (n <= 8: linear scan).
__device__ __forceinline__ int item_of(const ItemTable& tab, int64_t b)
{
    int i = 0;
    while (i + 1 < tab.n && b >= tab.prefix[i + 1]) ++i;
    return i;
}

// Whether word w (of the launch's word range) holds data.
__device__ __forceinline__ bool word_live(const ItemDesc& d, int64_t w)
{
    return d.live == nullptr || d.w0 + w < *d.live;
}

// Group (64-sample word of the whole batch) that keys word w's random numbers.
__device__ __forceinline__ uint64_t word_group(const ItemDesc& d, int64_t w)
{
    return d.group0 + (d.wsrc ? (uint64_t)d.wsrc[w] : (uint64_t)w);
}

// Blocks of a compacted single-item launch that hold live words.
__device__ __forceinline__ int64_t live_blocks(const ItemDesc& d)
{
    if (d.live_wpu <= 0) return d.blocks;   // launcher without a live layout: per-word checks only
    const int64_t lw = *d.live - d.w0;
    if (lw <= 0) return 0;
    const int64_t b = (lw + d.live_wpu - 1) / d.live_wpu * d.live_bpu;
    return b < d.blocks ? b : d.blocks;
}

// Persistent grid-stride walk over every item's blocks: f(item, local block).
// The bound is uniform across a thread block, so f may synchronise the block.
template <class F>
__device__ __forceinline__ void for_each_item_block(const ItemTable& tab, F&& f)
{
    int64_t total = tab.prefix[tab.n];
    if (tab.n == 1 && tab.it[0].live) total = live_blocks(tab.it[0]);
    for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = item_of(tab, b);
        f(tab.it[i], b - tab.prefix[i]);
    }
}

inline bool has_live(const ItemTable& tab)
{
    for (int i = 0; i < tab.n; ++i)
        if (tab.it[i].live) return true;
    return false;
}

inline void finish_table(ItemTable& tab)
{
    tab.prefix[0] = 0;
    for (int i = 0; i < tab.n; ++i) tab.prefix[i + 1] = tab.prefix[i] + tab.it[i].blocks;
}

}  // namespace t3d
