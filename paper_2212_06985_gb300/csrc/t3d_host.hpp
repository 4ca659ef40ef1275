// Host-side helpers shared by the toric3d translation units: the per-thread
// error message, argument checks, and launch-error capture.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/toric3d.h"
#include "t3d_device.cuh"

namespace t3d {

void set_error(const char* fmt, ...);
void clear_error();

// Largest lattice accepted: 3 L^3 must index comfortably in 32 bits.
constexpr int kMaxL = 256;

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Byte ranges [a, a + na) and [b, b + nb) share no byte.
inline bool disjoint(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x + na <= y || y + nb <= x;
}

inline uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ULL << 32;
    return (uint64_t)(p * 4294967296.0 + 0.5);
}

inline int64_t words_for(int64_t n_samples) { return (n_samples + 63) / 64; }
inline int64_t groups_for(int64_t n_samples) { return (n_samples + 31) / 32; }

inline cudaStream_t as_stream(t3d_stream s) { return reinterpret_cast<cudaStream_t>(s); }

#define T3D_REQUIRE(cond, ...)            \
    do {                                  \
        if (!(cond)) {                    \
            ::t3d::set_error(__VA_ARGS__); \
            return T3D_EINVAL;            \
        }                                 \
    } while (0)

#define T3D_CUDA_CHECK(expr)                                                              \
    do {                                                                                  \
        cudaError_t err_ = (expr);                                                        \
        if (err_ != cudaSuccess) {                                                        \
            ::t3d::set_error("%s failed: %s", #expr, cudaGetErrorString(err_));           \
            return T3D_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define T3D_LAUNCH_CHECK(what)                                                            \
    do {                                                                                  \
        cudaError_t err_ = cudaGetLastError();                                            \
        if (err_ != cudaSuccess) {                                                        \
            ::t3d::set_error("launch of %s failed: %s", what, cudaGetErrorString(err_));  \
            return T3D_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define T3D_TRY(expr)                      \
    do {                                   \
        t3d_status st_ = (expr);           \
        if (st_ != T3D_OK) return st_;     \
    } while (0)

// Kernel timing: prof_begin() returns a handle (or -1 when profiling is off
// or the stream is capturing) and records a start event; prof_end() records
// the matching stop event after the launch.
int prof_begin(int kind, cudaStream_t st);
void prof_end(int handle, cudaStream_t st);

struct ProfScope {
    int h;
    cudaStream_t st;
    ProfScope(int kind, cudaStream_t s) : h(prof_begin(kind, s)), st(s) {}
    ~ProfScope() { prof_end(h, st); }
};

t3d_status check_lattice(int L);
t3d_status check_words(const void* p, const char* name);

// Grid size for a grid-stride kernel with `blocks` work units: one block per
// unit by default; with a tuned cap of c blocks per SM, a persistent grid of
// SMs x min(c, resident blocks) that walks the units.
// device_bound: the launch's work is bounded by a device-side count (ItemDesc::live); the
// grid is then at most the resident blocks even when untuned.
unsigned persistent_grid(const void* kernel, int threads, int kind, int64_t blocks, bool device_bound = false,
                         size_t dynamic_smem = 0);
// Raise a kernel's dynamic shared-memory limit in the current context to at least `bytes`.
t3d_status allow_dynamic_smem(const void* kernel, size_t bytes);
// Unique id of the calling thread's current CUDA context, 0 if there is none yet.
t3d_status current_context_id(unsigned long long* id);

// Launch tuning chosen by the autotuner (0 = use the occupancy limit).
int tuned_blocks_per_sm(int kind);
void set_tuned_blocks_per_sm(int kind, int blocks_per_sm);

// Kernel launchers over an item table (see t3d_items.cuh).  Each fills the
// items' `blocks` (and `tx`) for its own kernel; no argument validation.
struct ItemTable;
t3d_status launch_noise(ItemTable& tab, uint64_t thr, uint64_t seed, uint32_t cycle, cudaStream_t st);
t3d_status launch_syndrome(ItemTable& tab, uint64_t thr, uint64_t seed, uint32_t cycle,
                           cudaStream_t st);
// n_apply applications cycling through `schedule`; uses each item's e, s and
// tmp and leaves the result in s.
// Flip until clear: up to max_sweeps flip applications, each item's stop after its syndrome
// clears (every item needs ItemDesc::stop, kStopWords words of device memory); the count of
// applications of item 0 that ran goes to *sweeps_done (device, nullable).
constexpr int kStopWords = 8;
t3d_status launch_flip_until_clear(ItemTable& tab, int max_sweeps, int32_t* sweeps_done, cudaStream_t st);
t3d_status launch_sweeps(ItemTable& tab, const char* schedule, int slen, int n_apply,
                         uint32_t sweep0, uint64_t seed, uint32_t cycle, cudaStream_t st);
t3d_status launch_logical(ItemTable& tab, cudaStream_t st);
// e ^= d, s ^= H d from decision words dec[word][site][4] (32-bit halves).
t3d_status launch_dec_apply(const Lattice& lat, int64_t W, int64_t words, const uint64_t* dec, uint64_t* e,
                            uint64_t* s, cudaStream_t st);
// gate[w] = 1 iff some sample of word w has more than max_weight unsatisfied
// checks in s; *n_flagged (nullable) += flagged words.  scratch holds
// gate_scratch_bytes(L, W) bytes.
size_t gate_scratch_bytes(int L, int64_t W);
// Fallback compaction: wsrc[0..*live) = the flagged words of gate[0..W), in
// order; then gather (or scatter back) those word columns of e and s into (from)
// the first *live columns of e_c and s_c (same row stride W).
t3d_status launch_compact_words(const uint8_t* gate, int64_t W, uint32_t* wsrc, int64_t* live, cudaStream_t st);
t3d_status launch_move_words(const Lattice& lat, int64_t W, const int64_t* live, const uint32_t* wsrc, uint64_t* e,
                             uint64_t* e_c, uint64_t* s, uint64_t* s_c, bool gather, cudaStream_t st);
t3d_status launch_gate(const Lattice& lat, int64_t W, const uint64_t* s, uint32_t max_weight, uint8_t* gate,
                       unsigned long long* n_flagged, uint64_t* scratch, cudaStream_t st);

// Learned pre-decoder pass (t3d_cnn.cu) on a batch or a chunk of one (rows of
// stride W words).
t3d_status launch_cnn_decode(int L, int64_t n_samples, int64_t W, const uint64_t* s_prev, uint64_t* s,
                             uint64_t* e, const void* blob, float* logits_out, void* work, cudaStream_t st);
size_t cnn_workspace_bytes(int L, int64_t n_samples);

// Bytes of BP workspace per 64-sample word (two message buffers + syndrome copy).
size_t bp_bytes_per_word(int L);
// BP over every item (e, s, n_samples, W of each); bufs[i] is item i's chunk
// workspace holding chunk_words[i] words.
t3d_status launch_bp(const ItemTable& items, double p, double q_meas, int iters, float* const* bufs,
                     const int64_t* chunk_words, float* llr_out, cudaStream_t st);
// Times the BP iteration on the items' first chunks under each blocks-per-SM
// cap and keeps the fastest in the tuning table (synchronises the stream).
t3d_status autotune_bp(const ItemTable& items, double p, double q_meas, float* const* bufs,
                       const int64_t* chunk_words, cudaStream_t st, int* best_cap, float* best_ms);

// BP with meta-checks (t3d_bp_meta.cu): workspace bytes per 64-sample word and
// the decoder on n_samples samples in rows of stride W words, chunked to fit.
namespace meta {
size_t bytes_per_word(int L);
t3d_status launch_bp_meta(const Lattice& lat, int64_t n_samples, int64_t W, uint64_t* e, uint64_t* s, double p,
                          double q, int iters, void* work, size_t work_bytes, float* llr_out, cudaStream_t st);
}  // namespace meta

}  // namespace t3d
