// Whole Monte Carlo runs: T code cycles of noise, noisy measurement and
// decoding (Sec. 3.1 Fig. 2, Sec. 3.2 schedules, Sec. 4.2 p-BP), an optional
// noiseless final round, and the logical readout.  A run covers a batch of up
// to eight ensembles of different lattice sizes; every step is one persistent
// launch over all of them (t3d_items.cuh).  The whole T-cycle sequence can be
// captured into a CUDA graph, instantiated once per distinct run and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "t3d_cnn.cuh"
#include "t3d_host.hpp"
#include "t3d_items.cuh"

namespace t3d {
namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t state_bytes(int L, int64_t n_samples)
{
    return (size_t)3 * L * L * L * (size_t)words_for(n_samples) * sizeof(uint64_t);
}


struct Plan {
    ItemTable items;
    float* bp[kMaxItems];
    int64_t chunk[kMaxItems];      // BP / pre-decoder chunk, words
    // learned decoder
    uint64_t* s_prev[kMaxItems];
    uint64_t* s_raw[kMaxItems];
    uint8_t* gate[kMaxItems];
    uint64_t* gate_scratch[kMaxItems];
    uint32_t gate_weight[kMaxItems];   // fallback threshold of each item
    uint32_t* wsrc[kMaxItems];         // flagged words, compacted
    int64_t* live[kMaxItems];          // their number (device)
    uint64_t* e_c[kMaxItems];          // the flagged words' e and s columns, compacted
    uint64_t* s_c[kMaxItems];
    uint64_t* e_pre[kMaxItems];        // the error state before the cycle's decoding
    unsigned long long* n_fallback[kMaxItems];
    void* cnn_work[kMaxItems];
    int64_t cnn_chunk[kMaxItems];  // pre-decoder chunk, words
    uint32_t* stop[kMaxItems];     // perfect round: the flags of the flip until clear
};

bool learned(const t3d_run_cfg& c) { return c.cnn_blob != nullptr; }

bool needs_bp(const t3d_run_cfg& c)
{
    return c.bp_iters > 0 && (c.use_bp || (learned(c) && c.fallback_max_weight >= 0));
}

// bp_meas_nodes == 2: BP with the cube meta-checks over the measurement variables
bool meta_checks(const t3d_run_cfg& c) { return c.use_bp && c.bp_meas_nodes == 2; }

size_t bp_word_bytes(const t3d_run_cfg& c, int L)
{
    return meta_checks(c) ? meta::bytes_per_word(L) : bp_bytes_per_word(L);
}

t3d_status validate_cfg(const t3d_run_cfg* c)
{
    T3D_REQUIRE(c != nullptr, "cfg is NULL");
    T3D_REQUIRE(c->T >= 0, "T must be >= 0");
    T3D_REQUIRE(c->p >= 0.0 && c->p <= 1.0 && c->q >= 0.0 && c->q <= 1.0, "p, q must lie in [0,1]");
    T3D_REQUIRE(c->n_apply >= 0 && c->n_apply <= (int)kMaxSweep, "n_apply must lie in [0, 2^22]");
    T3D_REQUIRE(!c->perfect_round || c->perfect_max_sweeps <= (int)kMaxSweep, "perfect_max_sweeps must be <= 2^22");
    size_t slen = strnlen(c->schedule, sizeof(c->schedule));
    T3D_REQUIRE(slen < sizeof(c->schedule), "schedule must be NUL-terminated");
    T3D_REQUIRE(c->n_apply == 0 || slen >= 1, "n_apply > 0 needs a schedule");
    for (size_t i = 0; i < slen; ++i)
        T3D_REQUIRE(c->schedule[i] == 'F' || c->schedule[i] == 'P', "schedule may hold only 'F' and 'P'");
    if (c->cnn_blob) {
        T3D_REQUIRE(!c->use_bp, "the learned decoder replaces BP: use_bp must be 0");
        T3D_REQUIRE(aligned(c->cnn_blob, 16), "cnn_blob must be 16-byte aligned");
        T3D_REQUIRE(c->fallback_max_weight < 0 || c->bp_iters > 0, "the BP fallback needs bp_iters > 0");
        T3D_REQUIRE(c->fallback_sigmas >= 0.0 && c->fallback_sigmas <= 1000.0, "fallback_sigmas must lie in [0, 1000]");
    }
    if (c->use_bp || (c->cnn_blob && c->fallback_max_weight >= 0)) {
        T3D_REQUIRE(c->p > 0.0 && c->p < 1.0, "BP needs 0 < p < 1");
        T3D_REQUIRE(c->bp_iters >= 0, "bp_iters must be >= 0");
        T3D_REQUIRE(c->bp_meas_nodes >= 0 && c->bp_meas_nodes <= 2, "bp_meas_nodes must be 0, 1 or 2");
        T3D_REQUIRE(!c->bp_meas_nodes || c->q < 0.5, "measurement nodes need q < 0.5");
        T3D_REQUIRE(c->bp_meas_nodes != 2 || (c->use_bp && c->q > 0.0),
                    "meta-checks (bp_meas_nodes = 2) need use_bp and q > 0");
        T3D_REQUIRE(c->bp_chunk_samples >= 0, "bp_chunk_samples must be >= 0");
    }
    T3D_REQUIRE(!c->perfect_round || c->perfect_max_sweeps >= 0, "perfect_max_sweeps must be >= 0");
    return T3D_OK;
}

t3d_status validate_items(const t3d_run_cfg* c, const t3d_batch_item* items, int n_items)
{
    T3D_REQUIRE(items != nullptr && n_items >= 1 && n_items <= kMaxItems, "need 1..%d batch items", kMaxItems);
    for (int i = 0; i < n_items; ++i) {
        const t3d_batch_item& it = items[i];
        T3D_TRY(check_lattice(it.L));
        T3D_REQUIRE(!needs_bp(*c) || it.L <= 128, "BP supports L <= 128 (item %d has L=%d)", i, it.L);
        T3D_REQUIRE(it.n_samples >= 1 && words_for(it.n_samples) <= (1LL << 31), "item %d: n_samples out of range", i);
        T3D_REQUIRE(it.sample0 % 64 == 0, "item %d: sample0 must be a multiple of 64", i);
        T3D_TRY(check_words(it.e, "item e"));
        T3D_REQUIRE(it.counts8 == nullptr || aligned(it.counts8, 8), "item %d: counts8 must be 8-byte aligned", i);
        if (c->cnn_blob) {
            T3D_REQUIRE(it.L <= 128, "the pre-decoder supports L <= 128 (item %d has L=%d)", i, it.L);
            T3D_TRY(check_words(it.s_prev, "item s_prev"));
            T3D_REQUIRE(it.fallback_words == nullptr || aligned(it.fallback_words, 8),
                        "item %d: fallback_words must be 8-byte aligned", i);
        }
    }
    return T3D_OK;
}

// 64-sample words per BP chunk for every item: all words (one round) when the
// workspace allows, else the fewest rounds that fit.
bool bp_chunks(const t3d_run_cfg& c, const t3d_batch_item* items, int n, size_t avail, int64_t* chunk)
{
    int64_t max_words = 0;
    for (int i = 0; i < n; ++i) max_words = std::max(max_words, words_for(items[i].n_samples));
    for (int64_t rounds = 1; rounds <= max_words; ++rounds) {
        size_t need = 0;
        for (int i = 0; i < n; ++i) {
            const int64_t Wi = words_for(items[i].n_samples);
            int64_t w = (Wi + rounds - 1) / rounds;
            if (c.bp_chunk_samples > 0) w = std::min(w, words_for(c.bp_chunk_samples));
            chunk[i] = w;
            need += round_up((size_t)w * bp_word_bytes(c, items[i].L));
        }
        if (need <= avail) return true;
    }
    return false;
}

// Pre-decoder chunk (words): cfg.bp_chunk_samples, or by default as many
// samples as keep the pre-decoder's activations within kCnnAutoBytes.
constexpr size_t kCnnAutoBytes = 16ull << 30;

int64_t cnn_chunk_words(const t3d_run_cfg& c, int L, int64_t n_samples)
{
    const int64_t Wi = words_for(n_samples);
    if (c.bp_chunk_samples > 0) return std::min(Wi, words_for(c.bp_chunk_samples));
    const size_t per_sample = cnn_workspace_bytes(L, 128) / 128 + 1;
    const int64_t fit = (int64_t)(kCnnAutoBytes / per_sample) / 128 * 128;
    return std::min(Wi, std::max<int64_t>(2, words_for(fit)));
}

// Fallback threshold of a lattice: fallback_max_weight, plus with
// fallback_sigmas > 0 the expected number of measurement errors among the 3L^3
// checks and that many standard deviations (binomial): a sample is sent back to
// BP when its decoded syndrome keeps more unsatisfied checks than the noisy
// measurement alone explains.
uint32_t fallback_weight(const t3d_run_cfg& c, int L)
{
    double w = (double)c.fallback_max_weight;
    if (c.fallback_sigmas > 0.0) {
        const double n = 3.0 * L * L * L;
        w += std::floor(c.q * n + c.fallback_sigmas * std::sqrt(c.q * (1.0 - c.q) * n));
    }
    return (uint32_t)std::min(w, 4294967295.0);
}

size_t learned_bytes(const t3d_run_cfg& c, int L, int64_t n_samples)
{
    const int64_t cw = cnn_chunk_words(c, L, n_samples);
    size_t b = round_up(state_bytes(L, n_samples)) + round_up(cnn_workspace_bytes(L, std::min(n_samples, cw * 64)));
    if (c.fallback_max_weight >= 0) {
        const int64_t Wi = words_for(n_samples);
        b += round_up((size_t)Wi) + round_up(gate_scratch_bytes(L, Wi)) + round_up((size_t)Wi * sizeof(uint32_t)) +
             round_up(sizeof(int64_t)) + 3 * round_up(state_bytes(L, n_samples));
    }
    return b;
}

size_t batch_workspace_bytes(const t3d_run_cfg& c, const t3d_batch_item* items, int n)
{
    size_t total = 0;
    for (int i = 0; i < n; ++i) total += 2 * round_up(state_bytes(items[i].L, items[i].n_samples));
    if (c.perfect_round) total += (size_t)n * round_up(kStopWords * sizeof(uint32_t));
    if (learned(c))
        for (int i = 0; i < n; ++i) total += learned_bytes(c, items[i].L, items[i].n_samples);
    if (needs_bp(c)) {
        for (int i = 0; i < n; ++i) {
            const int64_t Wi = words_for(items[i].n_samples);
            const int64_t w = c.bp_chunk_samples > 0 ? std::min(Wi, words_for(c.bp_chunk_samples)) : Wi;
            total += round_up((size_t)w * bp_word_bytes(c, items[i].L));
        }
    }
    return total;
}

t3d_status plan_workspace(const t3d_run_cfg& c, const t3d_batch_item* items, int n, void* work,
                          size_t work_bytes, Plan& pl)
{
    T3D_REQUIRE(work != nullptr && aligned(work, kAlign), "work must be a 256-byte aligned device pointer");
    std::memset(&pl, 0, sizeof(pl));
    char* base = static_cast<char*>(work);
    size_t used = 0;
    pl.items.n = n;
    for (int i = 0; i < n; ++i) {
        const size_t sb = round_up(state_bytes(items[i].L, items[i].n_samples));
        T3D_REQUIRE(used + 2 * sb <= work_bytes, "workspace too small: %zu bytes", work_bytes);
        ItemDesc& d = pl.items.it[i];
        d.lat = make_lattice_host(items[i].L);
        d.W = words_for(items[i].n_samples);
        d.n_samples = items[i].n_samples;
        d.group0 = items[i].sample0 / 64;
        d.e = items[i].e;
        d.s = reinterpret_cast<uint64_t*>(base + used);
        d.tmp = reinterpret_cast<uint64_t*>(base + used + sb);
        d.mask = items[i].mask;
        d.counts8 = reinterpret_cast<unsigned long long*>(items[i].counts8);
        used += 2 * sb;
    }
    if (c.perfect_round) {
        for (int i = 0; i < n; ++i) {
            T3D_REQUIRE(used + round_up(kStopWords * sizeof(uint32_t)) <= work_bytes, "workspace too small");
            pl.stop[i] = reinterpret_cast<uint32_t*>(base + used);
            used += round_up(kStopWords * sizeof(uint32_t));
        }
    }
    if (learned(c)) {
        for (int i = 0; i < n; ++i) {
            const size_t sb = round_up(state_bytes(items[i].L, items[i].n_samples));
            T3D_REQUIRE(used + learned_bytes(c, items[i].L, items[i].n_samples) <= work_bytes,
                        "workspace too small for the learned decoder");
            pl.s_prev[i] = items[i].s_prev;
            pl.s_raw[i] = reinterpret_cast<uint64_t*>(base + used);
            used += sb;
            pl.n_fallback[i] = reinterpret_cast<unsigned long long*>(items[i].fallback_words);
            if (c.fallback_max_weight >= 0) {
                const int64_t Wi = words_for(items[i].n_samples);
                pl.gate[i] = reinterpret_cast<uint8_t*>(base + used);
                used += round_up((size_t)Wi);
                pl.gate_scratch[i] = reinterpret_cast<uint64_t*>(base + used);
                used += round_up(gate_scratch_bytes(items[i].L, Wi));
                pl.wsrc[i] = reinterpret_cast<uint32_t*>(base + used);
                used += round_up((size_t)Wi * sizeof(uint32_t));
                pl.live[i] = reinterpret_cast<int64_t*>(base + used);
                used += round_up(sizeof(int64_t));
                pl.e_c[i] = reinterpret_cast<uint64_t*>(base + used);
                used += sb;
                pl.s_c[i] = reinterpret_cast<uint64_t*>(base + used);
                used += sb;
                pl.e_pre[i] = reinterpret_cast<uint64_t*>(base + used);
                used += sb;
                pl.gate_weight[i] = fallback_weight(c, items[i].L);
            }
            const int64_t cw = cnn_chunk_words(c, items[i].L, items[i].n_samples);
            pl.cnn_work[i] = base + used;
            used += round_up(cnn_workspace_bytes(items[i].L, std::min(items[i].n_samples, cw * 64)));
            pl.cnn_chunk[i] = cw;
        }
    }
    if (learned(c)) T3D_TRY(cnn::tc_prepare());   // before any stream capture
    if (needs_bp(c)) {
        T3D_REQUIRE(bp_chunks(c, items, n, work_bytes - used, pl.chunk), "workspace too small for BP chunks");
        for (int i = 0; i < n; ++i) {
            pl.bp[i] = reinterpret_cast<float*>(base + used);
            used += round_up((size_t)pl.chunk[i] * bp_word_bytes(c, items[i].L));
        }
    } else if (c.use_bp) {
        for (int i = 0; i < n; ++i) pl.chunk[i] = std::max<int64_t>(1, words_for(items[i].n_samples));
    }

    return T3D_OK;
}

// Copy a word range of a bit-sliced array (3 L^3 rows of stride W words).
t3d_status copy_rows(uint64_t* dst, const uint64_t* src, const ItemDesc& d, int64_t w0, int64_t nw, cudaStream_t st)
{
    const size_t pitch = (size_t)d.W * sizeof(uint64_t);
    T3D_CUDA_CHECK(cudaMemcpy2DAsync(dst + w0, pitch, src + w0, pitch, (size_t)nw * sizeof(uint64_t),
                                     (size_t)3 * d.lat.L3, cudaMemcpyDeviceToDevice, st));
    return T3D_OK;
}

// One cycle of the learned decoder: qubit noise and the noisy measurement of
// every item, the pre-decoder chunk by chunk (each chunk decodes from its own
// (s_prev, s) rows), the flip / p-flip schedule, the optional fallback (gate;
// the flagged words are decoded again from the cycle's start, the error after
// the noise and the measured syndrome, by BP and the schedule, whose result
// replaces the learned one), and s_prev <- the measured s.
// (Running chunks on two streams, so that one chunk's pre-decoder overlaps the
// other's sweeps, measured slower on GB300: the sweeps' blocks delay the
// persistent one-CTA-per-SM convolutions.)
t3d_status enqueue_learned_cycle(const t3d_run_cfg& c, const Plan& pl, uint32_t cycle, uint64_t thr_p,
                                 uint64_t thr_q, int slen, cudaStream_t st)
{
    ItemTable tab = pl.items;
    T3D_TRY(launch_noise(tab, thr_p, c.seed, cycle, st));
    tab = pl.items;
    T3D_TRY(launch_syndrome(tab, thr_q, c.seed, cycle, st));
    for (int i = 0; i < pl.items.n; ++i) {
        const ItemDesc& d = pl.items.it[i];
        T3D_TRY(copy_rows(pl.s_raw[i], d.s, d, 0, d.W, st));
        if (c.fallback_max_weight >= 0) T3D_TRY(copy_rows(pl.e_pre[i], d.e, d, 0, d.W, st));
        for (int64_t w0 = 0; w0 < d.W; w0 += pl.cnn_chunk[i]) {
            const int64_t n = std::min<int64_t>(pl.cnn_chunk[i] * 64, d.n_samples - w0 * 64);
            T3D_TRY(launch_cnn_decode(d.lat.L, n, d.W, pl.s_prev[i] + w0, d.s + w0, d.e + w0, c.cnn_blob, nullptr,
                                      pl.cnn_work[i], st));
        }
    }
    if (c.n_apply > 0) {
        tab = pl.items;
        T3D_TRY(launch_sweeps(tab, c.schedule, slen, c.n_apply, 0, c.seed, cycle, st));
    }
    if (c.fallback_max_weight >= 0) {
        // the flagged words' columns of the cycle's start (error after the noise, measured
        // syndrome) are compacted to the front of two scratch arrays, decoded there by BP + the
        // schedule (every launch walking only the live words), and replace the learned result
        for (int i = 0; i < pl.items.n; ++i) {
            const ItemDesc& d = pl.items.it[i];
            T3D_TRY(launch_gate(d.lat, d.W, d.s, pl.gate_weight[i], pl.gate[i], pl.n_fallback[i],
                                pl.gate_scratch[i], st));
            T3D_TRY(launch_compact_words(pl.gate[i], d.W, pl.wsrc[i], pl.live[i], st));
            T3D_TRY(launch_move_words(d.lat, d.W, pl.live[i], pl.wsrc[i], pl.e_pre[i], pl.e_c[i], pl.s_raw[i],
                                      pl.s_c[i], true, st));
            ItemTable one;
            std::memset(&one, 0, sizeof(one));
            one.n = 1;
            one.it[0] = d;
            one.it[0].e = pl.e_c[i];
            one.it[0].s = pl.s_c[i];
            one.it[0].live = pl.live[i];
            one.it[0].wsrc = pl.wsrc[i];
            T3D_TRY(launch_bp(one, c.p, c.bp_meas_nodes ? c.q : 0.0, c.bp_iters, &pl.bp[i], &pl.chunk[i], nullptr,
                              st));
            if (c.n_apply > 0) T3D_TRY(launch_sweeps(one, c.schedule, slen, c.n_apply, 0, c.seed, cycle, st));
            T3D_TRY(launch_move_words(d.lat, d.W, pl.live[i], pl.wsrc[i], d.e, pl.e_c[i], d.s, pl.s_c[i], false, st));
        }
    }
    for (int i = 0; i < pl.items.n; ++i) T3D_TRY(copy_rows(pl.s_prev[i], pl.s_raw[i], pl.items.it[i], 0, pl.items.it[i].W, st));
    return T3D_OK;
}

t3d_status enqueue_run(const t3d_run_cfg& c, const Plan& pl, cudaStream_t st)
{
    const uint64_t thr_p = prob_threshold(c.p), thr_q = prob_threshold(c.q);
    const int slen = (int)strnlen(c.schedule, sizeof(c.schedule));
    ItemTable tab;
    for (int t = 1; t <= c.T; ++t) {
        const uint32_t cycle = c.cycle0 + (uint32_t)t;
        if (learned(c)) {
            T3D_TRY(enqueue_learned_cycle(c, pl, cycle, thr_p, thr_q, slen, st));
            continue;
        }
        tab = pl.items;
        T3D_TRY(launch_noise(tab, thr_p, c.seed, cycle, st));
        tab = pl.items;
        T3D_TRY(launch_syndrome(tab, thr_q, c.seed, cycle, st));
        if (meta_checks(c)) {
            for (int i = 0; i < pl.items.n; ++i) {
                const ItemDesc& d = pl.items.it[i];
                T3D_TRY(meta::launch_bp_meta(d.lat, d.n_samples, d.W, d.e, d.s, c.p, c.q, c.bp_iters, pl.bp[i],
                                             (size_t)pl.chunk[i] * meta::bytes_per_word(d.lat.L), nullptr, st));
            }
        } else if (c.use_bp) {
            T3D_TRY(launch_bp(pl.items, c.p, c.bp_meas_nodes ? c.q : 0.0, c.bp_iters, pl.bp, pl.chunk,
                              nullptr, st));
        }
        if (c.n_apply > 0) {
            tab = pl.items;
            T3D_TRY(launch_sweeps(tab, c.schedule, slen, c.n_apply, 0, c.seed, cycle, st));
        }
    }
    if (c.perfect_round) {
        const uint32_t cycle = c.cycle0 + (uint32_t)c.T + 1;
        tab = pl.items;
        T3D_TRY(launch_syndrome(tab, 0, c.seed, cycle, st));
        if (c.perfect_max_sweeps > 0) {
            // flip until every item's syndrome clears, at most perfect_max_sweeps applications
            // (the applications after an item clears do no work; the results are those of
            // perfect_max_sweeps applications)
            tab = pl.items;
            for (int i = 0; i < tab.n; ++i) tab.it[i].stop = pl.stop[i];
            T3D_TRY(launch_flip_until_clear(tab, c.perfect_max_sweeps, nullptr, st));
        }
    }
    bool readout = false;
    for (int i = 0; i < pl.items.n; ++i) readout |= pl.items.it[i].mask || pl.items.it[i].counts8;
    if (readout) {
        tab = pl.items;
        T3D_TRY(launch_logical(tab, st));
    }
    return T3D_OK;
}

// ------------------------------------------------------------ graph cache
struct GraphKey {
    t3d_run_cfg cfg;
    t3d_batch_item items[kMaxItems];
    int n_items;
    const void* work;
    size_t work_bytes;
    cudaStream_t stream;
    int device;
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    cudaEvent_t done;    // recorded after every launch of exec
    bool used;
};

constexpr int kGraphCache = 8;
GraphEntry g_graphs[kGraphCache];
int g_graph_next = 0;
std::mutex g_graph_mutex;

t3d_status run_with_graph(const t3d_run_cfg& c, const t3d_batch_item* items, int n, const Plan& pl,
                          void* work, size_t work_bytes, cudaStream_t st)
{
    T3D_REQUIRE(st != nullptr, "use_graph needs a non-default stream");
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.cfg = c;
    std::memcpy(key.items, items, sizeof(t3d_batch_item) * n);
    key.n_items = n;
    key.work = work;
    key.work_bytes = work_bytes;
    key.stream = st;
    T3D_CUDA_CHECK(cudaGetDevice(&key.device));
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    for (auto& g : g_graphs) {
        if (g.used && std::memcmp(&g.key, &key, sizeof(GraphKey)) == 0) {
            T3D_CUDA_CHECK(cudaGraphLaunch(g.exec, st));
            T3D_CUDA_CHECK(cudaEventRecord(g.done, st));
            return T3D_OK;
        }
    }
    T3D_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    t3d_status stq = enqueue_run(c, pl, st);
    cudaGraph_t graph = nullptr;
    cudaError_t end = cudaStreamEndCapture(st, &graph);
    if (stq != T3D_OK) {
        if (graph) cudaGraphDestroy(graph);
        return stq;
    }
    if (end != cudaSuccess) {
        set_error("stream capture failed: %s", cudaGetErrorString(end));
        return T3D_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(inst));
        return T3D_ECUDA;
    }
    GraphEntry& slot = g_graphs[g_graph_next];
    if (slot.used) {
        // the evicted graph's last launch may still be running: wait for it (its event,
        // not its stream, which the caller may have destroyed since) before freeing it
        cudaError_t w = cudaEventSynchronize(slot.done);
        if (w != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            set_error("waiting for an evicted run graph failed: %s", cudaGetErrorString(w));
            return T3D_ECUDA;
        }
        cudaGraphExecDestroy(slot.exec);
        slot.used = false;
    } else {
        cudaError_t ce = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming);
        if (ce != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            set_error("cudaEventCreate failed: %s", cudaGetErrorString(ce));
            return T3D_ECUDA;
        }
    }
    g_graph_next = (g_graph_next + 1) % kGraphCache;
    slot.key = key;
    slot.exec = exec;
    slot.used = true;
    T3D_CUDA_CHECK(cudaGraphLaunch(exec, st));
    T3D_CUDA_CHECK(cudaEventRecord(slot.done, st));
    return T3D_OK;
}

t3d_status run_batch(const t3d_run_cfg* cfg, const t3d_batch_item* items, int n_items, void* work,
                     size_t work_bytes, t3d_stream stream)
{
    T3D_TRY(validate_cfg(cfg));
    T3D_TRY(validate_items(cfg, items, n_items));
    Plan pl;
    T3D_TRY(plan_workspace(*cfg, items, n_items, work, work_bytes, pl));
    cudaStream_t st = as_stream(stream);
    if (cfg->use_graph) return run_with_graph(*cfg, items, n_items, pl, work, work_bytes, st);
    return enqueue_run(*cfg, pl, st);
}

t3d_batch_item single(const t3d_run_cfg* cfg, uint64_t* e, uint8_t* mask, int64_t* counts8)
{
    t3d_batch_item it;
    std::memset(&it, 0, sizeof(it));
    it.L = cfg->L;
    it.n_samples = cfg->n_samples;
    it.sample0 = cfg->sample0;
    it.e = e;
    it.mask = mask;
    it.counts8 = counts8;
    return it;
}

}  // namespace
}  // namespace t3d

using namespace t3d;

extern "C" size_t toric3d_run_batch_workspace_bytes(const t3d_run_cfg* cfg, const t3d_batch_item* items,
                                                    int n_items)
{
    if (validate_cfg(cfg) != T3D_OK || items == nullptr || n_items < 1 || n_items > kMaxItems) return 0;
    for (int i = 0; i < n_items; ++i)
        if (items[i].L < 2 || items[i].L > kMaxL || items[i].n_samples < 1) return 0;
    return batch_workspace_bytes(*cfg, items, n_items);
}

extern "C" t3d_status toric3d_run_batch(const t3d_run_cfg* cfg, const t3d_batch_item* items, int n_items,
                                        void* work, size_t work_bytes, t3d_stream stream)
{
    clear_error();
    return run_batch(cfg, items, n_items, work, work_bytes, stream);
}

extern "C" t3d_status toric3d_autotune_batch(const t3d_run_cfg* cfg, const t3d_batch_item* items,
                                             int n_items, void* work, size_t work_bytes,
                                             int* bp_blocks_per_sm, float* bp_ms, t3d_stream stream)
{
    clear_error();
    T3D_TRY(validate_cfg(cfg));
    T3D_TRY(validate_items(cfg, items, n_items));
    T3D_REQUIRE(cfg->use_bp && cfg->bp_iters > 0, "autotuning needs a BP decoder");
    T3D_REQUIRE(!meta_checks(*cfg), "autotuning covers the plain BP kernels only");
    Plan pl;
    T3D_TRY(plan_workspace(*cfg, items, n_items, work, work_bytes, pl));
    cudaStream_t st = as_stream(stream);
    ItemTable tab = pl.items;
    // a realistic noisy syndrome in the workspace (the states e are only read)
    T3D_TRY(launch_syndrome(tab, prob_threshold(cfg->q), cfg->seed, cfg->cycle0 + 1, st));
    int cap = 0;
    float ms = 0.0f;
    T3D_TRY(autotune_bp(pl.items, cfg->p, cfg->bp_meas_nodes ? cfg->q : 0.0, pl.bp, pl.chunk, st, &cap, &ms));
    if (bp_blocks_per_sm) *bp_blocks_per_sm = cap;
    if (bp_ms) *bp_ms = ms;
    return T3D_OK;
}

extern "C" size_t toric3d_run_workspace_bytes(const t3d_run_cfg* cfg)
{
    if (validate_cfg(cfg) != T3D_OK || cfg->L < 2 || cfg->L > kMaxL || cfg->n_samples < 1) return 0;
    t3d_batch_item it = single(cfg, nullptr, nullptr, nullptr);
    return batch_workspace_bytes(*cfg, &it, 1);
}

extern "C" t3d_status toric3d_run_cycles(const t3d_run_cfg* cfg, uint64_t* e, void* work,
                                         size_t work_bytes, uint8_t* mask, int64_t* counts8,
                                         t3d_stream stream)
{
    clear_error();
    T3D_REQUIRE(cfg != nullptr, "cfg is NULL");
    T3D_REQUIRE(cfg->cnn_blob == nullptr, "the learned decoder keeps s_prev state: use toric3d_run_batch");
    t3d_batch_item it = single(cfg, e, mask, counts8);
    return run_batch(cfg, &it, 1, work, work_bytes, stream);
}
