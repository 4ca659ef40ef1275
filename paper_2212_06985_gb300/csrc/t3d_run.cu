// Whole Monte Carlo runs: T code cycles of noise, noisy measurement and
// decoding (Sec. 3.1 Fig. 2, Sec. 3.2 schedules, Sec. 4.2 p-BP), an optional
// noiseless final round, and the logical readout, enqueued on one stream and
// optionally captured into a CUDA graph that is instantiated once per distinct
// run and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "t3d_host.hpp"

namespace t3d {
namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t state_bytes(const t3d_run_cfg& c)
{
    return (size_t)3 * c.L * c.L * c.L * (size_t)words_for(c.n_samples) * sizeof(uint64_t);
}


struct Plan {
    uint64_t* s;
    uint64_t* tmp;
    float* bp;
    int64_t chunk_groups;
};

t3d_status validate(const t3d_run_cfg* c)
{
    T3D_REQUIRE(c != nullptr, "cfg is NULL");
    T3D_TRY(check_lattice(c->L));
    T3D_REQUIRE(c->T >= 0, "T must be >= 0");
    T3D_REQUIRE(c->p >= 0.0 && c->p <= 1.0 && c->q >= 0.0 && c->q <= 1.0, "p, q must lie in [0,1]");
    T3D_REQUIRE(c->n_samples >= 1 && words_for(c->n_samples) <= 65535LL * 32, "n_samples out of range");
    T3D_REQUIRE(c->sample0 % 64 == 0, "sample0 must be a multiple of 64");
    T3D_REQUIRE(c->n_apply >= 0, "n_apply must be >= 0");
    size_t slen = strnlen(c->schedule, sizeof(c->schedule));
    T3D_REQUIRE(slen < sizeof(c->schedule), "schedule must be NUL-terminated");
    T3D_REQUIRE(c->n_apply == 0 || slen >= 1, "n_apply > 0 needs a schedule");
    for (size_t i = 0; i < slen; ++i)
        T3D_REQUIRE(c->schedule[i] == 'F' || c->schedule[i] == 'P', "schedule may hold only 'F' and 'P'");
    if (c->use_bp) {
        T3D_REQUIRE(c->p > 0.0 && c->p < 1.0, "BP needs 0 < p < 1");
        T3D_REQUIRE(c->bp_iters >= 0, "bp_iters must be >= 0");
        T3D_REQUIRE(!c->bp_meas_nodes || c->q < 0.5, "measurement nodes need q < 0.5");
        T3D_REQUIRE(c->bp_chunk_samples >= 0, "bp_chunk_samples must be >= 0");
    }
    T3D_REQUIRE(!c->perfect_round || c->perfect_max_sweeps >= 0, "perfect_max_sweeps must be >= 0");
    return T3D_OK;
}

t3d_status plan_workspace(const t3d_run_cfg& c, void* work, size_t work_bytes, Plan& pl)
{
    const size_t sb = round_up(state_bytes(c));
    T3D_REQUIRE(work != nullptr && aligned(work, kAlign), "work must be a 256-byte aligned device pointer");
    T3D_REQUIRE(work_bytes >= 2 * sb, "workspace too small: %zu < %zu", work_bytes, 2 * sb);
    char* base = static_cast<char*>(work);
    pl.s = reinterpret_cast<uint64_t*>(base);
    pl.tmp = reinterpret_cast<uint64_t*>(base + sb);
    pl.bp = nullptr;
    pl.chunk_groups = 0;
    if (c.use_bp && c.bp_iters > 0) {
        const int64_t G = groups_for(c.n_samples);
        int64_t chunk = (int64_t)((work_bytes - 2 * sb) / bp_bytes_per_group(c.L));
        if (c.bp_chunk_samples > 0) chunk = std::min(chunk, groups_for(c.bp_chunk_samples));
        if (chunk < G) chunk &= ~1LL;
        T3D_REQUIRE(chunk >= 1, "workspace too small for one BP chunk");
        pl.chunk_groups = std::min(chunk, G);
        pl.bp = reinterpret_cast<float*>(base + 2 * sb);
    }
    return T3D_OK;
}

t3d_status enqueue_run(const t3d_run_cfg& c, uint64_t* e, const Plan& pl, uint8_t* mask,
                       int64_t* counts8, cudaStream_t st)
{
    const int L = c.L;
    const int64_t W = words_for(c.n_samples);
    const uint64_t group0 = c.sample0 / 64;
    const uint64_t thr_p = prob_threshold(c.p), thr_q = prob_threshold(c.q);
    const int slen = (int)strnlen(c.schedule, sizeof(c.schedule));
    for (int t = 1; t <= c.T; ++t) {
        const uint32_t cycle = c.cycle0 + (uint32_t)t;
        T3D_TRY(launch_noise(L, W, e, thr_p, c.seed, group0, cycle, st));
        T3D_TRY(launch_syndrome(L, W, e, pl.s, thr_q, c.seed, group0, cycle, st));
        if (c.use_bp)
            T3D_TRY(launch_bp(L, c.n_samples, e, pl.s, c.p, c.bp_meas_nodes ? c.q : 0.0, c.bp_iters,
                              pl.bp, pl.chunk_groups, nullptr, st));
        if (c.n_apply > 0)
            T3D_TRY(launch_sweeps(L, W, e, pl.s, pl.tmp, c.schedule, slen, c.n_apply, 0, c.seed,
                                  group0, cycle, st));
    }
    if (c.perfect_round) {
        const uint32_t cycle = c.cycle0 + (uint32_t)c.T + 1;
        T3D_TRY(launch_syndrome(L, W, e, pl.s, 0, c.seed, group0, cycle, st));
        if (c.perfect_max_sweeps > 0)
            T3D_TRY(launch_sweeps(L, W, e, pl.s, pl.tmp, "F", 1, c.perfect_max_sweeps, 0, c.seed,
                                  group0, cycle, st));
    }
    if (mask || counts8) T3D_TRY(launch_logical(L, c.n_samples, e, mask, counts8, st));
    return T3D_OK;
}

// ------------------------------------------------------------ graph cache
struct GraphKey {
    t3d_run_cfg cfg;
    const void* e;
    const void* work;
    size_t work_bytes;
    const void* mask;
    const void* counts8;
    cudaStream_t stream;
    int device;
};

bool same_key(const GraphKey& a, const GraphKey& b) { return std::memcmp(&a, &b, sizeof(GraphKey)) == 0; }

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    bool used;
};

constexpr int kGraphCache = 8;
GraphEntry g_graphs[kGraphCache];
int g_graph_next = 0;
std::mutex g_graph_mutex;

t3d_status run_with_graph(const t3d_run_cfg& c, uint64_t* e, const Plan& pl, void* work,
                          size_t work_bytes, uint8_t* mask, int64_t* counts8, cudaStream_t st)
{
    T3D_REQUIRE(st != nullptr, "use_graph needs a non-default stream");
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.cfg = c;
    key.e = e;
    key.work = work;
    key.work_bytes = work_bytes;
    key.mask = mask;
    key.counts8 = counts8;
    key.stream = st;
    T3D_CUDA_CHECK(cudaGetDevice(&key.device));
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    for (auto& g : g_graphs) {
        if (g.used && same_key(g.key, key)) {
            T3D_CUDA_CHECK(cudaGraphLaunch(g.exec, st));
            return T3D_OK;
        }
    }
    T3D_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    t3d_status stq = enqueue_run(c, e, pl, mask, counts8, st);
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
    g_graph_next = (g_graph_next + 1) % kGraphCache;
    if (slot.used) {
        // the evicted graph may still be running on its stream: wait before freeing it
        cudaStreamSynchronize(slot.key.stream);
        cudaGraphExecDestroy(slot.exec);
    }
    slot.key = key;
    slot.exec = exec;
    slot.used = true;
    T3D_CUDA_CHECK(cudaGraphLaunch(exec, st));
    return T3D_OK;
}

}  // namespace
}  // namespace t3d

using namespace t3d;

extern "C" size_t toric3d_run_workspace_bytes(const t3d_run_cfg* cfg)
{
    if (validate(cfg) != T3D_OK) return 0;
    size_t total = 2 * round_up(state_bytes(*cfg));
    if (cfg->use_bp && cfg->bp_iters > 0) {
        int64_t n = cfg->bp_chunk_samples > 0 ? std::min(cfg->bp_chunk_samples, cfg->n_samples)
                                              : cfg->n_samples;
        int64_t g = groups_for(n);
        if (g < groups_for(cfg->n_samples)) g += g & 1;
        total += (size_t)g * bp_bytes_per_group(cfg->L);
    }
    return total;
}

extern "C" t3d_status toric3d_run_cycles(const t3d_run_cfg* cfg, uint64_t* e, void* work,
                                         size_t work_bytes, uint8_t* mask, int64_t* counts8,
                                         t3d_stream stream)
{
    clear_error();
    T3D_TRY(validate(cfg));
    T3D_TRY(check_words(e, "e"));
    T3D_REQUIRE(counts8 == nullptr || aligned(counts8, 8), "counts8 must be 8-byte aligned");
    Plan pl;
    T3D_TRY(plan_workspace(*cfg, work, work_bytes, pl));
    cudaStream_t st = as_stream(stream);
    if (cfg->use_graph) return run_with_graph(*cfg, e, pl, work, work_bytes, mask, counts8, st);
    return enqueue_run(*cfg, e, pl, mask, counts8, st);
}
