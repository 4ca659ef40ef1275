// Library-wide host helpers: the per-thread error message behind
// toric3d_last_error() and the argument checks every entry point shares.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <mutex>
#include <vector>

#include "t3d_host.hpp"

namespace t3d {

namespace {
thread_local char g_error[512] = "";
}

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
}

void clear_error() { g_error[0] = '\0'; }

t3d_status check_lattice(int L)
{
    if (L < 2 || L > kMaxL) {
        set_error("L=%d outside [2, %d]", L, kMaxL);
        return T3D_EINVAL;
    }
    return T3D_OK;
}

t3d_status check_words(const void* p, const char* name)
{
    if (p == nullptr) {
        set_error("%s is NULL", name);
        return T3D_EINVAL;
    }
    if (!aligned(p, 8)) {
        set_error("%s must be 8-byte aligned", name);
        return T3D_EINVAL;
    }
    return T3D_OK;
}

// ------------------------------------------------------------ CUDA context ids
namespace {
// Driver calls reached through the runtime (the library does not link libcuda).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
std::mutex g_ctx_mutex;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

t3d_status resolve_driver_calls()
{
    if (g_ctx_get_current && g_ctx_get_id) return T3D_OK;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    T3D_CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
    T3D_CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
    T3D_REQUIRE(q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2,
                "the driver lacks cuCtxGetCurrent / cuCtxGetId");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    return T3D_OK;
}
}  // namespace

t3d_status current_context_id(unsigned long long* id)
{
    *id = 0;
    {
        std::lock_guard<std::mutex> lock(g_ctx_mutex);
        T3D_TRY(resolve_driver_calls());
    }
    CUcontext ctx = nullptr;
    T3D_REQUIRE(g_ctx_get_current(&ctx) == CUDA_SUCCESS, "cuCtxGetCurrent failed");
    if (ctx) T3D_REQUIRE(g_ctx_get_id(ctx, id) == CUDA_SUCCESS, "cuCtxGetId failed");
    return T3D_OK;
}

// ------------------------------------------------------------ persistent grids
namespace {

struct GridEntry {
    const void* kernel;
    int threads;
    int device;
    size_t smem;
    int blocks_per_sm;
};

struct SmemEntry {
    const void* kernel;
    unsigned long long ctx;
    size_t bytes;
};

std::mutex g_grid_mutex;
std::vector<GridEntry> g_grids;
std::vector<SmemEntry> g_smem;
int g_sms[64] = {0};
int g_tuned[T3D_K_COUNT] = {0};

}  // namespace

int tuned_blocks_per_sm(int kind)
{
    std::lock_guard<std::mutex> lock(g_grid_mutex);
    return (kind >= 0 && kind < T3D_K_COUNT) ? g_tuned[kind] : 0;
}

void set_tuned_blocks_per_sm(int kind, int blocks_per_sm)
{
    std::lock_guard<std::mutex> lock(g_grid_mutex);
    if (kind >= 0 && kind < T3D_K_COUNT) g_tuned[kind] = blocks_per_sm > 0 ? blocks_per_sm : 0;
}

// The attribute belongs to the current context: the cache is keyed by the context's id, so a
// new context (after a device reset) sets it again.
t3d_status allow_dynamic_smem(const void* kernel, size_t bytes)
{
    unsigned long long ctx = 0;
    T3D_TRY(current_context_id(&ctx));
    std::lock_guard<std::mutex> lock(g_grid_mutex);
    for (const auto& e : g_smem)
        if (e.kernel == kernel && e.ctx == ctx && ctx != 0 && e.bytes >= bytes) return T3D_OK;
    T3D_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (ctx != 0) g_smem.push_back(SmemEntry{kernel, ctx, bytes});
    return T3D_OK;
}

unsigned persistent_grid(const void* kernel, int threads, int kind, int64_t blocks, bool device_bound,
                         size_t dynamic_smem)
{
    const int64_t max_grid = 0x7fffffffLL;
    if (blocks < 1) return 1;
    int cap = tuned_blocks_per_sm(kind);
    // a launch whose work is bounded on the device (compacted words) walks only a few of its
    // blocks: resident blocks only, so the empty ones are not launched
    if (cap <= 0 && device_bound) cap = 1 << 20;
    if (cap <= 0) return (unsigned)std::min(blocks, max_grid);  // one block per work unit
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_grid_mutex);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_sms[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_sms[dev] = n;
    }
    int per_sm = 0;
    for (const auto& g : g_grids)
        if (g.kernel == kernel && g.threads == threads && g.device == dev && g.smem == dynamic_smem)
            per_sm = g.blocks_per_sm;
    if (per_sm == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, dynamic_smem) != cudaSuccess || n <= 0)
            n = 1;
        g_grids.push_back(GridEntry{kernel, threads, dev, dynamic_smem, n});
        per_sm = n;
    }
    per_sm = std::min(per_sm, cap);
    const int64_t grid = (int64_t)per_sm * g_sms[dev];
    return (unsigned)std::max<int64_t>(1, std::min(grid, blocks));
}

// ------------------------------------------------------------ kernel timing
namespace {

struct Record {
    int kind;
    cudaEvent_t start, stop;
};

std::mutex g_prof_mutex;
bool g_prof_on = false;
std::vector<Record> g_records;       // recorded pairs, in launch order
std::vector<cudaEvent_t> g_free;     // events ready for reuse

cudaEvent_t take_event()
{
    if (!g_free.empty()) {
        cudaEvent_t ev = g_free.back();
        g_free.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    return ev;
}

}  // namespace

int prof_begin(int kind, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (!g_prof_on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
    Record r{kind, take_event(), take_event()};
    if (!r.start || !r.stop) return -1;
    cudaEventRecord(r.start, st);
    g_records.push_back(r);
    return (int)g_records.size() - 1;
}

void prof_end(int handle, cudaStream_t st)
{
    if (handle < 0) return;
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (handle < (int)g_records.size()) cudaEventRecord(g_records[handle].stop, st);
}

}  // namespace t3d

extern "C" void toric3d_profile_enable(int on)
{
    std::lock_guard<std::mutex> lock(t3d::g_prof_mutex);
    t3d::g_prof_on = on != 0;
}

extern "C" void toric3d_profile_reset(void)
{
    std::lock_guard<std::mutex> lock(t3d::g_prof_mutex);
    for (auto& r : t3d::g_records) {
        cudaEventSynchronize(r.stop);
        t3d::g_free.push_back(r.start);
        t3d::g_free.push_back(r.stop);
    }
    t3d::g_records.clear();
}

extern "C" t3d_status toric3d_profile_read(int kind, double* total_ms, int64_t* launches)
{
    t3d::clear_error();
    if (kind < 0 || kind >= T3D_K_COUNT || !total_ms || !launches) {
        t3d::set_error("bad profile query");
        return T3D_EINVAL;
    }
    std::lock_guard<std::mutex> lock(t3d::g_prof_mutex);
    double sum = 0.0;
    int64_t n = 0;
    for (auto& r : t3d::g_records) {
        if (r.kind != kind) continue;
        cudaError_t err = cudaEventSynchronize(r.stop);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (err != cudaSuccess) {
            t3d::set_error("profile event: %s", cudaGetErrorString(err));
            return T3D_ECUDA;
        }
        sum += ms;
        ++n;
    }
    *total_ms = sum;
    *launches = n;
    return T3D_OK;
}

extern "C" void toric3d_set_blocks_per_sm(int kind, int blocks_per_sm)
{
    t3d::set_tuned_blocks_per_sm(kind, blocks_per_sm);
}

extern "C" int toric3d_get_blocks_per_sm(int kind) { return t3d::tuned_blocks_per_sm(kind); }

extern "C" const char* toric3d_last_error(void) { return t3d::g_error; }

extern "C" int toric3d_abi_version(void) { return 1; }
