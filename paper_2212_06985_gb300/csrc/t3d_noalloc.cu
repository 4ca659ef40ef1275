// toric3d_flip_noalloc: the parallel flip decoder without a caller-provided
// workspace.
//
// toric3d_flip needs one bit-sliced syndrome array of scratch for its
// synchronous applications (every qubit must decide from the same syndrome
// snapshot, so each application writes a second copy).  Some callers cannot
// hand the library fresh device memory: a decoder embedded in a control loop
// whose device memory is fixed when it starts, a plugin whose host
// application owns every device allocation through its own allocator, or a
// latency-critical caller that cannot afford the device-wide synchronisation
// cudaMalloc and cudaFree may cause.  For them this entry point keeps its
// scratch in a file-scope device array of fixed size, so a call allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// Costs and rules of the built-in scratch:
// * every GPU that loads this library holds the array (kScratchBytes) until
//   the process exits;
// * the array's device address is looked up on a device's first call (with
//   the device current) and again whenever the device's CUDA context has
//   changed since (after cudaDeviceReset the module is loaded anew and the
//   array moves); make those calls outside any stream capture;
// * all calls share the one array, so calls whose work overlaps on the GPU
//   (for example on two streams without ordering) race and corrupt each
//   other's results; order them;
// * the array keeps the last call's contents; nothing in it needs to start at
//   zero, because every application overwrites the whole syndrome copy
//   before reading it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "t3d_host.hpp"
#include "t3d_items.cuh"

namespace t3d {
namespace {

// 32 MiB: e.g. L = 16 with up to 341 words (21,824 samples), or L = 32 with
// up to 42 words (2,688 samples).
constexpr size_t kScratchBytes = 32u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint64_t g_flip_scratch[kScratchBytes / sizeof(uint64_t)];

std::mutex g_scratch_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;   // unique id of the CUDA context the address belongs to
    void* addr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array in the current device's current context:
// looked up on the first call and again whenever that context has changed.
t3d_status scratch_address(void** out)
{
    int dev = 0;
    T3D_CUDA_CHECK(cudaGetDevice(&dev));
    T3D_REQUIRE(dev >= 0 && dev < kMaxDevices, "device %d outside the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    T3D_TRY(current_context_id(&id));
    ScratchAddr& c = g_scratch_addr[dev];
    if (id == 0 || c.addr == nullptr || c.ctx_id != id) {
        void* p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_flip_scratch);   // creates the context if needed
        if (err != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress of the flip scratch failed: %s", cudaGetErrorString(err));
            return T3D_ECUDA;
        }
        T3D_TRY(current_context_id(&id));
        T3D_REQUIRE(id != 0, "no current CUDA context after the symbol lookup");
        c.ctx_id = id;
        c.addr = p;
    }
    *out = c.addr;
    return T3D_OK;
}

}  // namespace
}  // namespace t3d

using namespace t3d;

extern "C" t3d_status toric3d_flip_noalloc(int L, int64_t words, uint64_t* e, uint64_t* s, int sweeps,
                                           t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(words >= 1 && words <= 65535LL * 32, "words=%lld out of range", (long long)words);
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(sweeps >= 0, "negative number of sweeps");
    const size_t need = (size_t)3 * L * L * L * (size_t)words * sizeof(uint64_t);
    T3D_REQUIRE(need <= kScratchBytes,
                "L=%d with %lld words needs %zu bytes of scratch but the built-in scratch holds %zu; "
                "use toric3d_flip with a workspace",
                L, (long long)words, need, kScratchBytes);
    if (sweeps == 0) return T3D_OK;
    void* scratch = nullptr;
    T3D_TRY(scratch_address(&scratch));
    ItemTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = 1;
    ItemDesc& d = tab.it[0];
    d.lat = make_lattice_host(L);
    d.W = words;
    d.n_samples = words * 64;
    d.e = e;
    d.s = s;
    d.tmp = static_cast<uint64_t*>(scratch);
    return launch_sweeps(tab, "F", 1, sweeps, 0, 0, 0, as_stream(stream));
}
