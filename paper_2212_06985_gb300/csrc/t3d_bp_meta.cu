// BP with meta-checks (Sec. 4.1, last paragraph: the paper describes them
// and leaves them out of its simulations).  Every error-free syndrome of the
// 3D toric code is a union of closed loops, so the six faces of every unit
// cube have even parity; a cube whose measured faces have odd parity holds an
// odd number of measurement errors.  The factor graph gets one
// measurement-error variable per face (prior log((1-q)/q), degree 3: its
// face and the face's two cubes) and one meta-check per cube over the
// measurement variables of its six faces, with the measured cube parity as
// its syndrome.  Flooding schedule as in Eqs. 1-4: every iteration computes
// all check -> variable messages from the previous iteration's.
//
// Messages are FP32, sample-innermost ([index][sample], samples of a chunk
// padded to whole 64-sample words), double-buffered, 7 planes of 3L^3 rows:
//   F [face][4]   face -> its four edges (the a-edges at r and r + e_b, then
//                 the b-edges at r and r + e_a; a < b the in-plane axes)
//   Fm[face]      face -> its measurement variable
//   Cl[face]      cube at the face's site (the face is its lower face) -> the face's variable
//   Ch[face]      cube one step down along the face's normal (upper face) -> the variable
// One iteration is three kernels: the total of every edge (prior + its four
// face messages), the faces (inputs: edge total minus the face's own message,
// and the measurement variable's prior + both cube messages), the cubes
// (inputs: prior + face message + the other cube's message).  Check nodes use
// the plain BP's cancellation-free (t, d = 1 - t) arithmetic (t3d_bp_math.cuh),
// so magnitudes keep FP32 accuracy up to the +-30 clamp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "t3d_bp_math.cuh"
#include "t3d_device.cuh"
#include "t3d_host.hpp"

namespace t3d {
namespace meta {
namespace {

using bpm::add4;
using bpm::check_node;
using bpm::comp;
using bpm::ld4;
using bpm::st4;
using bpm::sub4;

constexpr int kThreads = 256;   // threads per block, each on consecutive samples of one index

struct Bufs {
    float* F;     // [3L^3][4][S]
    float* Fm;    // [3L^3][S]
    float* Cl;    // [3L^3][S]
    float* Ch;    // [3L^3][S]
};

struct Args {
    Lattice lat;
    int64_t S;              // padded samples of this chunk (multiple of 64)
    int64_t W;              // row stride of the bit-sliced arrays (words)
    const uint64_t* s;      // measured syndrome, chunk's first word at column 0
    float l0, lq;
    const float* T;         // edge totals [3L^3][S]
    Bufs in, out;
};


// Syndrome bits of samples smp .. smp + 3 (smp a multiple of 4) in bits 0..3.
__device__ __forceinline__ uint32_t syn_bits4(const Args& a, int64_t row, int64_t smp)
{
    return (uint32_t)(a.s[row * a.W + (smp >> 6)] >> (smp & 63)) & 0xFu;
}

__device__ __forceinline__ int64_t step_site(const Lattice& lat, const Coord& c, int ax, int delta)
{
    return site_index(lat, shifted(lat, c, ax, delta));
}

// The four (face, slot) pairs of edge (d, r): for each normal n != d with third axis
// c, the faces (n, r) and (n, r - e_c); the edge is slot 0 / 1 of them if d < c, else 2 / 3.
__device__ __forceinline__ void edge_slots(const Lattice& lat, int d, int r, int64_t (&f)[4], int (&slot)[4])
{
    const Coord c = site_coord(lat, r);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int n = i == 0 ? (d == 0 ? 1 : 0) : (d == 2 ? 1 : 2);   // the two normals n != d
        const int ax = 3 - d - n;
        const int lo = d < ax ? 0 : 2;
        f[2 * i] = (int64_t)n * lat.L3 + r;
        slot[2 * i] = lo;
        f[2 * i + 1] = (int64_t)n * lat.L3 + step_site(lat, c, ax, -1);
        slot[2 * i + 1] = lo + 1;
    }
}

// The iteration kernels give each thread four consecutive samples of one index:
// blockIdx.x is the index, blockIdx.y * blockDim.x + threadIdx.x the sample quad.
__device__ __forceinline__ int64_t quad_sample(const Args& a)
{
    return ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * 4;
}

__global__ void __launch_bounds__(kThreads) k_edge_totals(const Args a, float* __restrict__ T)
{
    const int64_t smp = quad_sample(a);
    const int64_t v = blockIdx.x;
    if (smp >= a.S) return;
    const int d = (int)(v / a.lat.L3), r = (int)(v % a.lat.L3);
    int64_t f[4];
    int slot[4];
    edge_slots(a.lat, d, r, f, slot);
    float4 t = make_float4(a.l0, a.l0, a.l0, a.l0);
#pragma unroll
    for (int k = 0; k < 4; ++k) t = add4(t, ld4(a.in.F, f[k] * 4 + slot[k], a.S, smp));
    st4(T, v, a.S, smp, t);
}

__global__ void __launch_bounds__(kThreads) k_faces(const Args a)
{
    const int64_t smp = quad_sample(a);
    const int64_t fc = blockIdx.x;
    if (smp >= a.S) return;
    const int n = (int)(fc / a.lat.L3), r = (int)(fc % a.lat.L3);
    const Coord c = site_coord(a.lat, r);
    const int ax = n == 0 ? 1 : 0, bx = n == 2 ? 1 : 2;   // in-plane axes a < b
    const int64_t L3 = a.lat.L3;
    const int64_t ed[4] = {ax * L3 + r, ax * L3 + step_site(a.lat, c, bx, 1), bx * L3 + r,
                           bx * L3 + step_site(a.lat, c, ax, 1)};
    float4 x4[5];
#pragma unroll
    for (int j = 0; j < 4; ++j) x4[j] = sub4(ld4(a.T, ed[j], a.S, smp), ld4(a.in.F, fc * 4 + j, a.S, smp));
    const float4 lq = make_float4(a.lq, a.lq, a.lq, a.lq);
    x4[4] = add4(add4(lq, ld4(a.in.Cl, fc, a.S, smp)), ld4(a.in.Ch, fc, a.S, smp));
    const uint32_t syn = syn_bits4(a, fc, smp);
    float o4[5][4];
#pragma unroll
    for (int cpt = 0; cpt < 4; ++cpt) {
        float x[5], o[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = comp(x4[j], cpt);
        check_node<5>(x, (syn >> cpt) & 1u, o);
#pragma unroll
        for (int j = 0; j < 5; ++j) o4[j][cpt] = o[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) st4(a.out.F, fc * 4 + j, a.S, smp, make_float4(o4[j][0], o4[j][1], o4[j][2], o4[j][3]));
    st4(a.out.Fm, fc, a.S, smp, make_float4(o4[4][0], o4[4][1], o4[4][2], o4[4][3]));
}

__global__ void __launch_bounds__(kThreads) k_cubes(const Args a)
{
    const int64_t smp = quad_sample(a);
    const int r = blockIdx.x;
    if (smp >= a.S) return;
    const Coord c = site_coord(a.lat, r);
    const int64_t L3 = a.lat.L3;
    int64_t fl[3], fu[3];   // lower faces (n, r), upper faces (n, r + e_n)
    uint32_t par = 0;
    float4 x4[6];
    const float4 lq = make_float4(a.lq, a.lq, a.lq, a.lq);
#pragma unroll
    for (int nn = 0; nn < 3; ++nn) {
        fl[nn] = nn * L3 + r;
        fu[nn] = nn * L3 + step_site(a.lat, c, nn, 1);
        par ^= syn_bits4(a, fl[nn], smp) ^ syn_bits4(a, fu[nn], smp);
        // this cube is the lower-face cube of fl (its message is Cl) and the upper-face cube of fu (Ch)
        x4[2 * nn] = add4(add4(lq, ld4(a.in.Fm, fl[nn], a.S, smp)), ld4(a.in.Ch, fl[nn], a.S, smp));
        x4[2 * nn + 1] = add4(add4(lq, ld4(a.in.Fm, fu[nn], a.S, smp)), ld4(a.in.Cl, fu[nn], a.S, smp));
    }
    float o4[6][4];
#pragma unroll
    for (int cpt = 0; cpt < 4; ++cpt) {
        float x[6], o[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) x[j] = comp(x4[j], cpt);
        check_node<6>(x, (par >> cpt) & 1u, o);
#pragma unroll
        for (int j = 0; j < 6; ++j) o4[j][cpt] = o[j];
    }
#pragma unroll
    for (int nn = 0; nn < 3; ++nn) {
        st4(a.out.Cl, fl[nn], a.S, smp, make_float4(o4[2 * nn][0], o4[2 * nn][1], o4[2 * nn][2], o4[2 * nn][3]));
        st4(a.out.Ch, fu[nn], a.S, smp,
            make_float4(o4[2 * nn + 1][0], o4[2 * nn + 1][1], o4[2 * nn + 1][2], o4[2 * nn + 1][3]));
    }
}

// Posteriors and decisions: qubit v: l = T_v; decision words (one ballot per 32
// samples) into dec[word][site][4] as 32-bit halves; optional posteriors.
__global__ void __launch_bounds__(kThreads) k_decide(const Args a, int64_t n_samples, uint32_t* __restrict__ dec32,
                                                      float* __restrict__ llr, int64_t llr_stride)
{
    const int64_t smp = (int64_t)blockIdx.y * kThreads + threadIdx.x;
    const int64_t v = blockIdx.x;
    const int64_t L3 = a.lat.L3, n = 3 * L3;
    if (smp >= a.S) return;   // S is a multiple of 64: whole warps
    const float l = a.T[v * a.S + smp];
    const bool valid = smp < n_samples;
    const uint32_t bits = __ballot_sync(0xffffffffu, valid && l < 0.0f);
    const int d = (int)(v / L3), r = (int)(v % L3);
    if ((threadIdx.x & 31) == 0) dec32[((smp >> 6) * L3 + r) * 8 + 2 * d + ((smp >> 5) & 1)] = bits;
    if (llr && valid) {
        llr[v * llr_stride + smp] = l;
        const float m = a.lq + a.in.Fm[v * a.S + smp] + a.in.Cl[v * a.S + smp] + a.in.Ch[v * a.S + smp];
        llr[(n + v) * llr_stride + smp] = m;
    }
}

// Messages of one iteration in a contiguous buffer of 7 planes of 3 L^3 x S floats.
Bufs split_messages(float* m, int64_t n, int64_t S)
{
    return Bufs{m, m + 4 * n * S, m + 5 * n * S, m + 6 * n * S};
}

// Quad-kernel block: S / 4 sample quads, at most kThreads a block, whole warps.
unsigned quad_threads(int64_t S) { return (unsigned)std::min<int64_t>(kThreads, (S / 4 + 31) / 32 * 32); }

unsigned quad_blocks(int64_t S) { return (unsigned)((S / 4 + quad_threads(S) - 1) / quad_threads(S)); }

// One flooding iteration: every check -> variable message of `out` from those of `in`.
t3d_status launch_iteration(Args& a, float* T, const Bufs& in, const Bufs& out, cudaStream_t st)
{
    const int64_t n = 3LL * a.lat.L3;
    const unsigned tx = quad_threads(a.S), gy = quad_blocks(a.S);
    a.in = in;
    a.out = out;
    ProfScope prof(T3D_K_BP_STEP, st);
    k_edge_totals<<<dim3((unsigned)n, gy), tx, 0, st>>>(a, T);
    T3D_LAUNCH_CHECK("meta-check BP edge totals");
    k_faces<<<dim3((unsigned)n, gy), tx, 0, st>>>(a);
    T3D_LAUNCH_CHECK("meta-check BP faces");
    k_cubes<<<dim3((unsigned)a.lat.L3, gy), tx, 0, st>>>(a);
    T3D_LAUNCH_CHECK("meta-check BP cubes");
    return T3D_OK;
}

Args make_args(const Lattice& lat, int64_t S, int64_t W, const uint64_t* s, double p, double q, float* T)
{
    Args a;
    std::memset(&a, 0, sizeof(a));
    a.lat = lat;
    a.S = S;
    a.W = W;
    a.s = s;
    a.l0 = (float)std::log((1.0 - p) / p);
    a.lq = (float)std::log((1.0 - q) / q);
    a.T = T;
    return a;
}

size_t floats_per_sample(int L)
{
    const size_t n = 3ull * L * L * L;
    return n /* T */ + 2 * 7 * n /* F, Fm, Cl, Ch x2 */;
}

}  // namespace

size_t bytes_per_word(int L)
{
    return 64 * floats_per_sample(L) * sizeof(float) + (size_t)L * L * L * 32 /* decision words */ + 4096;
}

// BP with meta-checks on n_samples samples (rows of stride W words), in chunks of
// whole words as large as the workspace allows; e ^= d, s ^= H d.
t3d_status launch_bp_meta(const Lattice& lat, int64_t n_samples, int64_t W, uint64_t* e, uint64_t* s, double p,
                          double q, int iters, void* work, size_t work_bytes, float* llr_out, cudaStream_t st)
{
    const int64_t words = words_for(n_samples);
    // at most 65535 sample blocks of kThreads per launch (grid y)
    const int64_t chunk = std::min<int64_t>({words, (int64_t)(work_bytes / bytes_per_word(lat.L)),
                                             65535LL * kThreads / 64});
    T3D_REQUIRE(chunk >= 1, "workspace too small: %zu bytes < %zu per 64-sample word", work_bytes,
                bytes_per_word(lat.L));
    T3D_REQUIRE(llr_out == nullptr || chunk == words, "llr_out needs a workspace for all samples at once");
    const int64_t n = 3LL * lat.L3;
    for (int64_t w0 = 0; w0 < words; w0 += chunk) {
        const int64_t cw = std::min(chunk, words - w0);
        const int64_t S = cw * 64, ns = std::min<int64_t>(S, n_samples - w0 * 64);
        char* base = static_cast<char*>(work);
        auto take = [&](size_t floats) {
            float* ptr = reinterpret_cast<float*>(base);
            base += (floats * sizeof(float) + 255) / 256 * 256;
            return ptr;
        };
        float* T = take(n * S);
        const Bufs b[2] = {split_messages(take(7 * n * S), n, S), split_messages(take(7 * n * S), n, S)};
        uint64_t* dec = reinterpret_cast<uint64_t*>(base);
        // every message starts at zero: the first iteration sees the priors alone
        T3D_CUDA_CHECK(cudaMemsetAsync(b[0].F, 0, 7 * n * S * sizeof(float), st));
        Args a = make_args(lat, S, W, s + w0, p, q, T);
        for (int it = 0; it < iters; ++it) T3D_TRY(launch_iteration(a, T, b[it & 1], b[(it + 1) & 1], st));
        a.in = b[iters & 1];
        ProfScope prof(T3D_K_BP_DECIDE, st);
        k_edge_totals<<<dim3((unsigned)n, quad_blocks(S)), quad_threads(S), 0, st>>>(a, T);
        T3D_LAUNCH_CHECK("meta-check BP posteriors");
        k_decide<<<dim3((unsigned)n, (unsigned)((S + kThreads - 1) / kThreads)), kThreads, 0, st>>>(a, ns, reinterpret_cast<uint32_t*>(dec), llr_out,
                                                             n_samples);
        T3D_LAUNCH_CHECK("meta-check BP decisions");
        T3D_TRY(launch_dec_apply(lat, W, cw, dec, e + w0, s + w0, st));
    }
    return T3D_OK;
}

}  // namespace meta
}  // namespace t3d

using namespace t3d;

extern "C" size_t toric3d_bp_meta_workspace_bytes(int L, int64_t chunk_samples)
{
    if (L < 2 || L > 1024 || chunk_samples < 1) return 0;
    return (size_t)words_for(chunk_samples) * meta::bytes_per_word(L);
}

extern "C" size_t toric3d_bp_meta_message_bytes(int L, int64_t n_samples)
{
    if (L < 2 || L > 1024 || n_samples < 1) return 0;
    return (size_t)7 * 3 * L * L * L * 64 * (size_t)words_for(n_samples) * sizeof(float);
}

extern "C" t3d_status toric3d_bp_meta_step(int L, int64_t n_samples, const uint64_t* s, double p, double q,
                                           const float* msg_in, float* msg_out, void* work, size_t work_bytes,
                                           t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(n_samples >= 1 && words_for(n_samples) <= 65535LL * meta::kThreads / 64, "n_samples out of range");
    T3D_TRY(check_words(s, "s"));
    T3D_REQUIRE(p > 0.0 && p < 1.0, "BP needs 0 < p < 1");
    T3D_REQUIRE(q > 0.0 && q < 1.0, "meta-checks need measurement errors: 0 < q < 1");
    T3D_REQUIRE(msg_in != nullptr && msg_out != nullptr && aligned(msg_in, 16) && aligned(msg_out, 16),
                "msg_in and msg_out must be 16-byte aligned device pointers");
    const size_t mb = toric3d_bp_meta_message_bytes(L, n_samples);
    const char *ib = reinterpret_cast<const char*>(msg_in), *ob = reinterpret_cast<const char*>(msg_out);
    T3D_REQUIRE(ib + mb <= ob || ob + mb <= ib, "msg_in and msg_out must not overlap");
    T3D_REQUIRE(work != nullptr && aligned(work, 16) && work_bytes >= mb / 7, "work: >= %zu bytes, 16-byte aligned",
                mb / 7);
    const Lattice lat = make_lattice_host(L);
    const int64_t n = 3LL * lat.L3, S = 64 * words_for(n_samples);
    float* T = static_cast<float*>(work);
    meta::Args a = meta::make_args(lat, S, words_for(n_samples), s, p, q, T);
    return meta::launch_iteration(a, T, meta::split_messages(const_cast<float*>(msg_in), n, S),
                                  meta::split_messages(msg_out, n, S), as_stream(stream));
}

extern "C" t3d_status toric3d_bp_meta(int L, int64_t n_samples, uint64_t* e, uint64_t* s, double p, double q,
                                      int iters, void* work, size_t work_bytes, float* llr_out, t3d_stream stream)
{
    clear_error();
    T3D_TRY(check_lattice(L));
    T3D_REQUIRE(n_samples >= 1 && words_for(n_samples) <= 65535LL * 32, "n_samples out of range");
    T3D_TRY(check_words(e, "e"));
    T3D_TRY(check_words(s, "s"));
    const size_t state = (size_t)3 * L * L * L * (size_t)words_for(n_samples) * 8;
    T3D_REQUIRE(disjoint(e, state, s, state), "e and s must not overlap");
    T3D_REQUIRE(p > 0.0 && p < 1.0, "BP needs 0 < p < 1");
    T3D_REQUIRE(q > 0.0 && q < 1.0, "meta-checks need measurement errors: 0 < q < 1");
    T3D_REQUIRE(iters >= 0, "negative iteration count");
    T3D_REQUIRE(work != nullptr && aligned(work, 256), "work must be a 256-byte aligned device pointer");
    T3D_REQUIRE(llr_out == nullptr || aligned(llr_out, 4), "llr_out must be 4-byte aligned");
    return meta::launch_bp_meta(make_lattice_host(L), n_samples, words_for(n_samples), e, s, p, q, iters, work,
                                work_bytes, llr_out, as_stream(stream));
}
