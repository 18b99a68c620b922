// nbody_force_noalloc: the split force evaluation with its scratch in a
// fixed, file-scope device array instead of memory obtained at run time.
//
// Who needs it: callers that must not allocate device memory while they
// run.  Examples are a host application that owns every byte of the GPU
// through its own pool allocator and forbids third-party cudaMalloc; code
// that runs under a real-time or latency budget where an allocation (and the
// implicit device synchronisation of cudaFree) is unacceptable; and embedded
// or plugin deployments whose memory footprint must be fixed when the library
// is loaded.  Such callers keep the predicted j-stream, the active list and
// the outputs in their own device buffers and hand them over here.
//
// The scratch array lives in this library's module, so every GPU that loads
// the library holds it until the process exits; its size is fixed below.
// Every call shares it and it keeps the previous call's contents: the
// partial sums are fully rewritten before they are read, and the status word
// is cleared at the start of each call.  Calls that overlap on the GPU (from
// two streams or two host threads) race on the array and must be serialised
// by the caller.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "nbody_internal.cuh"

namespace nb {
namespace {

// 4 Mi floats (16 MiB): j-split partial sums, at least two j-ranges per call.
constexpr size_t kNoAllocPartialFloats = size_t(1) << 22;
// Largest active block: two ranges of 14 partial sums (compensated) fit.
constexpr int64_t kNoAllocMaxActive = int64_t(1) << 17;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_partials[kNoAllocPartialFloats];
static __device__ __align__(256) DevStatus g_noalloc_status;

// Device addresses of the two arrays, looked up once per device (host code
// only sees a host-side stand-in for a __device__ variable's name).  The
// look-up runs under g_setup_lock; `ready` is published with release order
// after the addresses are written, so a thread that reads it as true with
// acquire order also sees the addresses.
struct SymbolAddrs {
    std::atomic<bool> ready;
    float *partials;
    DevStatus *status;
};
SymbolAddrs g_addrs[kMaxDevices];
std::mutex g_setup_lock;

int fail(int code, const char *msg) { return report_error(code, msg); }

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return report_error(NBODY_ECUDA, buf);
}

bool aligned(const void *p, uintptr_t align) { return reinterpret_cast<uintptr_t>(p) % align == 0; }

// True when p is device memory of device `dev` (or managed memory).
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Looks up the scratch arrays' device addresses for `dev` (current) once.
int setup_device(int dev, SymbolAddrs &A)
{
    if (A.ready.load(std::memory_order_acquire)) return NBODY_OK;
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (A.ready.load(std::memory_order_relaxed)) return NBODY_OK;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&A.partials), g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(partials)");
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&A.status), g_noalloc_status);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
    A.ready.store(true, std::memory_order_release);
    return NBODY_OK;
}

}  // namespace
}  // namespace nb

using namespace nb;

extern "C" int nbody_force_noalloc(const float *posm, const float *vel, const float *poslo, int64_t n,
                                   const int32_t *active, int64_t n_act, double eps2, int mode, double *acc,
                                   double *jerk, double *pot, void *stream)
{
    report_error(NBODY_OK, "");
    if (n < 1 || n > 2147483647LL) return fail(NBODY_EINVAL, "nbody_force_noalloc: n out of range");
    if (n_act < 0 || n_act > n) return fail(NBODY_EINVAL, "nbody_force_noalloc: n_act outside [0, n]");
    if (n_act > kNoAllocMaxActive)
        return fail(NBODY_EINVAL, "nbody_force_noalloc: n_act exceeds the fixed scratch limit of 131072 "
                                  "active particles");
    if (mode != NBODY_MODE_PLAIN && mode != NBODY_MODE_COMP)
        return fail(NBODY_EINVAL, "nbody_force_noalloc: unknown mode");
    if (!(eps2 >= 0.0)) return fail(NBODY_EINVAL, "nbody_force_noalloc: eps2 must be >= 0");
    if (n_act == 0) return NBODY_OK;
    if (!posm || !vel || !active || !acc || !jerk || !pot || (mode == NBODY_MODE_COMP && !poslo))
        return fail(NBODY_EINVAL, "nbody_force_noalloc: null pointer argument");

    // The kernels copy j-tiles with bulk asynchronous copies (16-byte aligned
    // sources) and load float4, double and int32 values: a misaligned pointer
    // is rejected here, before any CUDA call, instead of faulting there.
    const void *jstream[] = {posm, vel, mode == NBODY_MODE_COMP ? poslo : posm};
    const void *outs[] = {acc, jerk, pot};
    for (const void *q : jstream)
        if (!aligned(q, 16)) return fail(NBODY_EINVAL, "nbody_force_noalloc: posm, vel and poslo must be 16-byte aligned");
    for (const void *q : outs)
        if (!aligned(q, 8)) return fail(NBODY_EINVAL, "nbody_force_noalloc: acc, jerk and pot must be 8-byte aligned");
    if (!aligned(active, 4)) return fail(NBODY_EINVAL, "nbody_force_noalloc: active must be 4-byte aligned");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(NBODY_EINVAL, "nbody_force_noalloc: device ordinal too large");
    const void *all[] = {posm, vel, mode == NBODY_MODE_COMP ? poslo : posm, acc, jerk, pot, active};
    for (const void *q : all)
        if (!on_device(q, dev))
            return fail(NBODY_EINVAL, "nbody_force_noalloc: every buffer must be device memory of the current device");
    SymbolAddrs &A = g_addrs[dev];
    const int rs = setup_device(dev, A);  // first call on this device (with it current)
    if (rs != NBODY_OK) return rs;
    int sm_count = 0;
    e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "SM count");

    const int64_t n_pad = (n + kJTile - 1) / kJTile * kJTile;
    const int64_t nc = mode == NBODY_MODE_COMP ? 14 : 7;
    ForceConfig cfg{};
    if (force_choose(mode, n_act, n_pad, sm_count, 0, 0, 0, &cfg, 1) != NBODY_OK)  // the caller's stream is float4 only
        return fail(NBODY_EINVAL, "nbody_force_noalloc: no launch shape");
    // Always at least two j-ranges (the scratch is used), at most what fits.
    const int64_t fit = static_cast<int64_t>(kNoAllocPartialFloats) / (nc * n_act);
    const int n_tiles = static_cast<int>(n_pad / kJTile);
    int split = cfg.split < 2 ? 2 : cfg.split;
    if (split > fit) split = static_cast<int>(fit);
    if (split > n_tiles) split = n_tiles;
    if (split >= 2) {
        const int tps = (n_tiles + split - 1) / split;
        cfg.tiles_per_split = tps;
        cfg.split = (n_tiles + tps - 1) / tps;
    } else {  // a single tile of j: nothing to split
        cfg.tiles_per_split = n_tiles;
        cfg.split = 1;
    }

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(A.status, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return cuda_fail(e, "status clear");
    JStream js;
    js.posm = reinterpret_cast<float4 *>(const_cast<float *>(posm));
    js.vel = reinterpret_cast<float4 *>(const_cast<float *>(vel));
    js.poslo = reinterpret_cast<float4 *>(const_cast<float *>(mode == NBODY_MODE_COMP ? poslo : posm));
    js.vello = nullptr;
    js.soa = nullptr;  // the caller's stream is AoS only
    js.n_pad = n_pad;
    int64_t launches = 0;
    e = force_launch(mode, js, n, active, n_act, eps2, cfg, acc, jerk, pot, A.partials,
                     A.status, s, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "force kernel launch");
    DevStatus st;
    e = cudaMemcpyAsync(&st, A.status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "status read-back");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    if (st.flags & kFlagTimeout) return fail(NBODY_ETIMEOUT, "nbody_force_noalloc: a bounded tile wait gave up");
    if (st.flags & kFlagBadIndex) return fail(NBODY_EINVAL, "nbody_force_noalloc: active index out of range");
    return NBODY_OK;
}
