// lpsim_get_state_noalloc: the vehicle-state query without any allocation.
//
// lpsim_get_state gathers the slot state into vehicle-id order in device
// scratch that it allocates for the call (from cudaMalloc or the installed
// allocator callback).  Some callers cannot allocate at that point: a host
// whose allocator is pinned to a fixed pool that the simulation already
// filled, a caller inside code that must not change the device memory
// footprint (a memory-capped service sharing the GPU), or one that has no
// allocator callback to give.  This variant keeps its scratch in one
// file-scope device array of fixed size instead, so the call makes no
// cudaMalloc, cudaFree or allocator call; it only clears the array, runs the
// same scatter kernel and copies to the caller's host buffers.
#include <cstring>
#include <mutex>
#include <string>

#include <cuda.h>

#include "../../include/lpsim.h"
#include "ctx.h"
#include "lpsim_dev.cuh"

namespace {

// per vehicle: x, v (4 B each), edge, route index (4 B each), lane (1 B)
constexpr uint64_t kBytesPerVehicle = 17;
constexpr uint64_t kScratchBytes = (uint64_t)LPSIM_NOALLOC_MAX_VEHICLES * kBytesPerVehicle;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_state_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the scratch array's device address and the context it belongs to
struct ScratchAddr {
    void *ptr;
    unsigned long long ctx_id;
};
ScratchAddr g_scratch[kMaxDevices] = {};

int fail(int code, const std::string &m) { return lpsim_fail(code, m); }

// Unique id of the current context (driver entry points looked up through the
// runtime, so the library does not link the driver library).  0 if unknown.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(fn);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device.  Set up once
// per device and context: cudaGetSymbolAddress gives the address the kernels
// can use; a new context on the device (after cudaDeviceReset, say) holds the
// array at a new address, so a change of context id repeats the look-up.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(LPSIM_E_STATE, "device index out of range");
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev].ptr || id == 0 || g_scratch[dev].ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_state_scratch);
        if (e != cudaSuccess || !p)
            return fail(LPSIM_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch[dev] = ScratchAddr{p, id};
    }
    *out = g_scratch[dev].ptr;
    return LPSIM_OK;
}

}  // namespace

extern "C" int lpsim_get_state_noalloc(lpsim_ctx *c, uint64_t n, float *x, float *v, uint32_t *edge, uint8_t *lane,
                                       uint32_t *route_idx, uint8_t *status) {
    if (n > LPSIM_NOALLOC_MAX_VEHICLES)
        return fail(LPSIM_E_INVALID_ARG, "lpsim_get_state_noalloc: " + std::to_string(n) +
                                             " vehicles exceed the fixed scratch of " +
                                             std::to_string((unsigned long long)LPSIM_NOALLOC_MAX_VEHICLES) +
                                             " (use lpsim_get_state)");
    if (!c) return fail(LPSIM_E_INVALID_ARG, "ctx is NULL");
    if (!c->loaded) return fail(LPSIM_E_STATE, "lpsim_load_demand has not been called");
    if (n != c->n_trips) return fail(LPSIM_E_INVALID_ARG, "n does not match the trips loaded");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
        return fail(LPSIM_E_STATE, "the context's device must be current");
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc != LPSIM_OK) return rc;
    auto *tmp = static_cast<uint8_t *>(base);
    float *dx = reinterpret_cast<float *>(tmp);
    float *dv = dx + n;
    uint32_t *de = reinterpret_cast<uint32_t *>(dv + n);
    uint32_t *dr = de + n;
    uint8_t *dl = reinterpret_cast<uint8_t *>(dr + n);
    cudaStream_t st = c->stream;
    // the array keeps the previous call's contents: clear what must start empty
    cudaError_t e = cudaMemsetAsync(tmp, 0, n * kBytesPerVehicle, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(de, 0xFF, n * 4, st);
    if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("clear scratch: ") + cudaGetErrorString(e));
    lpsim::Dev d = c->d;
    d.s = c->sets[c->cur];
    lpsim::launch_state_scatter(d, c->k, dx, dv, de, dl, dr, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("state scatter: ") + cudaGetErrorString(e));
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } copies[] = {{x, dx, n * 4}, {v, dv, n * 4}, {edge, de, n * 4}, {route_idx, dr, n * 4}, {lane, dl, n},
                  {status, c->d.status, n}};
    for (auto &cp : copies) {
        if (!cp.dst) continue;
        e = cudaMemcpy(cp.dst, cp.src, cp.bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("copy to host: ") + cudaGetErrorString(e));
    }
    return LPSIM_OK;
}
