// noalloc.cu -- splat_bin_sort_noalloc: the binning sort for callers that cannot allocate
// device memory.
//
// Some callers of this library may not call cudaMalloc at all: a host simulator or game
// engine that owns a fixed device-memory budget handed out at start-up, a plug-in that
// runs inside someone else's frame loop where an allocation would synchronise the device
// and stall the frame, or a safety-reviewed runtime that forbids allocation after
// initialisation.  splat_bin_sort needs scratch memory besides its inputs and outputs;
// this entry point takes that scratch from a fixed array compiled into the library
// instead of from the caller, so it allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// its kStaticScratchBytes until the process exits.  Host code cannot use the array's name
// as a device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it together with the
// identity of the device's current CUDA context.  A call made after that context was
// torn down (cudaDeviceReset) sees a new context, in which the module and its array are
// loaded afresh, and looks the address up again.  A look-up cannot run inside a stream
// capture: make the first call on each device (and the first after a reset) before any
// capture; a call that needs a look-up while its stream is capturing is refused with
// SPLAT_ERR_INVALID_ARG.  All calls share the one array: two calls whose work overlaps on
// the GPU (different streams, or different threads on the same device without ordering)
// race on it.  Nothing in the scratch needs to start at zero -- every word the sort reads
// is written earlier in the same call -- so no clearing is done.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "types.cuh"

namespace splat {
splat_status record_error(splat_status code, const char* msg);
}

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_scratch[kStaticScratchBytes];

struct Slot {
    unsigned long long ctx_id;   // context the address belongs to (0: unknown)
    void* addr;
};

std::mutex g_mu;
Slot g_slot[kMaxDevices] = {};

using GetCurrentFn = CUresult (*)(CUcontext*);
using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Process-unique id of the calling thread's current context, 0 if there is none or the
// driver does not offer the query.  The driver entry points are fetched through the
// runtime, so the library does not link the driver library itself.  Called under g_mu.
unsigned long long current_context_id() {
    static bool tried = false;
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f);
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current device's current context (looked up
// once per context).
splat_status scratch_address(cudaStream_t stream, void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return splat::record_error(SPLAT_ERR_CUDA, "splat_bin_sort_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    Slot& sl = g_slot[dev];
    if (sl.addr && (id == 0 || id == sl.ctx_id)) {
        *out = sl.addr;
        return SPLAT_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return splat::record_error(SPLAT_ERR_INVALID_ARG,
                                   "splat_bin_sort_noalloc: the first call on a device (or after a device reset) "
                                   "looks up the scratch address and cannot run inside a stream capture");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess || !p)
        return splat::record_error(SPLAT_ERR_CUDA, "splat_bin_sort_noalloc: cudaGetSymbolAddress failed");
    sl.addr = p;
    sl.ctx_id = current_context_id();   // the look-up made the primary context current if it was not
    *out = p;
    return SPLAT_OK;
}

}  // namespace

extern "C" splat_status splat_bin_sort_noalloc(int64_t n, int32_t n_sensors, const splat_sensor* sensors,
                                               splat_projected proj, int64_t capacity, splat_bins bins,
                                               void* stream) {
    size_t need = 0;
    const splat_status st = splat_workspace_size(n, n_sensors, sensors, capacity, &need);
    if (st != SPLAT_OK) return st;
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "splat_bin_sort_noalloc: this frame needs %zu bytes of scratch but the built-in array holds %zu; "
                 "use splat_bin_sort with a caller workspace",
                 need, kStaticScratchBytes);
        return splat::record_error(SPLAT_ERR_INVALID_ARG, msg);
    }
    void* scratch = nullptr;
    const splat_status sa = scratch_address(static_cast<cudaStream_t>(stream), &scratch);
    if (sa != SPLAT_OK) return sa;
    return splat_bin_sort(n, n_sensors, sensors, proj, capacity, bins, scratch, kStaticScratchBytes, stream);
}
