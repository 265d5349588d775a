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
// cudaGetSymbolAddress (with that device current) and caches it; make that first call
// before any stream capture.  All calls share the one array: two calls whose work
// overlaps on the GPU (different streams, or different threads on the same device
// without ordering) race on it.  Nothing in the scratch needs to start at zero -- every
// word the sort reads is written earlier in the same call -- so no clearing is done.
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

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
splat_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return splat::record_error(SPLAT_ERR_CUDA, "splat_bin_sort_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || !p)
            return splat::record_error(SPLAT_ERR_CUDA, "splat_bin_sort_noalloc: cudaGetSymbolAddress failed");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
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
    const splat_status sa = scratch_address(&scratch);
    if (sa != SPLAT_OK) return sa;
    return splat_bin_sort(n, n_sensors, sensors, proj, capacity, bins, scratch, kStaticScratchBytes, stream);
}
