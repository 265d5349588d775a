// status.cuh -- the device status word of a translation unit.
//
// In the checked build (SPLAT_CHECKED) a kernel that finds an index out of its buffer's
// bounds skips the access, raises a bit of its unit's word and records the first site; a
// kernel whose bounded wait for its own tensor-core work runs out does the same.
// splat_sync_status reads and clears the words of every unit that includes this header.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace splat {

constexpr uint32_t kStatusTimeout = 1u;   // a bounded wait for the tensor core ran out
constexpr uint32_t kStatusBounds = 2u;    // checked build: an out-of-bounds index was skipped

// Checked-build sites of the units outside the rasterizer (which numbers its own from 1).
enum : uint32_t {
    kSiteScatter = 11,     // a radix pass's output position >= the key count
    kSiteEmit = 12,        // an emitted slot past the intersection capacity
    kSiteRayTile = 21,     // a free ray's tile >= the lidar's tiles
    kSiteRaySlot = 22,     // a binned ray's slot >= the ray count
};

struct StatusReader {
    void (*take)(uint32_t* bits, uint32_t* site);
    StatusReader* next;
};
void register_status_reader(StatusReader* r);    // api.cu
void take_all_status(uint32_t* bits, uint32_t* site);

namespace {
__device__ uint32_t g_status_bits;
__device__ uint32_t g_status_site;

__device__ __forceinline__ void raise_status(uint32_t bits, uint32_t site) {
    atomicOr(&g_status_bits, bits);
    atomicCAS(&g_status_site, 0u, site);
}

void take_unit_status(uint32_t* bits, uint32_t* site) {
    uint32_t b = 0, s = 0;
    if (cudaMemcpyFromSymbol(&b, g_status_bits, sizeof(b)) != cudaSuccess || !b) return;
    cudaMemcpyFromSymbol(&s, g_status_site, sizeof(s));
    const uint32_t z = 0;
    cudaMemcpyToSymbol(g_status_bits, &z, sizeof(z));
    cudaMemcpyToSymbol(g_status_site, &z, sizeof(z));
    *bits |= b;
    if (!*site) *site = s;
}

StatusReader g_unit_status_reader{take_unit_status, nullptr};
const bool g_unit_status_registered = (register_status_reader(&g_unit_status_reader), true);
}  // namespace

// Checked build: `if (SPLAT_OUT_OF_BOUNDS(i < n, site)) skip;` raises the bounds bit and takes
// the skip branch when the condition fails; in the normal build the test is compiled out.
#ifdef SPLAT_CHECKED
#define SPLAT_OUT_OF_BOUNDS(ok, site) \
    (!(ok) ? (::splat::raise_status(::splat::kStatusBounds, (site)), true) : false)
#else
#define SPLAT_OUT_OF_BOUNDS(ok, site) false
#endif

}  // namespace splat
