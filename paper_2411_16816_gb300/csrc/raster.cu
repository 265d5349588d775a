// raster.cu -- channel-bucket dispatch of the rasterizer kernels (raster_impl.cuh).
#include "types.cuh"

namespace splat {

template <int CM, bool LIDAR>
bool dispatch_shape(int tw, int th, const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out,
                    const RasterGrad* g, bool recompute, cudaStream_t st);

template <int CM>
bool dispatch_list(const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out, const RasterGrad* g,
                   bool recompute, cudaStream_t st);

static int bucket(int C) { return C <= 4 ? 4 : C <= 8 ? 8 : C <= 16 ? 16 : C <= 32 ? 32 : 0; }

template <bool LIDAR>
static bool dispatch(int C, int tw, int th, const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out,
                     const RasterGrad* g, bool recompute, cudaStream_t st) {
    switch (bucket(C)) {
        case 4: return dispatch_shape<4, LIDAR>(tw, th, fr, blocks, in, out, g, recompute, st);
        case 8: return dispatch_shape<8, LIDAR>(tw, th, fr, blocks, in, out, g, recompute, st);
        case 16: return dispatch_shape<16, LIDAR>(tw, th, fr, blocks, in, out, g, recompute, st);
        case 32: return dispatch_shape<32, LIDAR>(tw, th, fr, blocks, in, out, g, recompute, st);
        default: return false;
    }
}

bool launch_raster_fwd(bool lidar, int C, int tw, int th, const Frame& fr, int blocks, const RasterIn& in,
                       const RasterOut& out, cudaStream_t st) {
    if (blocks <= 0) return true;
    return lidar ? dispatch<true>(C, tw, th, fr, blocks, in, &out, nullptr, false, st)
                 : dispatch<false>(C, tw, th, fr, blocks, in, &out, nullptr, false, st);
}

bool launch_raster_bwd(bool lidar, int C, int tw, int th, const Frame& fr, int blocks, const RasterIn& in,
                       const RasterGrad& g, bool recompute, cudaStream_t st) {
    if (blocks <= 0) return true;
    return lidar ? dispatch<true>(C, tw, th, fr, blocks, in, nullptr, &g, recompute, st)
                 : dispatch<false>(C, tw, th, fr, blocks, in, nullptr, &g, recompute, st);
}

static bool dispatch_list_c(int C, const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out,
                            const RasterGrad* g, bool recompute, cudaStream_t st) {
    switch (bucket(C)) {
        case 4: return dispatch_list<4>(fr, blocks, in, out, g, recompute, st);
        case 8: return dispatch_list<8>(fr, blocks, in, out, g, recompute, st);
        case 16: return dispatch_list<16>(fr, blocks, in, out, g, recompute, st);
        case 32: return dispatch_list<32>(fr, blocks, in, out, g, recompute, st);
        default: return false;
    }
}

bool launch_raster_list_fwd(int C, const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out,
                            cudaStream_t st) {
    if (blocks <= 0) return true;
    return dispatch_list_c(C, fr, blocks, in, &out, nullptr, false, st);
}

bool launch_raster_list_bwd(int C, const Frame& fr, int blocks, const RasterIn& in, const RasterGrad& g,
                            bool recompute, cudaStream_t st) {
    if (blocks <= 0) return true;
    return dispatch_list_c(C, fr, blocks, in, nullptr, &g, recompute, st);
}

bool raster_shape_supported(bool lidar, int tw, int th) {
    if (!lidar) return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8) || (tw == 16 && th == 32);
    return (tw == 32 && th == 8) || (tw == 16 && th == 8) || (tw == 32 && th == 16) || (tw == 64 && th == 8);
}

bool raster_channels_supported(int C) { return C >= 1 && C <= 32; }

}  // namespace splat
