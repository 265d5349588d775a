// raster_c8.cu -- rasterizer kernels for up to 8 channels (one translation unit per
// channel bucket so that the kernels compile in parallel).
#include "raster_impl.cuh"

namespace splat {
SPLAT_INSTANTIATE_CM(8)
}  // namespace splat
