// raster_c32.cu -- rasterizer kernels for up to 32 channels (one translation unit per
// channel bucket so that the kernels compile in parallel).
#include "raster_impl.cuh"

namespace splat {
SPLAT_INSTANTIATE_CM(32)
}  // namespace splat
