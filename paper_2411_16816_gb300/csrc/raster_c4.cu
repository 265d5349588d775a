// raster_c4.cu -- rasterizer kernels for up to 4 channels (one translation unit per
// channel bucket so that the kernels compile in parallel).
#include "raster_impl.cuh"

namespace splat {
SPLAT_INSTANTIATE_CM(4)
}  // namespace splat
