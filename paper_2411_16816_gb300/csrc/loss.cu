// loss.cu -- L1 photometric term of the paper's loss (Eq. loss_fn, lambda_r L1): the
// scaled sum of |pred - target| and its gradient scale * sign(pred - target).
#include "types.cuh"

namespace splat {

__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ pred, const float* __restrict__ target,
                                            int64_t count, float scale, float* __restrict__ grad, float* loss) {
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = count / 4;
    const float4* p4 = reinterpret_cast<const float4*>(pred);
    const float4* t4 = reinterpret_cast<const float4*>(target);
    const bool vec = (((uintptr_t)pred | (uintptr_t)target | (uintptr_t)grad) & 15u) == 0;
    int64_t tail_start = 0;
    if (vec) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 p = p4[i], t = t4[i];
            const float d0 = p.x - t.x, d1 = p.y - t.y, d2 = p.z - t.z, d3 = p.w - t.w;
            acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
            if (grad) {
                auto sg = [](float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); };
                reinterpret_cast<float4*>(grad)[i] =
                    make_float4(scale * sg(d0), scale * sg(d1), scale * sg(d2), scale * sg(d3));
            }
        }
        tail_start = n4 * 4;
    }
    for (int64_t i = tail_start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float d = pred[i] - target[i];
        acc += fabsf(d);
        if (grad) grad[i] = scale * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float sm[8];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += sm[w];
        atomicAdd(loss, s * scale);
    }
}

void launch_l1(const float* pred, const float* target, int64_t count, float scale, float* grad, float* loss,
               cudaStream_t st) {
    if (count <= 0) return;
    int64_t blocks = (count / 4 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_l1<<<(unsigned)blocks, 256, 0, st>>>(pred, target, count, scale, grad, loss);
}

}  // namespace splat
