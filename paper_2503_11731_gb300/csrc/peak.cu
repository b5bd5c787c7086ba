// peak.cu -- a measurement kernel for the compositing roofline: the FP32
// fused multiply-add issue rate of the GPU, measured rather than derived
// from the SM count and clock.

#include "gsr_internal.cuh"

namespace gsr {

// Each thread runs kChains independent FMA dependency chains of `iters`
// steps (enough independent work per warp to keep the FP32 pipes issuing
// every cycle); the sum is stored so that nothing is eliminated.
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_chains(float* out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gsr

extern "C" gsr_status gsr_fma_peak_kernel(float* out, int32_t blocks, int32_t iters, int64_t* fmas, void* stream)
{
    if (!out || blocks <= 0 || iters <= 0 || !fmas) return GSR_ERR_INVALID_ARG;
    gsr::k_fma_chains<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.999f, 1e-3f);
    *fmas = (int64_t)blocks * 256 * gsr::kChains * iters;
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}
