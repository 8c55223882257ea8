// Roofline probe: the FP32 fused-multiply-add throughput of the GPU, measured rather than
// derived, as the denominator of the CUDA-core X-step's ALU roofline.  Every thread runs
// 16 independent FMA chains (enough in flight to cover the FMA latency at full occupancy);
// the chains' results are folded into one store so the compiler keeps every FMA.
#include "mwax_internal.cuh"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) fma_probe_kernel(float* sink, int iters, float a, float b)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // practically never taken
}

}  // namespace

extern "C" long long mwax_probe_fma(int blocks, int iters, float* sink, void* cuda_stream)
{
    if (blocks < 1 || iters < 1 || !sink) return -1;
    fma_probe_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(sink, iters, 0.9999999f, 1e-7f);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return (long long)blocks * 256 * iters * 8 * kChains;   // FMAs issued
}
