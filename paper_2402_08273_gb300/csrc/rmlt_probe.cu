// Device ceilings of the traversal roofline, measured on the device at hand:
// the L2 read bandwidth that node and triangle fetches draw on (the BVH of
// the bench scenes fits in L2), and the FP32 fused multiply-add rate that the
// slab and triangle tests draw on.
#include <cuda_runtime.h>

#include <cstdint>

#include "rmlt.h"
#include "rmlt_internal.h"

namespace rmlt {
namespace {

// Every thread streams 16-byte words through the buffer with L2-only loads
// (ld.global.cg skips L1), four independent loads per iteration, `reps`
// passes; one warp load instruction moves 512 bytes, so issue never limits it.
__global__ void __launch_bounds__(256) probe_l2_kernel(const float4* __restrict__ buf, size_t n, int reps,
                                                       unsigned* __restrict__ sink)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nt = (size_t)gridDim.x * blockDim.x;
    unsigned acc = 0u;
    for (int r = 0; r < reps; ++r) {
        for (size_t i = tid; i + 3 * nt < n; i += 4 * nt) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + nt);
            const float4 c = __ldcg(buf + i + 2 * nt), d = __ldcg(buf + i + 3 * nt);
            acc ^= __float_as_uint(a.x) ^ __float_as_uint(a.y) ^ __float_as_uint(a.z) ^ __float_as_uint(a.w);
            acc ^= __float_as_uint(b.x) ^ __float_as_uint(b.y) ^ __float_as_uint(b.z) ^ __float_as_uint(b.w);
            acc ^= __float_as_uint(c.x) ^ __float_as_uint(c.y) ^ __float_as_uint(c.z) ^ __float_as_uint(c.w);
            acc ^= __float_as_uint(d.x) ^ __float_as_uint(d.y) ^ __float_as_uint(d.z) ^ __float_as_uint(d.w);
        }
    }
    if (acc == 0x12345678u) sink[tid] = acc;   // never true for the zero buffer; keeps the loads
}

// Eight independent FMA chains per thread.
__global__ void __launch_bounds__(256) probe_fma_kernel(int iters, float seed, unsigned* __restrict__ sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + (float)(threadIdx.x + k);
    const float m = 0.999999f, c = 1e-7f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = __float_as_uint(s);
}

}  // namespace
}  // namespace rmlt

using namespace rmlt;

extern "C" rmlt_status rmlt_probe_peaks(int device, void* cuda_stream, double* l2_read_gbs, double* fp32_tflops)
{
    if (!l2_read_gbs || !fp32_tflops) return RMLT_E_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return RMLT_E_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int sms = 0, l2 = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    if (sms <= 0 || l2 <= 0) return RMLT_E_CUDA;
    // a buffer of a quarter of L2 stays resident across passes
    const size_t bytes = ((size_t)l2 / 4) & ~(size_t)4095;
    const size_t n = bytes / sizeof(float4);
    float4* buf = nullptr;
    unsigned* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rmlt_status status = RMLT_E_CUDA;
    const unsigned blocks = (unsigned)sms * 8u;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return RMLT_E_OOM;
    if (cudaMalloc(&sink, sizeof(unsigned) * blocks * 256) != cudaSuccess) {
        cudaFree(buf);
        return RMLT_E_OOM;
    }
    do {
        if (cudaMemsetAsync(buf, 0, bytes, st) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        const int reps = 200;
        probe_l2_kernel<<<blocks, 256, 0, st>>>(buf, n, 2, sink);   // warm L2
        cudaEventRecord(e0, st);
        probe_l2_kernel<<<blocks, 256, 0, st>>>(buf, n, reps, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const size_t per_pass = (n / (4 * (size_t)blocks * 256)) * 4 * (size_t)blocks * 256 * sizeof(float4);
        *l2_read_gbs = (double)per_pass * reps / (ms * 1e-3) / 1e9;
        const int iters = 1 << 12;
        probe_fma_kernel<<<blocks, 256, 0, st>>>(1024, 1.0f, sink);   // warm clocks
        cudaEventRecord(e0, st);
        probe_fma_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
        *fp32_tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
        status = cudaGetLastError() == cudaSuccess ? RMLT_OK : RMLT_E_CUDA;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    return status;
}
