// FP64 peak calibration for the roofline of the branch and bus kernels (no
// counterpart in the paper).  GB300 runs FP64 on a narrow pipe (one warp
// instruction per 64 cycles per SM sub-partition, whatever the number of active
// lanes), so the roofline of an FP64-bound kernel is that pipe's rate.  This
// kernel issues nothing but independent FP64 FMAs (eight chains per thread) and
// reads the SM clock and the global timer at both ends, so one call gives the
// achieved FMA rate, the clock it ran at and the rate per clock per
// sub-partition.
#include <cuda_runtime.h>

#include "../../include/admm.h"

namespace {

constexpr int kCalBlock = 256;

__global__ void __launch_bounds__(kCalBlock)
fp64_fma_kernel(double *out, long long *ticks, int iters)
{
    const double m = 0.999999, c = 1e-7;
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
    double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
    long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        ticks[0] = clock64() - c0;
        ticks[1] = t1 - t0;
    }
}

}  // namespace

extern "C" int admm_fp64_peak(int32_t iters, void *cuda_stream, double *out3)
{
    if (iters < 1 || !out3) return ADMM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return ADMM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = 2 * sms;               // 16 warps per SM: the pipe stays busy
    double *out = nullptr;
    long long *ticks = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * kCalBlock) != cudaSuccess) return ADMM_ERR_OOM;
    if (cudaMalloc(&ticks, 2 * sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        return ADMM_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = ADMM_ERR_CUDA;
    long long ht[2] = {0, 0};
    float ms = 0.f;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        fp64_fma_kernel<<<blocks, kCalBlock, 0, s>>>(out, ticks, 64);   // warm-up
        cudaEventRecord(e0, s);
        fp64_fma_kernel<<<blocks, kCalBlock, 0, s>>>(out, ticks, iters);
        cudaEventRecord(e1, s);
        if (cudaPeekAtLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaMemcpy(ht, ticks, sizeof(ht), cudaMemcpyDeviceToHost) == cudaSuccess && ms > 0.f &&
            ht[1] > 0)
            rc = ADMM_OK;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(ticks);
    if (rc != ADMM_OK) return rc;
    const double fmas = (double)blocks * kCalBlock * 8.0 * iters;
    const double mhz = (double)ht[0] / (double)ht[1] * 1e3;      // cycles per ns -> MHz
    out3[0] = 2.0 * fmas / (ms * 1e-3) / 1e9;                     // GFLOP/s
    out3[1] = mhz;
    out3[2] = fmas / (ms * 1e-3) / (mhz * 1e6) / (4.0 * sms);      // FMA per clock per sub-partition
    return ADMM_OK;
}
