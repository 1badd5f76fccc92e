// admm_dual_update_noalloc: the z / y update and residual reduction of one ADMM
// iteration on caller-owned device buffers, with no device allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc -- for example a control
// loop whose device memory budget is fixed once at start-up, or a program whose
// device memory is all owned by another allocator (a framework's caching
// allocator) and which must not create allocations behind its back.  Such a
// caller passes its own inputs and outputs; the only scratch the reduction
// needs (one partial sum per block plus a ticket counter) lives in the
// file-scope array below, which every GPU that loads this library keeps for
// the life of the process (kNoallocMaxBlocks * 4 + 4 doubles = 128 KiB + 32 B).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/admm.h"
#include "admm_internal.cuh"

namespace {

constexpr int kNoallocBlock = 256;
constexpr int kNoallocPerThread = 16;
constexpr long long kNoallocChunk = (long long)kNoallocBlock * kNoallocPerThread;
constexpr int kNoallocMaxBlocks = 4096;
constexpr long long kNoallocMaxM = kNoallocChunk * kNoallocMaxBlocks;   // 16,777,216
constexpr int kMaxDevices = 64;

// [0]: ticket counter (first 4 bytes), [1..3] unused, [4 + 4b .. 4 + 4b + 3]:
// the four partial sums of block b.
static __device__ __align__(256) double g_noalloc_scratch[4 + 4 * kNoallocMaxBlocks];

// device address of the scratch array per device, looked up on the first
// call that succeeds on that device (a failed lookup is retried next call)
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices];

__global__ void __launch_bounds__(kNoallocBlock)
dual_update_noalloc_kernel(double *scratch, long long m, const double *__restrict__ u,
                           const double *__restrict__ xbar, const double *__restrict__ xbar_prev,
                           const double *__restrict__ rho, const double *__restrict__ lam,
                           double beta, int two_level, double *z, double *y, double *norms)
{
    __shared__ double sh[kNoallocBlock / 32][4];
    __shared__ bool last;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kNoallocChunk;
    for (int j = threadIdx.x; j < kNoallocChunk; j += kNoallocBlock) {
        const long long c = base + j;
        if (c >= m) break;
        const double r0 = u[c] - xbar[c];
        const double rc = rho[c];
        const double zn = two_level ? -(lam[c] + y[c] + rc * r0) / (beta + rc) : 0.0;
        const double yn = y[c] + rc * (r0 + zn);
        const double dx = rc * (xbar[c] - xbar_prev[c]);
        z[c] = zn;
        y[c] = yn;
        acc[0] += r0 * r0;
        acc[1] += (r0 + zn) * (r0 + zn);
        acc[2] += dx * dx;
        acc[3] += zn * zn;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) sh[w][k] = acc[k];
    __syncthreads();
    unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch);
    double *partials = scratch + 4;
    if (threadIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int ww = 0; ww < kNoallocBlock / 32; ++ww)
            for (int k = 0; k < 4; ++k) s[k] += sh[ww][k];
        for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = s[k];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = 0; b < gridDim.x; ++b) {
        const volatile double *pp = partials + 4 * b;
        for (int k = 0; k < 4; ++k) s[k] += pp[k];
    }
    // primal ||u - xbar||, primal_z ||u - xbar + z||, dual ||rho dxbar||, ||z||
    for (int k = 0; k < 4; ++k) norms[k] = sqrt(s[k]);
    *ticket = 0u;
}

}  // namespace

extern "C" int admm_dual_update_noalloc(int64_t m, const double *d_u, const double *d_xbar,
                                        const double *d_xbar_prev, const double *d_rho,
                                        const double *d_lambda, double beta, int32_t two_level,
                                        double *d_z, double *d_y, double *d_norms,
                                        void *cuda_stream)
{
    if (m < 1 || m > kNoallocMaxM) return ADMM_ERR_INVALID_ARG;
    if (!d_u || !d_xbar || !d_xbar_prev || !d_rho || !d_lambda || !d_z || !d_y || !d_norms)
        return ADMM_ERR_INVALID_ARG;
    if (!(beta >= 0.0)) return ADMM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADMM_ERR_CUDA;
    // set-up, once per device, with that device current: the device address
    // of the scratch array (its host-side name is only a stand-in)
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADMM_ERR_CUDA;
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the ticket counter must start at zero
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s) != cudaSuccess) return ADMM_ERR_CUDA;
    const int blocks = (int)((m + kNoallocChunk - 1) / kNoallocChunk);
    dual_update_noalloc_kernel<<<blocks, kNoallocBlock, 0, s>>>(
        scratch, (long long)m, d_u, d_xbar, d_xbar_prev, d_rho, d_lambda, beta, two_level, d_z,
        d_y, d_norms);
    // the launch's own error only: peeking leaves errors of unrelated earlier
    // work where their owner will find them
    return cudaPeekAtLastError() == cudaSuccess ? ADMM_OK : ADMM_ERR_CUDA;
}
