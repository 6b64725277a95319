// noalloc.cu -- exact all-pairs repulsion for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a framework whose caching
// allocator owns the whole device pool and forbids side allocations, and
// latency-critical loops, where cudaMalloc / cudaFree may synchronise the device and
// stall other streams. tfdp_exact_repulsion_noalloc serves them: it takes caller-owned
// input and output buffers and keeps its only scratch (per-chunk partial sums) in the
// file-scope device array below, of fixed size. Every GPU that loads this library
// holds that array until the process exits.
//
// The paper has no counterpart of this entry point; the arithmetic is the exact
// repulsion of Eq. (repfK), as in the graph API's exact path.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/tfdp.h"

namespace {

constexpr int kNaMaxN = TFDP_NOALLOC_MAX_N;
constexpr int kNaChunks = 16;     // source chunks, one partial sum each
constexpr int kNaThreads = 256;   // targets per CTA
constexpr int kNaMaxDevices = 128;

// Partial sums [chunk][target]: kNaChunks * kNaMaxN float2 = 2 MiB. Every call
// overwrites all the entries it later reads, so nothing needs clearing between calls.
static __device__ __align__(256) float2 g_noalloc_part[kNaChunks * kNaMaxN];

// Device address of g_noalloc_part per device (host code must not use the symbol itself,
// which on the host is only a stand-in, not a device address).
void* g_part_addr[kNaMaxDevices];
cudaError_t g_setup_err[kNaMaxDevices];
std::once_flag g_setup_once[kNaMaxDevices];

__device__ __forceinline__ float na_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float na_lg2(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float na_ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// (1 + d^2)^-gamma from u = 1 + d^2; integer gamma in {2, 4, 8} by squaring.
__device__ __forceinline__ float na_kernel(float u, float gamma, int gi) {
    if (gi == 0) return na_ex2(-gamma * na_lg2(u));
    float k = na_rcp(u);
    k = k * k;
    if (gi >= 4) k = k * k;
    if (gi >= 8) k = k * k;
    return k;
}

// Partial repulsion of source chunk blockIdx.y on the targets of this CTA.
__global__ void __launch_bounds__(kNaThreads) k_na_pairs(const float2* __restrict__ xy, int n, float gamma,
                                                         int gi, float2* __restrict__ part) {
    __shared__ float2 tile[kNaThreads];
    const int i = blockIdx.x * kNaThreads + threadIdx.x;
    const float2 pi = (i < n) ? xy[i] : make_float2(0.0f, 0.0f);
    const int csize = (n + kNaChunks - 1) / kNaChunks;
    const int j0 = blockIdx.y * csize;
    const int j1 = min(n, j0 + csize);
    float fx = 0.0f, fy = 0.0f;
    for (int s0 = j0; s0 < j1; s0 += kNaThreads) {
        const int j = s0 + threadIdx.x;
        tile[threadIdx.x] = (j < j1) ? xy[j] : pi;
        __syncthreads();
        const int cnt = min(kNaThreads, j1 - s0);
        for (int jj = 0; jj < cnt; ++jj) {
            const float2 q = tile[jj];
            const float dx = pi.x - q.x, dy = pi.y - q.y;
            const float K = na_kernel(fmaf(dx, dx, fmaf(dy, dy, 1.0f)), gamma, gi);
            fx = fmaf(K, dx, fx);
            fy = fmaf(K, dy, fy);
        }
        __syncthreads();
    }
    if (i < n) part[(size_t)blockIdx.y * n + i] = make_float2(fx, fy);
}

// frep[i] = sum over chunks of part[chunk][i], in chunk order.
__global__ void __launch_bounds__(kNaThreads) k_na_reduce(const float2* __restrict__ part, int n,
                                                          float2* __restrict__ frep) {
    const int i = blockIdx.x * kNaThreads + threadIdx.x;
    if (i >= n) return;
    float fx = 0.0f, fy = 0.0f;
    for (int c = 0; c < kNaChunks; ++c) {
        const float2 v = part[(size_t)c * n + i];
        fx += v.x;
        fy += v.y;
    }
    frep[i] = make_float2(fx, fy);
}

int na_gamma_int(double g) {
    if (g == 2.0) return 2;
    if (g == 4.0) return 4;
    if (g == 8.0) return 8;
    return 0;
}

}  // namespace

extern "C" tfdp_status tfdp_exact_repulsion_noalloc(const float* xy, int64_t n, double gamma, float* frep,
                                                    void* stream) {
    if (n < 0 || (n > 0 && (!xy || !frep))) return TFDP_ERR_INVALID_ARG;
    // the kernels read and write whole float2 pairs: both pointers must be 8-byte aligned
    if ((((uintptr_t)xy) | ((uintptr_t)frep)) & 7u) return TFDP_ERR_INVALID_ARG;
    if (n > kNaMaxN) return TFDP_ERR_PARAM_RANGE;  // beyond the fixed scratch
    if (!(gamma > 1.0) || gamma > 1e6) return TFDP_ERR_PARAM_RANGE;
    if (n == 0) return TFDP_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return TFDP_ERR_CUDA;
    // both buffers must be device (or managed) memory that the current device owns;
    // cudaPointerGetAttributes allocates nothing
    for (const void* ptr : {(const void*)xy, (const void*)frep}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return TFDP_ERR_INVALID_ARG;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return TFDP_ERR_INVALID_ARG;
        if (at.type == cudaMemoryTypeDevice && at.device != dev) return TFDP_ERR_INVALID_ARG;
    }
    // One-time set-up on this device, with the device current: the device address of
    // the scratch array.
    std::call_once(g_setup_once[dev], [dev]() {
        g_setup_err[dev] = cudaGetSymbolAddress(&g_part_addr[dev], g_noalloc_part);
    });
    if (g_setup_err[dev] != cudaSuccess || !g_part_addr[dev]) return TFDP_ERR_CUDA;
    float2* part = (float2*)g_part_addr[dev];
    cudaStream_t s = (cudaStream_t)stream;
    const int nn = (int)n;
    dim3 grid((nn + kNaThreads - 1) / kNaThreads, kNaChunks);
    k_na_pairs<<<grid, kNaThreads, 0, s>>>((const float2*)xy, nn, (float)gamma, na_gamma_int(gamma), part);
    k_na_reduce<<<(nn + kNaThreads - 1) / kNaThreads, kNaThreads, 0, s>>>(part, nn, (float2*)frep);
    return cudaGetLastError() == cudaSuccess ? TFDP_OK : TFDP_ERR_CUDA;
}
