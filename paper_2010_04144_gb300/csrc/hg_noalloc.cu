// hg_noalloc.cu -- total-mass reduction that allocates no device memory.
//
// Who needs this: an application that has already handed the whole device
// heap to its own memory pool (so a cudaMalloc would fail or fragment it), or
// a watchdog thread that checks the mass of a running simulation and must not
// call cudaMalloc/cudaFree, because those calls can synchronise the device and
// stall the solver's streams.  The regular hg_mass takes its scratch from the
// context's allocator; this variant keeps its scratch in a fixed array inside
// the library instead, so the caller only provides the input state and the
// output location.
//
// The scratch is a file-scope __device__ array: every GPU that loads this
// library holds it (kNoallocPartials doubles) until the process exits.  All
// calls share it: two calls whose kernels overlap on the GPU (different
// streams without ordering between them) race on it and may return wrong
// sums.  Calls ordered on one stream are safe.  Each call overwrites every
// partial it reads, so nothing has to start at zero.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/hemegb.h"

namespace {

constexpr int kChunk = 8192;                   // sites per partial sum
constexpr int kThreads = 256;
constexpr int64_t kNoallocPartials = 16384;   // 128 KiB of FP64 partials per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

double *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__device__ __forceinline__ double weight_d(int i) {
    return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}

template <int S> __device__ __forceinline__ double load_dev(const void *f, int64_t idx, int i) {
    if (S == HG_STORE_F32) return (double)((const float *)f)[idx];
    if (S == HG_STORE_F16) return __dmul_rn((double)__half2float(((const __half *)f)[idx]), weight_d(i));
    return __dmul_rn((double)__bfloat162float(((const __nv_bfloat16 *)f)[idx]), weight_d(i));
}

__device__ __forceinline__ double block_sum(double a) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        a = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    }
    return a;
}

// Same partition, order and rounding as the context's mass reduction: block b
// sums the 19 rows of sites [b*8192, (b+1)*8192) in FP64, thread t taking every
// 256th site, with explicit rounding intrinsics (no contraction).
template <int S>
__global__ void __launch_bounds__(kThreads) k_mass_partials_static(const void *f, int64_t n,
                                                                   int64_t stride,
                                                                   double *partials) {
    const int64_t lo = (int64_t)blockIdx.x * kChunk;
    const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
    double a = 0.0;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
#pragma unroll
        for (int i = 0; i < 19; ++i) a = __dadd_rn(a, load_dev<S>(f, (int64_t)i * stride + s, i));
    }
    a = block_sum(a);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

__global__ void __launch_bounds__(kThreads) k_mass_final_static(const double *partials,
                                                                int64_t count, double *out) {
    double a = 0.0;
    for (int64_t j = threadIdx.x; j < count; j += blockDim.x) a = __dadd_rn(a, partials[j]);
    a = block_sum(a);
    if (threadIdx.x == 0) *out = a;
}

// Device address of the scratch array for the current device, looked up once
// and kept: it is valid for the primary context that existed at the lookup, so
// a process that resets the device must not call this entry point afterwards.
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int hg_mass_noalloc(const void *f_dev, int32_t storage, int64_t n, int64_t row_stride,
                               double *out_dev, void *stream) {
    if (n < 0 || row_stride < n || (n > 0 && !f_dev) || !out_dev) return HG_ERR_ARG;
    if (storage < HG_STORE_F32 || storage > HG_STORE_BF16) return HG_ERR_ARG;
    const int64_t parts = n > 0 ? (n + kChunk - 1) / kChunk : 0;
    if (parts > kNoallocPartials) return HG_ERR_ARG;  // more than 134,217,728 sites
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return HG_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(out_dev, 0, sizeof(double), st) == cudaSuccess ? HG_OK : HG_ERR_CUDA;
    if (storage == HG_STORE_F32)
        k_mass_partials_static<HG_STORE_F32><<<(unsigned)parts, kThreads, 0, st>>>(f_dev, n, row_stride, scratch);
    else if (storage == HG_STORE_F16)
        k_mass_partials_static<HG_STORE_F16><<<(unsigned)parts, kThreads, 0, st>>>(f_dev, n, row_stride, scratch);
    else
        k_mass_partials_static<HG_STORE_BF16><<<(unsigned)parts, kThreads, 0, st>>>(f_dev, n, row_stride, scratch);
    if (cudaGetLastError() != cudaSuccess) return HG_ERR_CUDA;
    k_mass_final_static<<<1, kThreads, 0, st>>>(scratch, parts, out_dev);
    return cudaGetLastError() == cudaSuccess ? HG_OK : HG_ERR_CUDA;
}
