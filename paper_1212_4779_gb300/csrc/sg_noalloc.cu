// sg_noalloc.cu -- argmax over a caller's gain vector without allocating.
//
// Who needs this: code that cannot call cudaMalloc (or any allocator) at
// the moment it needs the argmax -- for example code recording a CUDA graph
// (an allocation inside stream capture breaks the capture), a latency-bound
// serving loop that must not stall on a synchronous allocation, or a
// plug-in running inside a host framework that owns every byte of device
// memory through its own pool.  Such callers pass their own input and
// output buffers; the only scratch used here is the statically sized
// `na_scratch` array below, which the CUDA runtime places in device memory
// when the library is loaded.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "sg_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;
constexpr int NA_MAX_DEVICES = 64;

// Per-block partial maxima and the arrival counter of the last-block
// reduction: 1024 x 12 bytes + 4 bytes.
struct NaScratch {
    long long gain[NA_MAX_BLOCKS];
    int id[NA_MAX_BLOCKS];
    unsigned int arrivals;
};

// One copy per device that loads the library, kept until the process
// exits.  Host code must not use this name as a pointer: its device
// address comes from cudaGetSymbolAddress (na_scratch_address below).
static __device__ __align__(256) NaScratch na_scratch;

std::mutex na_mu;
NaScratch *na_addr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ bool na_better(long long g1, int i1, long long g2, int i2)
{
    return g1 > g2 || (g1 == g2 && (unsigned)i1 < (unsigned)i2);
}

__device__ __forceinline__ void na_warp_best(long long &bg, int &bi)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long og = __shfl_xor_sync(0xffffffffu, bg, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || na_better(og, oi, bg, bi))) {
            bg = og;
            bi = oi;
        }
    }
}

// argmax over v with s[v] >= 0, lowest id on ties; (-1, -1) if none.
__global__ void __launch_bounds__(NA_THREADS) na_argmax_kernel(const long long *s, int n, NaScratch *sc,
                                                               int32_t *out_id, long long *out_gain)
{
    __shared__ long long wg[NA_THREADS / 32];
    __shared__ int wi[NA_THREADS / 32];
    __shared__ int last;
    long long bg = -1;
    int bi = -1;
    for (int v = blockIdx.x * NA_THREADS + threadIdx.x; v < n; v += gridDim.x * NA_THREADS) {
        const long long x = s[v];
        if (x > bg) {
            bg = x;
            bi = v;
        }
    }
    na_warp_best(bg, bi);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        wg[w] = bg;
        wi[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < NA_THREADS / 32; ++k)
            if (wi[k] >= 0 && (bi < 0 || na_better(wg[k], wi[k], bg, bi))) {
                bg = wg[k];
                bi = wi[k];
            }
        sc->gain[blockIdx.x] = bg;
        sc->id[blockIdx.x] = bi;
        __threadfence();
        last = atomicAdd(&sc->arrivals, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    bg = -1;
    bi = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NA_THREADS) {
        const long long og = *(volatile long long *)&sc->gain[b];
        const int oi = *(volatile int *)&sc->id[b];
        if (oi >= 0 && (bi < 0 || na_better(og, oi, bg, bi))) {
            bg = og;
            bi = oi;
        }
    }
    na_warp_best(bg, bi);
    __syncthreads();
    if (lane == 0) {
        wg[w] = bg;
        wi[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < NA_THREADS / 32; ++k)
            if (wi[k] >= 0 && (bi < 0 || na_better(wg[k], wi[k], bg, bi))) {
                bg = wg[k];
                bi = wi[k];
            }
        *out_id = bi;
        *out_gain = bi >= 0 ? bg : -1;
        sc->arrivals = 0;
    }
}

// Device address of na_scratch on the current device, looked up once per
// device (cudaGetSymbolAddress with that device current).
sg_status na_scratch_address(NaScratch **out)
{
    int dev = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        sgi::set_error("sg_argmax_noalloc: device ordinal %d is beyond %d", dev, NA_MAX_DEVICES);
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(na_mu);
    if (!na_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p) {
            sgi::set_error("sg_argmax_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SG_ECUDA;
        }
        na_addr[dev] = static_cast<NaScratch *>(p);
    }
    *out = na_addr[dev];
    return SG_OK;
}

}  // namespace

extern "C" sg_status sg_argmax_noalloc(const int64_t *s, int64_t n, void *stream, int32_t *out_id,
                                       int64_t *out_gain)
{
    sgi::clear_error();
    if (!s || !out_id || !out_gain) {
        sgi::set_error("sg_argmax_noalloc: NULL argument");
        return SG_EINVAL;
    }
    if (n < 1 || n > (int64_t)INT32_MAX) {
        sgi::set_error("sg_argmax_noalloc: n = %lld is outside [1, 2^31 - 1]", (long long)n);
        return SG_EINVAL;
    }
    NaScratch *sc = nullptr;
    SG_TRY(na_scratch_address(&sc));
    cudaStream_t st = (cudaStream_t)stream;
    // the arrival counter must start at zero (the last block also resets it)
    SG_CUDA_TRY(cudaMemsetAsync(&sc->arrivals, 0, sizeof(unsigned int), st));
    const int blocks = (int)std::min<int64_t>(NA_MAX_BLOCKS, (n + NA_THREADS - 1) / NA_THREADS);
    na_argmax_kernel<<<blocks, NA_THREADS, 0, st>>>(reinterpret_cast<const long long *>(s), (int)n, sc, out_id,
                                                    reinterpret_cast<long long *>(out_gain));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}
