// sg_noalloc.cu -- argmax over a caller's gain vector without allocating.
//
// Who needs this: code that cannot call cudaMalloc (or any allocator) at
// the moment it needs the argmax -- for example a latency-bound serving
// loop that must not stall on a synchronous allocation, or a plug-in
// running inside a host framework that owns every byte of device memory
// through its own pool and hands out only the buffers it manages.  Such
// callers pass their own input and output buffers; the only scratch used
// here is the statically sized `na_scratch` array below, which the CUDA
// runtime places in device memory when the library is loaded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "sg_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;
constexpr int NA_MAX_CONTEXTS = 64;

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

// The looked-up address is only valid in the CUDA context it was looked up
// in, so it is cached per context, keyed by the driver's process-unique
// context id (a context created after a device reset gets a new id).
std::mutex na_mu;
struct NaEntry {
    unsigned long long ctx_id;
    NaScratch *addr;
};
NaEntry na_cache[NA_MAX_CONTEXTS] = {};
int na_cached = 0;

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
    // 64-bit index: n may lie within one grid stride of 2^31
    for (long long v = (long long)blockIdx.x * NA_THREADS + threadIdx.x; v < n;
         v += (long long)gridDim.x * NA_THREADS) {
        const long long x = s[v];
        if (x > bg) {
            bg = x;
            bi = (int)v;
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

// Id of the current CUDA context (the current device's primary context
// when no context is current yet), via the driver entry points the runtime
// exposes, so no link against the driver library is needed.
sg_status na_context_id(unsigned long long *id)
{
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    if (!get_cur || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            sgi::set_error("sg_argmax_noalloc: driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
            return SG_ECUDA;
        }
        get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) == CUDA_SUCCESS && !ctx) {
        // nothing current yet: bind the current device's primary context
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) get_cur(&ctx);
    }
    if (!ctx || get_id(ctx, id) != CUDA_SUCCESS) {
        sgi::set_error("sg_argmax_noalloc: no current CUDA context");
        return SG_ECUDA;
    }
    return SG_OK;
}

// Device address of na_scratch in the current context, looked up once per
// context (cudaGetSymbolAddress with that context's device current).
sg_status na_scratch_address(NaScratch **out)
{
    unsigned long long id = 0;
    SG_TRY(na_context_id(&id));
    std::lock_guard<std::mutex> lock(na_mu);
    for (int i = 0; i < na_cached; ++i)
        if (na_cache[i].ctx_id == id) {
            *out = na_cache[i].addr;
            return SG_OK;
        }
    if (na_cached >= NA_MAX_CONTEXTS) {
        sgi::set_error("sg_argmax_noalloc: more than %d CUDA contexts", NA_MAX_CONTEXTS);
        return SG_EINVAL;
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
    if (e != cudaSuccess || !p) {
        sgi::set_error("sg_argmax_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    na_cache[na_cached++] = NaEntry{id, static_cast<NaScratch *>(p)};
    *out = static_cast<NaScratch *>(p);
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
