// sg_cc.cu -- the undirected variant: uniform cascade on a symmetric graph
// with one coin per undirected edge (both arcs hash the lower of their two
// canonical arc ids).  Each snapshot is then an undirected graph, as Section
// 3.4.1 treats undirected snapshots, and R(G'_r, v) is v's connected
// component.  So Algorithm 2 reduces to component bookkeeping:
//   initial gains   s_v = sum_r |C_r(v)| (union-find per snapshot);
//   a round's seed  v*: in every snapshot where C_r(v*) is not yet covered,
//                   its |C_r(v*)| nodes are newly covered, and each of them
//                   (each reaches every newly covered node) loses |C_r(v*)|.
// The snapshot-edge counters follow from per-component sizes and degree
// sums, equal to the dynamic update's counts: init = sum_{v,r} degsum(C_r(v));
// forward = sum over newly covered components of degsum; reverse = sum over
// them of |C| * degsum (every node of C is reached backwards from each of the
// |C| newly covered nodes, and in-degree = out-degree).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "sg_internal.cuh"

using namespace sgi;

namespace {

constexpr int CC_T = 256;
constexpr long long CC_SPIN = 1LL << 24;


// Source of every arc and the lower id of each arc and its reverse;
// *asym is set if some arc has no reverse.
__global__ void cc_coupling_kernel(int n, long long m, const int32_t *rp, const int32_t *col, int32_t *esrc,
                                   int32_t *pmin, int32_t *asym)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;  // the row holding arc e: largest u with rp[u] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(rp + mid) <= e) lo = mid;
            else hi = mid - 1;
        }
        const int u = lo, v = __ldg(col + e);
        int a = __ldg(rp + v), b = __ldg(rp + v + 1);
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (__ldg(col + mid) < u) a = mid + 1;
            else b = mid;
        }
        const bool found = a < __ldg(rp + v + 1) && __ldg(col + a) == u;
        if (!found) *asym = 1;
        esrc[e] = u;
        pmin[e] = found ? (int32_t)min((long long)a, e) : (int32_t)e;
    }
}

__device__ __forceinline__ int cc_find(int32_t *lab, int x)
{
    // path halving; the shortcuts written are ancestors, so races only
    // leave longer paths, never wrong roots
    while (true) {
        const int p = *(volatile int32_t *)&lab[x];
        if (p == x) return x;
        const int gp = *(volatile int32_t *)&lab[p];
        if (gp != p) *(volatile int32_t *)&lab[x] = gp;
        x = gp;
    }
}

// Root without writing: used once hooking is over, while other threads
// store their final roots (a shortcut written then could overwrite a final
// root with an intermediate ancestor).
__device__ __forceinline__ int cc_root(const int32_t *lab, int x)
{
    while (true) {
        const int p = *(volatile const int32_t *)&lab[x];
        if (p == x) return x;
        x = p;
    }
}

__global__ void cc_init_kernel(int n, long long total, int32_t *lab)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        lab[i] = (int32_t)(i % n);
}

// Union the endpoints of every live undirected edge {u, v} (u < v, arc
// u->v is the lower id) in every snapshot; the larger root is hooked under
// the smaller by compare-and-swap.  A bounded number of retries per edge;
// on expiry the error flag is set.
__global__ void cc_hook_kernel(int n, long long m, int R, uint64_t seed, uint32_t tm1, int none_live,
                               const int32_t *esrc, const int32_t *col, int32_t *lab, int32_t *flags)
{
    if (none_live) return;
    const long long total = (long long)R * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / m);
        const long long e = i - (long long)r * m;
        int a = __ldg(esrc + e), b = __ldg(col + e);
        if (a >= b) continue;
        if (coin_hi32(seed ^ (uint64_t)e, (uint32_t)r) > tm1) continue;
        int32_t *L = lab + (size_t)r * n;
        long long tries = 0;
        while (true) {
            a = cc_find(L, a);
            b = cc_find(L, b);
            if (a == b) break;
            if (a > b) {
                const int t = a;
                a = b;
                b = t;
            }
            const int old = atomicCAS(&L[b], b, a);
            if (old == b) break;
            b = old;
            if (++tries > CC_SPIN) {
                atomicOr(flags, 8);
                break;
            }
        }
    }
}

// lab[r][v] = its root; component sizes and out-degree sums at the roots
// (csz, cdg zero on entry).
__global__ void cc_compress_kernel(int n, long long total, const int32_t *rp, int32_t *lab, int32_t *csz,
                                   unsigned long long *cdg)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / n);
        const int v = (int)(i - (long long)r * n);
        int32_t *L = lab + (size_t)r * n;
        const int root = cc_root(L, v);
        L[v] = root;  // only this thread writes L[v] here
        atomicAdd(&csz[(size_t)r * n + root], 1);
        atomicAdd(&cdg[(size_t)r * n + root], (unsigned long long)(__ldg(rp + v + 1) - __ldg(rp + v)));
    }
}

// s_v = sum_r |C_r(v)|; the initial snapshot-edge count.
__global__ void __launch_bounds__(CC_T) cc_gains_kernel(int n, int R, const int32_t *lab, const int32_t *csz,
                                                        const unsigned long long *cdg, long long *s,
                                                        unsigned long long *init_edges)
{
    __shared__ unsigned long long red[CC_T / 32];
    unsigned long long ed = 0;
    for (long long v = (long long)blockIdx.x * CC_T + threadIdx.x; v < n; v += (long long)gridDim.x * CC_T) {
        long long acc = 0;
        for (int r = 0; r < R; ++r) {
            const size_t q = (size_t)r * n + __ldg(lab + (size_t)r * n + v);
            acc += __ldg(csz + q);
            ed += __ldg(cdg + q);
        }
        s[v] = acc;
    }
    for (int o = 16; o > 0; o >>= 1) ed += __shfl_xor_sync(0xffffffffu, ed, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ed;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < CC_T / 32; ++w) t += red[w];
        if (t) atomicAdd(init_edges, t);
    }
}

// The round's seed v* (ctl->vstar): per snapshot, cover its component if it
// is not yet covered; nsz[r] = its size then (else 0), root[r] = its root.
__global__ void __launch_bounds__(CC_T) cc_cover_kernel(int n, int R, const int32_t *lab, const int32_t *csz,
                                                        const unsigned long long *cdg, uint8_t *cov, Ctl *ctl,
                                                        int32_t *root, int32_t *nsz)
{
    const int v = *(volatile int32_t *)&ctl->vstar;
    unsigned long long fwd = 0, rev = 0;
    for (int r = threadIdx.x; r < R; r += CC_T) {
        int c = -1, sz = 0;
        if (v >= 0) {
            c = lab[(size_t)r * n + v];
            const size_t q = (size_t)r * n + c;
            if (!cov[q]) {
                cov[q] = 1;
                sz = csz[q];
                fwd += cdg[q];
                rev += (unsigned long long)sz * cdg[q];
            }
        }
        root[r] = c;
        nsz[r] = sz;
    }
    if (fwd) atomicAdd(&ctl->fwd_edges, fwd);
    if (rev) atomicAdd(&ctl->rev_edges, rev);
}

// Every node in a newly covered component loses its size.
__global__ void __launch_bounds__(CC_T) cc_dec_kernel(int n, int R, const int32_t *lab, const int32_t *root,
                                                      const int32_t *nsz, long long *s)
{
    extern __shared__ int32_t sh[];  // root[R], nsz[R]
    for (int r = threadIdx.x; r < R; r += CC_T) {
        sh[r] = root[r];
        sh[R + r] = nsz[r];
    }
    __syncthreads();
    for (long long v = (long long)blockIdx.x * CC_T + threadIdx.x; v < n; v += (long long)gridDim.x * CC_T) {
        long long dec = 0;
        for (int r = 0; r < R; ++r)
            if (sh[R + r] && __ldg(lab + (size_t)r * n + v) == sh[r]) dec += sh[R + r];
        if (dec) s[v] -= dec;
    }
}

// Spread of S: per snapshot, the sizes of the distinct components S meets
// (mark zero on entry, reused as the "counted" flags).
__global__ void __launch_bounds__(CC_T) cc_spread_kernel(int n, int R, const int32_t *lab, const int32_t *csz,
                                                         const unsigned long long *cdg, const int32_t *S, int ns,
                                                         uint8_t *mark, long long *total, unsigned long long *edges)
{
    __shared__ long long rt[CC_T / 32];
    __shared__ unsigned long long re[CC_T / 32];
    long long t = 0;
    unsigned long long ed = 0;
    const long long work = (long long)R * ns;
    for (long long i = blockIdx.x * (long long)CC_T + threadIdx.x; i < work; i += (long long)gridDim.x * CC_T) {
        const int r = (int)(i / ns);
        const int v = __ldg(S + (i - (long long)r * ns));
        const size_t q = (size_t)r * n + __ldg(lab + (size_t)r * n + v);
        // one byte flag per (r, root): claim it with an atomic on its word
        unsigned int *wordp = (unsigned int *)(mark + (q & ~(size_t)3));
        const unsigned int bit = 1u << (8 * (q & 3));
        if (!(atomicOr(wordp, bit) & bit)) {
            t += __ldg(csz + q);
            ed += __ldg(cdg + q);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        ed += __shfl_xor_sync(0xffffffffu, ed, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rt[threadIdx.x >> 5] = t;
        re[threadIdx.x >> 5] = ed;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        unsigned long long b = 0;
        for (int w = 0; w < CC_T / 32; ++w) {
            a += rt[w];
            b += re[w];
        }
        if (a) atomicAdd((unsigned long long *)total, (unsigned long long)a);
        if (b) atomicAdd(edges, b);
    }
}

int grid_for(const sg_graph *g, long long work)
{
    return (int)std::max<long long>(1, std::min<long long>((work + CC_T - 1) / CC_T, (long long)g->num_sms * 16));
}

}  // namespace

namespace sgi {

// Coupling arrays of a symmetric graph, built on first use; SG_EINVAL for a
// graph with an arc whose reverse is missing.
sg_status cc_prepare_graph(sg_graph *g, cudaStream_t st)
{
    if (g->cc_sym == 0) {
        set_error("the undirected cascade needs a symmetric graph (every arc's reverse present)");
        return SG_EINVAL;
    }
    if (g->cc_sym == 1) return SG_OK;
    const long long m = g->m;
    DBuf<int32_t> flag;
    SG_TRY(dbuf_alloc(g->cc_esrc, (size_t)std::max<long long>(1, m), st));
    SG_TRY(dbuf_alloc(g->cc_pmin, (size_t)std::max<long long>(1, m), st));
    SG_TRY(dbuf_alloc(flag, 1, st));
    SG_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 4, st));
    if (m > 0) {
        cc_coupling_kernel<<<grid_for(g, m), CC_T, 0, st>>>((int)g->n, m, g->rp.p, g->col.p, g->cc_esrc.p,
                                                            g->cc_pmin.p, flag.p);
        SG_CUDA_TRY(cudaGetLastError());
        ++g_launches;
    }
    int32_t h = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(&h, flag.p, 4, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    dbuf_free(flag, st);
    g->cc_sym = h ? 0 : 1;
    if (!g->cc_sym) {
        set_error("the undirected cascade needs a symmetric graph (every arc's reverse present)");
        return SG_EINVAL;
    }
    return SG_OK;
}

size_t cc_workspace_bytes(const sg_graph *g, int32_t R)
{
    const size_t rn = (size_t)R * (size_t)g->n;
    return rn * (4 + 4 + 8 + 1) + (size_t)R * 8 + 64;
}

sg_status cc_ensure(sg_graph *g, sg_workspace &ws, int32_t R, cudaStream_t st)
{
    const size_t rn = (size_t)R * (size_t)g->n;
    if (ws.cc_cap < rn || ws.cc_rcap < R) {
        dbuf_free(ws.cc_lab, st);
        dbuf_free(ws.cc_size, st);
        dbuf_free(ws.cc_deg, st);
        dbuf_free(ws.cc_cov, st);
        dbuf_free(ws.cc_root, st);
        ws.cc_cap = 0;
        ws.cc_rcap = 0;
        SG_TRY(dbuf_alloc(ws.cc_lab, rn, st));
        SG_TRY(dbuf_alloc(ws.cc_size, rn, st));
        SG_TRY(dbuf_alloc(ws.cc_deg, rn, st));
        SG_TRY(dbuf_alloc(ws.cc_cov, rn + 8, st));
        SG_TRY(dbuf_alloc(ws.cc_root, (size_t)R * 2, st));
        ws.cc_cap = rn;
        ws.cc_rcap = R;
    }
    return SG_OK;
}

// Components of every snapshot (lab, csz, cdg) for R snapshots of `seed`.
sg_status cc_components(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    const long long total = (long long)co.R * g->n;
    SG_CUDA_TRY(cudaMemsetAsync(ws.cc_size.p, 0, (size_t)total * 4, st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.cc_deg.p, 0, (size_t)total * 8, st));
    cc_init_kernel<<<grid_for(g, total), CC_T, 0, st>>>((int)g->n, total, ws.cc_lab.p);
    if (g->m > 0)
        cc_hook_kernel<<<grid_for(g, (long long)co.R * g->m), CC_T, 0, st>>>(
            (int)g->n, g->m, co.R, co.seed, co.uic_tm1, co.none_live, g->cc_esrc.p, g->col.p, ws.cc_lab.p,
            &ws.ctl.p->flags);
    cc_compress_kernel<<<grid_for(g, total), CC_T, 0, st>>>((int)g->n, total, g->rp.p, ws.cc_lab.p, ws.cc_size.p,
                                                             reinterpret_cast<unsigned long long *>(ws.cc_deg.p));
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 3;
    return SG_OK;
}

// Initial gains into ws.s and the init counter (ctl zeroed by the caller).
sg_status cc_init_gains(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    SG_TRY(cc_components(g, ws, co, st));
    cc_gains_kernel<<<grid_for(g, g->n), CC_T, 0, st>>>((int)g->n, co.R, ws.cc_lab.p, ws.cc_size.p,
                                                         reinterpret_cast<const unsigned long long *>(ws.cc_deg.p),
                                                         ws.s.p, &ws.ctl.p->init_edges);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

// One selection round after the argmax has chosen ctl->vstar.
sg_status cc_round(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    int32_t *root = ws.cc_root.p, *nsz = ws.cc_root.p + co.R;
    cc_cover_kernel<<<1, CC_T, 0, st>>>((int)g->n, co.R, ws.cc_lab.p, ws.cc_size.p,
                                        reinterpret_cast<const unsigned long long *>(ws.cc_deg.p), ws.cc_cov.p,
                                        ws.ctl.p, root, nsz);
    cc_dec_kernel<<<grid_for(g, g->n), CC_T, (size_t)co.R * 8, st>>>((int)g->n, co.R, ws.cc_lab.p, root, nsz,
                                                                      ws.s.p);
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 2;
    return SG_OK;
}

sg_status cc_clear_cover(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    SG_CUDA_TRY(cudaMemsetAsync(ws.cc_cov.p, 0, (size_t)co.R * (size_t)g->n + 8, st));
    return SG_OK;
}

// sum_r |union of the components S meets|, and their degree sums.
sg_status cc_spread(sg_graph *g, sg_workspace &ws, const Coins &co, const int32_t *d_S, int32_t ns, long long *d_total,
                    unsigned long long *d_edges, cudaStream_t st)
{
    SG_TRY(cc_components(g, ws, co, st));
    SG_TRY(cc_clear_cover(g, ws, co, st));
    cc_spread_kernel<<<grid_for(g, (long long)co.R * ns), CC_T, 0, st>>>(
        (int)g->n, co.R, ws.cc_lab.p, ws.cc_size.p, reinterpret_cast<const unsigned long long *>(ws.cc_deg.p), d_S,
        ns, ws.cc_cov.p, d_total, d_edges);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

}  // namespace sgi
