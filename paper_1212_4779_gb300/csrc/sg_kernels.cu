// sg_kernels.cu -- device kernels of the StaticGreedy-DU path on sm_103a.
//
// Snapshots are bit-sliced: one 64-bit word per (node, task) covers 64
// snapshots, so a single traversal of the graph serves 64 snapshots at
// once.  A node x carrying frontier bits F expands each arc e = (x, y) by
// computing the arc's live bits for exactly the snapshots in F from the
// splitmix64 hash in registers; the bits new to y are OR-ed into y's
// visited word and, if y had no pending bits, y is queued.  Every
// (snapshot, node) pair is therefore expanded exactly once per traversal.
//
// Two traversal engines share that step:
//   warp engine  one warp per task, visited/pending words in a per-warp
//                shared-memory open-addressing table; the frontier is
//                expanded 32 arcs at a time with a load-balanced
//                (prefix-sum + shuffle search) arc assignment.  A task
//                whose table passes half full is aborted and queued for
//   CTA engine   one 512-thread block per task with dense visited/pending
//                arrays in global memory, level-synchronous, block-wide
//                load-balanced arc expansion.  The same engine runs the
//                forward dynamic-update BFS on the coverage bitsets.
// Tasks:
//   init (Algorithm 2, first loop): (v, word) -> s_v += sum_x popc(vis_x)
//   reverse DU (Algorithm 2, inner loops): (w, word, M_w) newly covered ->
//       s_u -= popc(vis_u) for every u reaching w in the snapshots of M_w
//   forward DU: from v*, the nodes newly covered in every snapshot.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sg_internal.cuh"

namespace sgi {

namespace {

constexpr int EMPTY_KEY = -1;
constexpr unsigned FULL = 0xffffffffu;
constexpr long long SEED_MARK = -(1LL << 62);

enum { DIR_FWD = 0, DIR_REV = 1 };
enum { TASK_INIT = 0, TASK_REV = 1, TASK_FWD = 2 };

// ------------------------------------------------------------------ coins
// High 32 bits of splitmix64(base ^ (r << 40)) (Steele, Lea, Flood 2014,
// with Stafford's Mix13 finaliser), base = seed ^ e.
__device__ __forceinline__ uint32_t coin_hi32(uint64_t base, uint32_t r)
{
    uint64_t z = (base ^ ((uint64_t)r << 40)) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    uint32_t hi = (uint32_t)(z >> 32);
    return hi ^ (hi >> 31);
}

// Live bits, among the snapshot bits F of the word starting at snapshot r0,
// of arc eid with threshold-1 tm1 (live iff hi32 <= thr - 1).
__device__ __forceinline__ uint64_t live_bits(const Coins &co, uint32_t eid, uint32_t r0, uint64_t F,
                                              uint32_t tm1)
{
    if (co.none_live) return 0;
    const uint64_t base = co.seed ^ (uint64_t)eid;
    uint64_t m = 0;
    while (F) {
        const int b = __ffsll((long long)F) - 1;
        F &= F - 1;
        if (coin_hi32(base, r0 + (uint32_t)b) <= tm1) m |= 1ull << b;
    }
    return m;
}

__device__ __forceinline__ uint64_t word_mask(int word, int R)
{
    const int rem = R - word * 64;
    return rem >= 64 ? ~0ull : ((1ull << rem) - 1ull);
}

// --------------------------------------------------------------- the graph
template <int DIR>
__device__ __forceinline__ void row_of(const GraphView &g, int x, int &beg, int &end)
{
    if (DIR == DIR_FWD) {
        beg = __ldg(g.rp + x);
        end = __ldg(g.rp + x + 1);
    } else {
        beg = __ldg(g.crp + x);
        end = __ldg(g.crp + x + 1);
    }
}

// threshold-1 shared by every arc of x's row (UIC scalar; reverse WIC: the
// in-arcs of x all point at x, so they share 1/indeg(x)); forward WIC arcs
// carry their own and ignore this value.
template <int DIR, int MODEL>
__device__ __forceinline__ uint32_t row_tm1(const GraphView &g, const Coins &co, int x)
{
    if (MODEL == MODEL_WIC && DIR == DIR_REV) return __ldg(g.tmi + x);
    return co.uic_tm1;
}

template <int DIR, int MODEL>
__device__ __forceinline__ void arc_at(const GraphView &g, int j, uint32_t rtm1, int &y, uint32_t &eid,
                                       uint32_t &tm1)
{
    if (DIR == DIR_FWD) {
        if (MODEL == MODEL_WIC) {
            const uint2 a = __ldg(g.fw + j);
            y = (int)a.x;
            tm1 = a.y;
        } else {
            y = __ldg(g.col + j);
            tm1 = rtm1;
        }
        eid = (uint32_t)j;
    } else {
        const int2 a = __ldg(g.cin + j);
        y = a.x;
        eid = (uint32_t)a.y;
        tm1 = rtm1;
    }
}

__device__ __forceinline__ int find_word(const long long *off, int W, long long t)
{
    int lo = 0, hi = W - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// ============================================================ warp engine

template <int LOGC>
struct __align__(16) WarpTab {
    static constexpr int C = 1 << LOGC;
    unsigned long long vis[C];
    unsigned long long pend[C];
    int key[C];
    unsigned short queue[C];
    unsigned short touched[C];
    int qtail;
    int ntouched;
    int overflow;
    int pad;
};

// Find y's slot, inserting it if absent.  Returns -1 (and flags overflow)
// once the table holds `limit` keys; at most 31 racing lanes can pass the
// check, so the touched list never exceeds limit + 31 < C entries.
template <int LOGC>
__device__ __forceinline__ int table_slot(WarpTab<LOGC> &T, int y, int limit)
{
    constexpr int C = 1 << LOGC;
    uint32_t h = ((uint32_t)y * 2654435761u) >> (32 - LOGC);
    volatile int *keys = T.key;
    for (int probe = 0; probe < C; ++probe) {
        const int k = keys[h];
        if (k == y) return (int)h;
        if (k == EMPTY_KEY) {
            if (*(volatile int *)&T.ntouched >= limit) {
                T.overflow = 1;
                return -1;
            }
            const int old = atomicCAS(&T.key[h], EMPTY_KEY, y);
            if (old == EMPTY_KEY) {
                const int t = atomicAdd(&T.ntouched, 1);
                T.touched[t] = (unsigned short)h;
                return (int)h;
            }
            if (old == y) return (int)h;
        }
        h = (h + 1) & (C - 1);
    }
    T.overflow = 1;
    return -1;
}

struct EngineArgs {
    GraphView g;
    Coins co;
    Ctl *ctl;
    long long *s;
    const long long *du_off;
    const int32_t *du_x;
    const unsigned long long *du_m;
    int32_t *big_list;
    long long ntasks;  // TASK_INIT only; TASK_REV reads ctl->du_total
    int chunk;
};

template <int LOGC, int DIR, int MODEL, int TASK>
__global__ void __launch_bounds__(128) warp_engine_kernel(EngineArgs a)
{
    constexpr int C = 1 << LOGC;
    constexpr int LIMIT = C / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    WarpTab<LOGC> &T = reinterpret_cast<WarpTab<LOGC> *>(smem_raw)[threadIdx.x >> 5];

    for (int i = lane; i < C; i += 32) {
        T.key[i] = EMPTY_KEY;
        T.vis[i] = 0;
        T.pend[i] = 0;
    }
    if (lane == 0) {
        T.qtail = 0;
        T.ntouched = 0;
        T.overflow = 0;
    }
    __syncwarp();

    const GraphView &g = a.g;
    const Coins &co = a.co;
    const long long ntasks = (TASK == TASK_INIT) ? a.ntasks : *(volatile long long *)&a.ctl->du_total;
    const int n = g.n;
    unsigned long long my_edges = 0;

    while (true) {
        long long base = 0;
        if (lane == 0) base = (long long)atomicAdd(&a.ctl->task_next, (unsigned long long)a.chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= ntasks) break;
        const long long tend = min(base + (long long)a.chunk, ntasks);
        for (long long t = base; t < tend; ++t) {
            int x0, word;
            uint64_t M0;
            if (TASK == TASK_INIT) {
                x0 = (int)(t / co.W);
                word = (int)(t - (long long)x0 * co.W);
                M0 = word_mask(word, co.R);
            } else {
                word = find_word(a.du_off, co.W, t);
                const long long i = t - a.du_off[word];
                x0 = a.du_x[(long long)word * n + i];
                M0 = a.du_m[(long long)word * n + i];
            }
            if (lane == 0) {
                const uint32_t h = ((uint32_t)x0 * 2654435761u) >> (32 - LOGC);
                T.key[h] = x0;
                T.vis[h] = M0;
                T.pend[h] = M0;
                T.touched[0] = (unsigned short)h;
                T.ntouched = 1;
                T.queue[0] = (unsigned short)h;
                T.qtail = 1;
            }
            __syncwarp();
            const uint32_t r0 = (uint32_t)word * 64u;
            unsigned long long tedges = 0;
            int qhead = 0;
            while (true) {
                const int qtail = *(volatile int *)&T.qtail;
                const int ovf = *(volatile int *)&T.overflow;
                if (ovf || qhead >= qtail) break;
                const int nb = min(32, qtail - qhead);
                int beg = 0, end = 0;
                uint64_t F = 0;
                uint32_t rtm1 = co.uic_tm1;
                if (lane < nb) {
                    const int h = T.queue[(qhead + lane) & (C - 1)];
                    const int x = T.key[h];
                    F = T.pend[h];
                    T.pend[h] = 0;
                    row_of<DIR>(g, x, beg, end);
                    rtm1 = row_tm1<DIR, MODEL>(g, co, x);
                    tedges += (unsigned long long)__popcll(F) * (unsigned long long)(end - beg);
                }
                qhead += nb;
                __syncwarp();
                const int deg = end - beg;
                int incl = deg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(FULL, incl, 31);
                const int excl = incl - deg;
                for (int abase = 0; abase < total; abase += 32) {
                    const int j = abase + lane;
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int cand = lo + step;
                        const int ex = __shfl_sync(FULL, excl, cand & 31);
                        if (cand < nb && ex <= j) lo = cand;
                    }
                    const int ibeg = __shfl_sync(FULL, beg, lo);
                    const int iex = __shfl_sync(FULL, excl, lo);
                    const uint64_t iF = __shfl_sync(FULL, F, lo);
                    const uint32_t itm1 = __shfl_sync(FULL, rtm1, lo);
                    if (j < total) {
                        int y;
                        uint32_t eid, tm1;
                        arc_at<DIR, MODEL>(g, ibeg + (j - iex), itm1, y, eid, tm1);
                        const uint64_t ml = live_bits(co, eid, r0, iF, tm1);
                        if (ml) {
                            const int h = table_slot<LOGC>(T, y, LIMIT);
                            if (h >= 0) {
                                const uint64_t old = atomicOr(&T.vis[h], (unsigned long long)ml);
                                const uint64_t nw = ml & ~old;
                                if (nw) {
                                    const uint64_t oldp = atomicOr(&T.pend[h], (unsigned long long)nw);
                                    if (oldp == 0) {
                                        const int pos = atomicAdd(&T.qtail, 1);
                                        T.queue[pos & (C - 1)] = (unsigned short)h;
                                    }
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
            __syncwarp();
            const int ovf = *(volatile int *)&T.overflow;
            const int nt = *(volatile int *)&T.ntouched;
            long long cnt = 0;
            for (int i = lane; i < nt; i += 32) {
                const int h = T.touched[i];
                if (!ovf) {
                    const int c = __popcll(T.vis[h]);
                    if (TASK == TASK_INIT) cnt += c;
                    else atomicAdd((unsigned long long *)&a.s[T.key[h]], (unsigned long long)(-(long long)c));
                }
                T.key[h] = EMPTY_KEY;
                T.vis[h] = 0;
                T.pend[h] = 0;
            }
            if (TASK == TASK_INIT) cnt = warp_sum(cnt);
            if (!ovf) my_edges += tedges;
            __syncwarp();
            if (lane == 0) {
                if (ovf) {
                    const unsigned long long idx = atomicAdd(&a.ctl->big_count, 1ull);
                    a.big_list[idx] = (int32_t)t;
                } else if (TASK == TASK_INIT) {
                    atomicAdd((unsigned long long *)&a.s[x0], (unsigned long long)cnt);
                }
                T.qtail = 0;
                T.ntouched = 0;
                T.overflow = 0;
            }
            __syncwarp();
        }
    }
    my_edges = warp_sum(my_edges);
    if (lane == 0 && my_edges)
        atomicAdd(TASK == TASK_INIT ? &a.ctl->init_edges : &a.ctl->rev_edges, my_edges);
}

// ============================================================= CTA engine

constexpr int BT = 512;  // threads of the CTA engine
constexpr int BW = BT / 32;

struct CtaShared {
    unsigned long long F[BT];
    int x[BT];
    int beg[BT];
    int ex[BT];
    uint32_t tm1[BT];
    int wsum[BW];
    int qlen, qnext, ntouch, ndu, total;
    long long red_ll[BW];
    unsigned long long red_ull[BW];
};

// Block-wide exclusive scan of v; returns the exclusive prefix, *total the sum.
__device__ __forceinline__ int block_excl_scan(int v, CtaShared &S, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) S.wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < BW ? S.wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < BW) S.wsum[lane] = wi - w;
        if (lane == BW - 1) S.total = wi;
    }
    __syncthreads();
    const int r = S.wsum[wid] + incl - v;
    *total = S.total;
    return r;
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < BW; ++i) r += red[i];
    return r;  // valid in thread 0
}

struct CtaTask {
    unsigned long long *vis;
    unsigned long long *pend;
    int32_t *qa;
    int32_t *qb;
    int32_t *touched;        // TASK_INIT / TASK_REV
    unsigned long long *nbits;  // TASK_FWD
    int32_t *du_x;           // TASK_FWD (this word's list)
    unsigned long long *du_m;   // TASK_FWD
};

// One traversal by the whole block.  TASK_INIT / TASK_REV: vis/pend are a
// zeroed slot and are zero again on return.  TASK_FWD: vis is the word's
// coverage bitset, the start bits are M0 minus what is already covered, and
// every node gaining bits is listed once with its merged new bits.
template <int DIR, int MODEL, int TASK>
__device__ void cta_bfs(const GraphView &g, const Coins &co, Ctl *ctl, long long *s, CtaTask w, int x0,
                        int word, uint64_t M0, CtaShared &S)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.qlen = 0;
        S.qnext = 0;
        S.ntouch = 0;
        S.ndu = 0;
        uint64_t M = M0;
        if (TASK == TASK_FWD) M &= ~w.vis[x0];
        if (M) {
            w.vis[x0] |= M;
            w.pend[x0] = M;
            w.qa[0] = x0;
            S.qlen = 1;
            if (TASK == TASK_FWD) {
                w.nbits[x0] |= M;
                w.du_x[0] = x0;
                S.ndu = 1;
            } else {
                w.touched[0] = x0;
                S.ntouch = 1;
            }
        }
    }
    long long cnt = (TASK == TASK_INIT && tid == 0) ? (long long)__popcll(M0) : 0;
    unsigned long long edges = 0;
    const uint32_t r0 = (uint32_t)word * 64u;
    int32_t *cur = w.qa, *nxt = w.qb;
    __syncthreads();
    while (true) {
        const int L = S.qlen;
        if (L == 0) break;
        for (int cbase = 0; cbase < L; cbase += BT) {
            const int i = cbase + tid;
            int deg = 0;
            if (i < L) {
                const int x = cur[i];
                const uint64_t F = atomicExch(&w.pend[x], 0ull);
                int beg, end;
                row_of<DIR>(g, x, beg, end);
                deg = F ? end - beg : 0;
                S.x[tid] = x;
                S.F[tid] = F;
                S.beg[tid] = beg;
                S.tm1[tid] = row_tm1<DIR, MODEL>(g, co, x);
                edges += (unsigned long long)__popcll(F) * (unsigned long long)(end - beg);
            }
            int total;
            const int ex = block_excl_scan(deg, S, &total);
            S.ex[tid] = ex;
            __syncthreads();
            const int nb = min(BT, L - cbase);
            for (int abase = 0; abase < total; abase += BT) {
                const int j = abase + tid;
                if (j < total) {
                    int lo = 0, hi = nb - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (S.ex[mid] <= j) lo = mid;
                        else hi = mid - 1;
                    }
                    int y;
                    uint32_t eid, tm1;
                    arc_at<DIR, MODEL>(g, S.beg[lo] + (j - S.ex[lo]), S.tm1[lo], y, eid, tm1);
                    const uint64_t ml = live_bits(co, eid, r0, S.F[lo], tm1);
                    if (ml) {
                        const uint64_t old = atomicOr(&w.vis[y], (unsigned long long)ml);
                        const uint64_t nw = ml & ~old;
                        if (nw) {
                            if (TASK == TASK_INIT) cnt += __popcll(nw);
                            if (TASK != TASK_FWD && old == 0) w.touched[atomicAdd(&S.ntouch, 1)] = y;
                            if (TASK == TASK_FWD) {
                                const uint64_t ob = atomicOr(&w.nbits[y], (unsigned long long)nw);
                                if (ob == 0) w.du_x[atomicAdd(&S.ndu, 1)] = y;
                            }
                            const uint64_t op = atomicOr(&w.pend[y], (unsigned long long)nw);
                            if (op == 0) nxt[atomicAdd(&S.qnext, 1)] = y;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            S.qlen = S.qnext;
            S.qnext = 0;
        }
        int32_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
        __syncthreads();
    }
    // epilogue
    if (TASK == TASK_FWD) {
        const int nd = S.ndu;
        for (int i = tid; i < nd; i += BT) {
            const int y = w.du_x[i];
            w.du_m[i] = w.nbits[y];
            w.nbits[y] = 0;
        }
    } else {
        const int nt = S.ntouch;
        for (int i = tid; i < nt; i += BT) {
            const int y = w.touched[i];
            if (TASK == TASK_REV)
                atomicAdd((unsigned long long *)&s[y], (unsigned long long)(-(long long)__popcll(w.vis[y])));
            w.vis[y] = 0;
        }
    }
    const unsigned long long e_tot = block_sum(edges, S.red_ull);
    if (TASK == TASK_INIT) {
        const long long c_tot = block_sum(cnt, S.red_ll);
        if (tid == 0) atomicAdd((unsigned long long *)&s[x0], (unsigned long long)c_tot);
    }
    if (tid == 0 && e_tot) {
        unsigned long long *dst =
            TASK == TASK_INIT ? &ctl->init_edges : (TASK == TASK_REV ? &ctl->rev_edges : &ctl->fwd_edges);
        atomicAdd(dst, e_tot);
    }
    __syncthreads();
}

struct BigArgs {
    GraphView g;
    Coins co;
    Ctl *ctl;
    long long *s;
    const long long *du_off;
    const int32_t *du_x;
    const unsigned long long *du_m;
    const int32_t *big_list;
    unsigned long long *slot_vis, *slot_pend;
    int32_t *slot_qa, *slot_qb, *slot_touched;
};

// Tasks the warp engine gave up on, one per block, dense per-block slots.
template <int DIR, int MODEL, int TASK>
__global__ void __launch_bounds__(BT) cta_engine_kernel(BigArgs a)
{
    __shared__ CtaShared S;
    __shared__ long long sh_t;
    const int n = a.g.n;
    const size_t so = (size_t)blockIdx.x * (size_t)n;
    CtaTask w;
    w.vis = a.slot_vis + so;
    w.pend = a.slot_pend + so;
    w.qa = a.slot_qa + so;
    w.qb = a.slot_qb + so;
    w.touched = a.slot_touched + so;
    w.nbits = nullptr;
    w.du_x = nullptr;
    w.du_m = nullptr;
    const long long count = (long long)*(volatile unsigned long long *)&a.ctl->big_count;
    while (true) {
        if (threadIdx.x == 0) sh_t = (long long)atomicAdd(&a.ctl->big_next, 1ull);
        __syncthreads();
        const long long k = sh_t;
        __syncthreads();
        if (k >= count) break;
        const long long t = a.big_list[k];
        int x0, word;
        uint64_t M0;
        if (TASK == TASK_INIT) {
            x0 = (int)(t / a.co.W);
            word = (int)(t - (long long)x0 * a.co.W);
            M0 = word_mask(word, a.co.R);
        } else {
            word = find_word(a.du_off, a.co.W, t);
            const long long i = t - a.du_off[word];
            x0 = a.du_x[(long long)word * n + i];
            M0 = a.du_m[(long long)word * n + i];
        }
        cta_bfs<DIR, MODEL, TASK>(a.g, a.co, a.ctl, a.s, w, x0, word, M0, S);
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (TASK == TASK_INIT) atomicAdd(&a.ctl->init_big, (unsigned long long)count);
        else atomicAdd(&a.ctl->rev_big, (unsigned long long)count);
    }
}

struct FwdArgs {
    GraphView g;
    Coins co;
    Ctl *ctl;
    unsigned long long *cov, *nbits, *pendf, *du_m;
    int32_t *fq_a, *fq_b, *du_x;
    long long *du_off;  // [W+1]
    int32_t *du_cnt;    // [W]
};

// Forward DU (Algorithm 2 inner loops, first half): block `word` walks from
// v* over live arcs of the 64 snapshots of its word, with the word's
// coverage bitset as the visited set, listing newly covered (w, M_w).  The
// last block to finish turns the per-word counts into offsets.
template <int MODEL>
__global__ void __launch_bounds__(BT) fwd_du_kernel(FwdArgs a)
{
    __shared__ CtaShared S;
    __shared__ int sh_last;
    const int n = a.g.n;
    const int word = blockIdx.x;
    const int vstar = *(volatile int32_t *)&a.ctl->vstar;
    const size_t so = (size_t)word * (size_t)n;
    if (vstar >= 0) {
        CtaTask w;
        w.vis = a.cov + so;
        w.pend = a.pendf + so;
        w.qa = a.fq_a + so;
        w.qb = a.fq_b + so;
        w.touched = nullptr;
        w.nbits = a.nbits + so;
        w.du_x = a.du_x + so;
        w.du_m = a.du_m + so;
        cta_bfs<DIR_FWD, MODEL, TASK_FWD>(a.g, a.co, a.ctl, nullptr, w, vstar, word, word_mask(word, a.co.R), S);
    } else {
        if (threadIdx.x == 0) S.ndu = 0;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.du_cnt[word] = S.ndu;
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctl->fwd_arrivals, 1u);
        sh_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // last block: exclusive prefix of the per-word counts, in chunks of BT
    long long carry = 0;
    const int W = gridDim.x;
    for (int base = 0; base < W; base += BT) {
        const int i = base + threadIdx.x;
        const int v = i < W ? *(volatile int32_t *)&a.du_cnt[i] : 0;
        int total;
        const int ex = block_excl_scan(v, S, &total);
        if (i < W) a.du_off[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.du_off[W] = carry;
        a.ctl->du_total = carry;
        a.ctl->du_entries += (unsigned long long)carry;
        a.ctl->fwd_arrivals = 0;
    }
}

// ================================================================= argmax

constexpr int AM_T = 256;

__device__ __forceinline__ bool better(long long g1, int i1, long long g2, int i2)
{
    return g1 > g2 || (g1 == g2 && (unsigned)i1 < (unsigned)i2);
}

// v* = argmax over non-seeds (s >= 0) of s, lowest id on ties; the last
// block publishes it, marks v* as a seed, and resets the round's counters.
__global__ void __launch_bounds__(AM_T) argmax_kernel(long long *s, int n, Ctl *ctl, long long *pg, int *pi,
                                                      int32_t *out_seeds, long long *out_gains, int round)
{
    __shared__ long long sg[AM_T / 32];
    __shared__ int si[AM_T / 32];
    __shared__ int sh_last;
    long long bg = -1;
    int bi = -1;
    for (int v = blockIdx.x * AM_T + threadIdx.x; v < n; v += gridDim.x * AM_T) {
        const long long x = s[v];
        if (x > bg) {
            bg = x;
            bi = v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long og = __shfl_xor_sync(FULL, bg, o);
        const int oi = __shfl_xor_sync(FULL, bi, o);
        if (better(og, oi, bg, bi)) {
            bg = og;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sg[wid] = bg;
        si[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < AM_T / 32; ++w)
            if (better(sg[w], si[w], bg, bi)) {
                bg = sg[w];
                bi = si[w];
            }
        pg[blockIdx.x] = bg;
        pi[blockIdx.x] = bi;
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->argmax_arrivals, 1u);
        sh_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    bg = -1;
    bi = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += AM_T) {
        const long long og = *(volatile long long *)&pg[b];
        const int oi = *(volatile int *)&pi[b];
        if (oi >= 0 && better(og, oi, bg, bi)) {
            bg = og;
            bi = oi;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long og = __shfl_xor_sync(FULL, bg, o);
        const int oi = __shfl_xor_sync(FULL, bi, o);
        if (oi >= 0 && (bi < 0 || better(og, oi, bg, bi))) {
            bg = og;
            bi = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sg[wid] = bg;
        si[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < AM_T / 32; ++w)
            if (si[w] >= 0 && (bi < 0 || better(sg[w], si[w], bg, bi))) {
                bg = sg[w];
                bi = si[w];
            }
        out_seeds[round] = bi;
        out_gains[round] = bg;
        ctl->vstar = bi;
        if (bi >= 0) s[bi] = SEED_MARK;
        else ctl->flags |= 1;
        ctl->argmax_arrivals = 0;
        ctl->task_next = 0;
        ctl->big_next = 0;
        ctl->big_count = 0;
    }
}

// ============================================================== live masks

__global__ void live_masks_kernel(Coins co, long long m, const uint2 *fw, uint32_t uic_tm1, int wic,
                                  unsigned long long *out)
{
    const long long total = m * co.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / co.W;
        const int word = (int)(i - e * co.W);
        const uint32_t tm1 = wic ? fw[e].y : uic_tm1;
        out[i] = live_bits(co, (uint32_t)e, (uint32_t)word * 64u, word_mask(word, co.R), tm1);
    }
}

// ================================================================ launches

constexpr int WE_LOGC = 9;  // 512-entry table per warp
constexpr int WE_THREADS = 128;

template <int DIR, int MODEL, int TASK>
sg_status launch_warp_engine(sg_graph *g, const EngineArgs &a, cudaStream_t st)
{
    auto kern = warp_engine_kernel<WE_LOGC, DIR, MODEL, TASK>;
    const size_t smem = (WE_THREADS / 32) * sizeof(WarpTab<WE_LOGC>);
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WE_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    kern<<<g->num_sms * per_sm, WE_THREADS, smem, st>>>(a);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

template <int DIR, int MODEL, int TASK>
sg_status launch_cta_engine(sg_graph *g, const BigArgs &a, cudaStream_t st)
{
    cta_engine_kernel<DIR, MODEL, TASK><<<g->ws.nslots, BT, 0, st>>>(a);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

EngineArgs engine_args(sg_graph *g, const Coins &co)
{
    sg_workspace &ws = g->ws;
    EngineArgs a;
    a.g = view_of(g);
    a.co = co;
    a.ctl = ws.ctl.p;
    a.s = ws.s.p;
    a.du_off = ws.du_off.p;
    a.du_x = ws.du_x.p;
    a.du_m = ws.du_m.p;
    a.big_list = ws.big_list.p;
    a.ntasks = 0;
    a.chunk = 8;
    return a;
}

BigArgs big_args(sg_graph *g, const Coins &co)
{
    sg_workspace &ws = g->ws;
    BigArgs a;
    a.g = view_of(g);
    a.co = co;
    a.ctl = ws.ctl.p;
    a.s = ws.s.p;
    a.du_off = ws.du_off.p;
    a.du_x = ws.du_x.p;
    a.du_m = ws.du_m.p;
    a.big_list = ws.big_list.p;
    a.slot_vis = ws.slot_vis.p;
    a.slot_pend = ws.slot_pend.p;
    a.slot_qa = ws.slot_qa.p;
    a.slot_qb = ws.slot_qb.p;
    a.slot_touched = ws.slot_touched.p;
    return a;
}

template <int MODEL>
sg_status init_gains_t(sg_graph *g, const Coins &co, cudaStream_t st, cudaEvent_t after_warp)
{
    EngineArgs a = engine_args(g, co);
    a.ntasks = (long long)g->n * co.W;
    SG_TRY((launch_warp_engine<DIR_FWD, MODEL, TASK_INIT>(g, a, st)));
    if (after_warp) SG_CUDA_TRY(cudaEventRecord(after_warp, st));
    SG_TRY((launch_cta_engine<DIR_FWD, MODEL, TASK_INIT>(g, big_args(g, co), st)));
    return SG_OK;
}

template <int MODEL>
sg_status round_t(sg_graph *g, const Coins &co, int32_t round, cudaStream_t st)
{
    sg_workspace &ws = g->ws;
    argmax_kernel<<<ws.am_blocks, AM_T, 0, st>>>(ws.s.p, (int)g->n, ws.ctl.p, ws.am_gain.p, ws.am_id.p,
                                                 ws.out_seeds.p, ws.out_gains.p, round);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    FwdArgs f;
    f.g = view_of(g);
    f.co = co;
    f.ctl = ws.ctl.p;
    f.cov = ws.cov.p;
    f.nbits = ws.nbits.p;
    f.pendf = ws.pendf.p;
    f.du_m = ws.du_m.p;
    f.fq_a = ws.fq_a.p;
    f.fq_b = ws.fq_b.p;
    f.du_x = ws.du_x.p;
    f.du_off = ws.du_off.p;
    f.du_cnt = ws.du_cnt.p;
    fwd_du_kernel<MODEL><<<co.W, BT, 0, st>>>(f);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    EngineArgs a = engine_args(g, co);
    SG_TRY((launch_warp_engine<DIR_REV, MODEL, TASK_REV>(g, a, st)));
    SG_TRY((launch_cta_engine<DIR_REV, MODEL, TASK_REV>(g, big_args(g, co), st)));
    return SG_OK;
}

}  // namespace

thread_local int g_launches = 0;

sg_status run_init_gains(sg_graph *g, const Coins &co, int model, cudaStream_t st, cudaEvent_t after_warp)
{
    return model == MODEL_WIC ? init_gains_t<MODEL_WIC>(g, co, st, after_warp)
                              : init_gains_t<MODEL_UIC>(g, co, st, after_warp);
}

sg_status run_round(sg_graph *g, const Coins &co, int model, int32_t round, cudaStream_t st)
{
    return model == MODEL_WIC ? round_t<MODEL_WIC>(g, co, round, st) : round_t<MODEL_UIC>(g, co, round, st);
}

sg_status run_live_masks(sg_graph *g, const Coins &co, int model, uint64_t *out, cudaStream_t st)
{
    const long long total = g->m * co.W;
    if (total == 0) return SG_OK;
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)g->num_sms * 16);
    live_masks_kernel<<<blocks, 256, 0, st>>>(co, g->m, g->fw.p, co.uic_tm1, model == MODEL_WIC,
                                              reinterpret_cast<unsigned long long *>(out));
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

}  // namespace sgi
