// sg_kernels.cu -- device kernels of the StaticGreedy-DU path on sm_103a.
//
// Snapshots are bit-sliced: a 64-bit word per (node, task) carries 64
// independent traversal states at once.  Two slicings are used:
//   snapshot-sliced  bit b = snapshot 64w+b.  Initial gains (Algorithm 2,
//                    first loop) run one task per (source v, word w); the
//                    forward dynamic update runs one per word from v*.
//   target-sliced    bit j = the j-th of up to 64 newly covered targets of
//                    ONE snapshot r.  The reverse dynamic update (Algorithm
//                    2, inner loops) runs one task per (r, 64 targets): each
//                    node u ends with the set of those targets it reaches,
//                    and s_u drops by its popcount -- exactly the per-(w, r)
//                    reverse BFS of the paper, with ancestors shared by the
//                    64 targets walked once.
// Expanding a node x with state F over an arc e = (x, y) ORs the arc's live
// bits into y: snapshot-sliced, live(e, 64w+b) for each b in F;
// target-sliced, F itself if live(e, r).  Coins come from the splitmix64
// hash in registers, except on heavy rows (degree >= a threshold) whose
// per-word live masks are computed once per query into a compact index
// (nonzero masks only), since hub rows are re-expanded by many tasks.
//
// Traversal engines, by task size:
//   tier 1  one warp per task, visited/pending words in a 512-slot
//           shared-memory hash table; frontier expanded 32 elements at a
//           time with a load-balanced (prefix sum + shuffle search) split.
//   tier 2  one 8-warp block per task sharing a 2048-slot shared-memory
//           table and an asynchronous ring queue, for tasks that filled the
//           tier-1 table past its limit with a small frontier left.
//   tier 3  the same cooperative engine over dense per-block arrays in
//           global memory (no limit): initial gains in 12-warp blocks
//           (the first queue positions in shared memory), reverse tasks in
//           4-warp blocks.
//   The forward dynamic update, the landmark walks and the ancestor walk
//   run level-synchronous block traversals over the coverage bitsets.
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
enum { TASK_INIT = 0, TASK_REVT = 1, TASK_FWD = 2, TASK_ANC = 3, TASK_LMK = 4, TASK_SPREAD = 5 };
enum { SLICE_SNAP = 0, SLICE_TGT = 1 };

constexpr int T1_LOGC = 9;   // tier-1 table: 512 slots per warp (shared memory)
constexpr int WE_THREADS = 128;
constexpr int MAX_LMK = 8;     // landmarks for the initial gains
// An initial-gain task expands a node whose state has at most this many
// snapshot bits through the per-snapshot live lists, one bit at a time
// (the other bits go back to pending); denser states scan the word's index.
constexpr int SPARSE_BITS = 4;
// Newly covered targets of one snapshot walked together by one reverse
// (dynamic-update) task, one state bit each (at most 64).
constexpr int REV_GROUP = 64;

// ------------------------------------------------------------------ coins
// coin_hi32 (sg_internal.cuh): the high 32 bits of the coin hash.

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

// Position of the (j+1)-th lowest set bit of m (j < popc(m)): a binary
// search on population counts of halves.
__device__ __forceinline__ int nth_bit(uint64_t m, int j)
{
    int pos = 0;
#pragma unroll
    for (int w = 32; w >= 1; w >>= 1) {
        const int c = __popcll(m & ((1ull << w) - 1ull));
        if (j >= c) {
            j -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// The elements one frontier entry expands: its arcs (light row) or its
// row's index entries for the word (heavy row).
struct Row {
    long long base;
    int vdeg;   // elements to expand
    int deg;    // degree in the canonical graph (work counter)
    int heavy;
    uint32_t rtm1;
    uint64_t live;    // snapshots of the word with a live out-arc (forward descriptors)
    long long lbase;  // start of the word's per-snapshot lists when `single`
    int single;       // every nonempty list of the word holds one arc
};

template <int DIR, int MODEL, int SLICE = SLICE_SNAP>
__device__ __forceinline__ Row row_ref(const GraphView &g, const Coins &co, int x, int word, uint32_t rs = 0)
{
    Row r;
    r.live = ~0ull;
    r.lbase = 0;
    r.single = 0;
    if (DIR == DIR_FWD && g.rdesc) {
        // one 32-byte sector instead of the row offsets, index ordinal,
        // segment prefix and list offsets one after another
        const int4 *p = g.rdesc + 2 * ((size_t)word * (size_t)g.n + x);
        const int4 d = __ldg(p), e = __ldg(p + 1);
        r.base = (long long)(((unsigned long long)(unsigned)d.y << 32) | (unsigned)d.x);
        r.vdeg = d.z;
        r.deg = d.w & 0x7fffffff;
        r.heavy = (int)((unsigned)d.w >> 31);
        r.rtm1 = co.uic_tm1;
        r.live = ((unsigned long long)(unsigned)e.y << 32) | (unsigned)e.x;
        r.lbase = (long long)(((unsigned long long)((unsigned)e.w & 0x7fffffffu) << 32) | (unsigned)e.z);
        r.single = (int)((unsigned)e.w >> 31);
        return r;
    }
    int beg, end;
    if (DIR == DIR_FWD) {
        beg = __ldg(g.rp + x);
        end = __ldg(g.rp + x + 1);
    } else {
        beg = __ldg(g.crp + x);
        end = __ldg(g.crp + x + 1);
    }
    r.deg = end - beg;
    // UIC: one threshold; reverse WIC: all in-arcs of x share 1/indeg(x);
    // forward WIC arcs carry their own threshold.
    r.rtm1 = (MODEL == MODEL_WIC && DIR == DIR_REV) ? __ldg(g.tmi + x) : co.uic_tm1;
    const HeavyView &hv = DIR == DIR_FWD ? g.hout : g.hin;
    const int h = g.heavy_on ? __ldg(hv.hid + x) : -1;
    if (DIR == DIR_REV && SLICE == SLICE_TGT && h >= 0 && hv.soff && __ldg(hv.svalid)) {
        // one snapshot: its live in-arcs directly
        const long long q = (long long)h * (64 * co.W) + rs;
        r.heavy = 2;
        r.base = __ldg(hv.soff + q);
        r.vdeg = (int)(__ldg(hv.soff + q + 1) - r.base);
    } else if (h >= 0) {
        r.heavy = 1;
        r.base = __ldg(hv.hpref + h) * co.W + (long long)word * r.deg;
        r.vdeg = __ldg(hv.hcnt + (long long)h * co.W + word);
    } else {
        r.heavy = 0;
        r.base = beg;
        r.vdeg = r.deg;
    }
    return r;
}

// Live state carried from x to the element's neighbour y.
template <int DIR, int MODEL, int SLICE>
__device__ __forceinline__ uint64_t elem(const GraphView &g, const Coins &co, long long base, int heavy,
                                         uint32_t rtm1, int j, uint64_t F, uint32_t rs, int &y, uint64_t live = 0)
{
    const HeavyView &hv = DIR == DIR_FWD ? g.hout : g.hin;
    if (SLICE == SLICE_TGT && DIR == DIR_REV && heavy == 2) {
        y = __ldg(hv.snbr + base + j);
        return F;
    }
    if (DIR == DIR_FWD && SLICE == SLICE_SNAP && heavy == 3) {
        // one snapshot's live out-arcs; F is that snapshot's bit
        y = __ldg(g.fsnbr + base + j);
        return F;
    }
    if (DIR == DIR_FWD && SLICE == SLICE_SNAP && heavy == 4) {
        // one-arc lists: element j is the j-th state bit b, whose arc is the
        // list of rank popc(live below b) from the word's list base
        const int b = nth_bit(F, j);
        y = __ldg(g.fsnbr + base + __popcll(live & ((1ull << b) - 1ull)));
        return 1ull << b;
    }
    const unsigned long long *lm = DIR == DIR_FWD ? g.lm_out : g.lm_in;
    if (!heavy && lm) {
        // cached live bits of the arc at this CSR / CSC position
        const long long q = base + j;
        y = DIR == DIR_FWD ? __ldg(g.col + q) : __ldg(&g.cin[q].x);
        const uint64_t mk = __ldg(lm + (long long)((int)(rs >> 6) - g.lm_w0) * g.m + q);
        if (SLICE == SLICE_SNAP) return mk & F;
        return ((mk >> (rs & 63u)) & 1ull) ? F : 0ull;
    }
    if (heavy) {
        const long long q = base + j;
        y = __ldg(hv.hnbr + q);
        const uint64_t mk = __ldg(hv.hmask + q);
        if (SLICE == SLICE_SNAP) return mk & F;
        return ((mk >> (rs & 63u)) & 1ull) ? F : 0ull;
    }
    uint32_t eid, tm1;
    arc_at<DIR, MODEL>(g, (int)(base + j), rtm1, y, eid, tm1);
    if (SLICE == SLICE_SNAP) return live_bits(co, eid, rs, F, tm1);
    if (co.none_live) return 0ull;
    return coin_hi32(co.seed ^ (uint64_t)eid, rs) <= tm1 ? F : 0ull;
}

// Snapshot-sliced forward rows with per-snapshot lists (the caller has
// checked that the lists are valid).  State bits whose snapshot has no live
// out-arc at x need no expansion and are dropped from F.  A row whose
// nonempty lists in this word hold one arc each expands one element per
// remaining bit (heavy 4).  Otherwise a state of at most SPARSE_BITS bits
// takes its lowest bit through that snapshot's list (heavy 3) and the other
// bits are returned for the caller to put back to pending; larger states
// keep the index.  Returns the bits put back (0 when none).
template <int DIR, int SLICE>
__device__ __forceinline__ uint64_t pick_rows(const GraphView &g, const Coins &co, int x, int word, uint64_t &F,
                                              Row &rr)
{
    if (DIR != DIR_FWD || SLICE != SLICE_SNAP || !g.fsoff || !F || rr.heavy != 1) return 0;
    F &= rr.live;
    if (!F) return 0;
    if (rr.single) {
        rr.base = rr.lbase;
        rr.vdeg = __popcll(F);
        rr.heavy = 4;
        return 0;
    }
    if (__popcll(F) > SPARSE_BITS) return 0;
    const int b = __ffsll((long long)F) - 1;
    const long long q = (long long)x * (64 * co.W) + 64 * word + b;
    const long long o0 = __ldg(g.fsoff + q), o1 = __ldg(g.fsoff + q + 1);
    const uint64_t rest = F & (F - 1);
    F = 1ull << b;
    rr.base = o0;
    rr.vdeg = (int)(o1 - o0);
    rr.heavy = 3;
    return rest;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// largest i in [0, count) with off[i] <= t (off non-decreasing, off[0] <= t)
__device__ __forceinline__ int find_off(const long long *off, int count, long long t)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct EngineArgs;

struct EngineArgs {
    GraphView g;
    Coins co;
    Ctl *ctl;
    long long *s;
    const int32_t *tl;      // per-snapshot target lists
    const long long *toff;  // [64W] list offsets
    const int32_t *tcnt;    // [64W] list lengths
    const long long *coff;  // [64W+1] chunk-task offsets
    int32_t *list1, *list2;
    const unsigned long long *anc;  // [W][n] ancestors of v*, per snapshot bit (this round)
    // landmarks x_0..x_{K-1} (initial gains), 8 words per (w, y) side by side:
    // bit b of lmk_rx[((w*n + y) << 3) + i] = y in R(G'_{64w+b}, x_i), bit b
    // of lmk_ux[...] = y reaches x_i in G'_{64w+b}; lmk_U / lmk_E [(r << K) + I]: the size of the
    // union over i in I of R(G'_r, x_i), and the out-degree sum over it
    int lmk_k;
    int lmk_x[MAX_LMK];
    const unsigned long long *lmk_rx;
    const unsigned long long *lmk_ux;
    const unsigned long long *lmk_any;  // [W][n]: OR over i of the lmk_rx words
    const int32_t *lmk_U;
    const unsigned long long *lmk_E;
    long long ntasks;       // TASK_INIT: n * W
    int limit;              // keys a warp table may hold before the task moves up a tier
    long long spin;         // polls a bounded wait makes before it gives up
    int bu_mode;            // level-synchronous walks: 0 top-down only, 1 switch by frontier size, 2 bottom-up after level 0
    int bu_div;             // mode 1: a level runs bottom-up when its frontier holds more than n / bu_div nodes
    int scc;                // initial gains: condense sources inside a landmark's strongly connected component
    int word_major;         // initial-gain task t: 1 -> (source t mod n, word t / n), 0 -> (t / W, t mod W)
    int t1_direct;          // a warp-tier overflow with this many frontier entries left skips tier 2 (0: never)
};


// Initial gains with landmarks x_i.  A task from v reaches x_i in snapshot
// r exactly when v does (v in U(G'_r, x_i), one reverse walk per landmark),
// and then R(G'_r, v) contains all of R(G'_r, x_i): the task starts with
// xbits[i] = those snapshots, is credited at the end with the size of the
// union of the reached landmarks' sets, and its bits of such snapshots need
// not travel inside those sets (every node reached through a node of the
// union is in the union).  lmk_filter returns the bits of ml that still
// have to be recorded at y; xany = OR of xbits.  The seed's own bits inside
// the union are masked out at the end (lmk_effective).
__device__ __forceinline__ const unsigned long long *lmk_bits(const unsigned long long *base, const EngineArgs &a,
                                                              int word, int y)
{
    return base + (((size_t)word * (size_t)a.g.n + (size_t)y) << 3);
}

// PRE: first test the union word lmk_any (8 bytes) and read the eight
// per-landmark words only where y lies in some landmark's set in a snapshot
// the task credits.  It pays in the shared-memory tiers; in the dense tier,
// whose arrivals mostly need the per-landmark words anyway, the extra
// dependent load made the launch slower (269.0 against 263.4 ms on R-MAT
// 20, while the block-shared tier went from 9.7 to 5.1 ms).
template <bool PRE>
__device__ __forceinline__ uint64_t lmk_filter(const EngineArgs &a, int word, int y, uint64_t ml,
                                               const unsigned long long *xbits, uint64_t xany)
{
    if (!(ml & xany)) return ml;
    if (PRE && !(ml & xany & __ldg(a.lmk_any + (size_t)word * (size_t)a.g.n + (size_t)y))) return ml;
    const unsigned long long *p = lmk_bits(a.lmk_rx, a, word, y);
    uint64_t drop = 0;
#pragma unroll
    for (int i = 0; i < MAX_LMK; ++i) {
        if (i >= a.lmk_k) break;
        const uint64_t xb = xbits[i];
        if (xb & ml) drop |= __ldg(p + i) & xb;
    }
    return ml & ~drop;
}

// Snapshots of word `word` in which node v reaches landmark i.
__device__ __forceinline__ uint64_t lmk_reaches(const EngineArgs &a, int word, int v, int i)
{
    return __ldg(lmk_bits(a.lmk_ux, a, word, v) + i);
}

// State bits of a finished initial-gain task that count at u: those not
// credited through a landmark.
__device__ __forceinline__ uint64_t lmk_effective(const EngineArgs &a, int word, int u, uint64_t vis,
                                                  const uint64_t *xb)
{
    uint64_t drop = 0;
#pragma unroll
    for (int i = 0; i < MAX_LMK; ++i) {
        if (i >= a.lmk_k) break;
        if (xb[i]) drop |= __ldg(lmk_bits(a.lmk_rx, a, word, u) + i) & xb[i];
    }
    return vis & ~drop;
}

// For every snapshot some landmark was reached in: the size of the union of
// the reached landmarks' sets, and its out-degree sum.
__device__ __forceinline__ void lmk_totals(const EngineArgs &a, int word, const uint64_t *xb, long long &cnt,
                                           unsigned long long &edges)
{
    uint64_t any = 0;
#pragma unroll
    for (int i = 0; i < MAX_LMK; ++i)
        if (i < a.lmk_k) any |= xb[i];
    while (any) {
        const int b = __ffsll((long long)any) - 1;
        any &= any - 1;
        int I = 0;
#pragma unroll
        for (int i = 0; i < MAX_LMK; ++i)
            if (i < a.lmk_k) I |= (int)((xb[i] >> b) & 1ull) << i;
        const long long q = ((long long)(64 * word + b) << a.lmk_k) + I;
        cnt += a.lmk_U[q];
        edges += a.lmk_E[q];
    }
}

// Snapshot bits of word `word` in which source v lies in the strongly
// connected component of a landmark x_i (v in R(G'_r, x_i) and v reaches
// x_i: forward-backward from the landmark as pivot, exact).  There
// R(G'_r, v) = R(G'_r, x_i), which the landmark credit already counts, so
// the source's walk for those snapshots is skipped (condensation); without
// the switch the walk runs and every arrival is filtered out.
__device__ __forceinline__ uint64_t lmk_scc_bits(const EngineArgs &a, int word, int v)
{
    if (!a.scc) return 0;
    const unsigned long long *rx = lmk_bits(a.lmk_rx, a, word, v), *ux = lmk_bits(a.lmk_ux, a, word, v);
    uint64_t m = 0;
#pragma unroll
    for (int i = 0; i < MAX_LMK; ++i) {
        if (i >= a.lmk_k) break;
        m |= __ldg(rx + i) & __ldg(ux + i);
    }
    return m;
}

// Source and word of initial-gain task t.  Word-major numbering runs all of
// one word's tasks before the next word's, so the tasks in flight share
// that word's row descriptors, lists and landmark records in L2.
__device__ __forceinline__ void init_task(const EngineArgs &a, long long t, int &x0, int &word)
{
    if (a.word_major) {
        word = (int)(t / a.g.n);
        x0 = (int)(t - (long long)word * a.g.n);
    } else {
        x0 = (int)(t / a.co.W);
        word = (int)(t - (long long)x0 * a.co.W);
    }
}

// ============================================================ warp engine

struct WTab {
    unsigned long long *vis, *pend;
    int *key;
    unsigned short *queue, *touched;
    int *ctr;                  // [0] queue tail, [1] keys, [2] overflow
    unsigned long long *xbits; // [MAX_LMK] snapshots in which the task reached each landmark
};

template <int LOGC>
__host__ __device__ constexpr size_t tab_bytes()
{
    return (size_t)(1 << LOGC) * 24 + 16 + 8 * MAX_LMK;
}

template <int LOGC>
__device__ __forceinline__ WTab tab_at(unsigned char *p)
{
    constexpr int C = 1 << LOGC;
    WTab t;
    t.vis = reinterpret_cast<unsigned long long *>(p);
    t.pend = t.vis + C;
    t.key = reinterpret_cast<int *>(t.pend + C);
    t.queue = reinterpret_cast<unsigned short *>(t.key + C);
    t.touched = t.queue + C;
    t.ctr = reinterpret_cast<int *>(t.touched + C);
    t.xbits = reinterpret_cast<unsigned long long *>(t.ctr + 4);
    return t;
}

template <int LOGC>
__device__ __forceinline__ uint32_t slot_of(int y)
{
    return ((uint32_t)y * 2654435761u) >> (32 - LOGC);
}

// Find y's slot, inserting it if absent.  Returns -1 (and flags overflow)
// once the table holds `limit` keys; at most 31 racing lanes can pass the
// check, so the touched list never exceeds limit + 31 < C entries.
template <int LOGC>
__device__ __forceinline__ int table_slot(const WTab &T, int y, int limit)
{
    constexpr int C = 1 << LOGC;
    uint32_t h = slot_of<LOGC>(y);
    volatile int *keys = T.key;
    for (int probe = 0; probe < C; ++probe) {
        const int k = keys[h];
        if (k == y) return (int)h;
        if (k == EMPTY_KEY) {
            if (*(volatile int *)&T.ctr[1] >= limit) {
                T.ctr[2] = 1;
                return -1;
            }
            const int old = atomicCAS(&T.key[h], EMPTY_KEY, y);
            if (old == EMPTY_KEY) {
                const int t = atomicAdd(&T.ctr[1], 1);
                T.touched[t] = (unsigned short)h;
                return (int)h;
            }
            if (old == y) return (int)h;
        }
        h = (h + 1) & (C - 1);
    }
    T.ctr[2] = 1;
    return -1;
}

// One task by one warp.  Returns 0 when it completed, else (nothing of the
// task applied; the table is clean again either way) 1 to move it to the
// block-shared tier, 2 straight to the dense tier.
template <int LOGC, int DIR, int MODEL, int TASK>
__device__ __forceinline__ int warp_task(const EngineArgs &a, const WTab &T, long long t, int lane,
                                          unsigned long long &edges_acc, unsigned long long &wk,
                                          unsigned long long &lel)
{
    constexpr int C = 1 << LOGC;
    const int LIMIT = a.limit;  // in [1, C/2]
    constexpr int SLICE = TASK == TASK_REVT ? SLICE_TGT : SLICE_SNAP;
    const GraphView &g = a.g;
    const Coins &co = a.co;
    int x0 = 0, word;
    uint32_t rs;
    if (TASK == TASK_INIT) {
        init_task(a, t, x0, word);
        rs = (uint32_t)word * 64u;
        int own = -1;
#pragma unroll
        for (int i = 0; i < MAX_LMK; ++i)
            if (i < a.lmk_k && x0 == a.lmk_x[i]) own = i;
        if (own >= 0) {  // a landmark's own task: its reach is known
            if (lane == 0) {
                uint64_t xb[MAX_LMK] = {};
                xb[own] = word_mask(word, co.R);
                long long c = 0;
                unsigned long long e = 0;
                lmk_totals(a, word, xb, c, e);
                atomicAdd((unsigned long long *)&a.s[x0], (unsigned long long)c);
                edges_acc += e;
            }
            return false;
        }
        if (lane < MAX_LMK)
            T.xbits[lane] = lane < a.lmk_k ? lmk_reaches(a, word, x0, lane) & word_mask(word, co.R) : 0ull;
        if (lane == 0) {
            const uint64_t M0 = word_mask(word, co.R) & ~lmk_scc_bits(a, word, x0);
            const uint32_t h = slot_of<LOGC>(x0);
            T.key[h] = x0;
            T.vis[h] = M0;
            T.pend[h] = M0;
            T.touched[0] = (unsigned short)h;
            T.queue[0] = (unsigned short)h;
            T.ctr[0] = 1;
            T.ctr[1] = 1;
        }
    } else {
        const int r = find_off(a.coff, 64 * co.W, t);
        const long long c = t - a.coff[r];
        word = r >> 6;
        rs = (uint32_t)r;
        const long long b0 = a.toff[r] + (long long)REV_GROUP * c;
        const int cnt = (int)min((long long)REV_GROUP, (long long)a.tcnt[r] - (long long)REV_GROUP * c);
        for (int j = lane; j < cnt; j += 32) {
            const int x = a.tl[b0 + j];
            const int h = table_slot<LOGC>(T, x, LIMIT);
            if (h < 0) continue;  // table full: the task moves up a tier
            T.vis[h] = 1ull << j;
            T.pend[h] = 1ull << j;
            const int pos = atomicAdd(&T.ctr[0], 1);
            T.queue[pos & (C - 1)] = (unsigned short)h;
        }
    }
    __syncwarp();
    uint64_t xany = 0;  // snapshots credited through some landmark (fixed for the task)
    if (TASK == TASK_INIT)
        for (int i = 0; i < a.lmk_k; ++i) xany |= T.xbits[i];
    const bool flists = TASK == TASK_INIT && g.fsoff && __ldg(g.fsvalid);
    unsigned long long tedges = 0;
    int qhead = 0, left = 0;
    while (true) {
        const int qtail = *(volatile int *)&T.ctr[0];
        const int ovf = *(volatile int *)&T.ctr[2];
        if (ovf || qhead >= qtail) {
            left = qtail - qhead;  // frontier entries not yet expanded (on overflow)
            break;
        }
        const int nb = min(32, qtail - qhead);
        long long base = 0;
        int vdeg = 0, heavy = 0;
        uint32_t rtm1 = 0;
        uint64_t F = 0, live = 0;
        if (lane < nb) {
            const int h = T.queue[(qhead + lane) & (C - 1)];
            const int x = T.key[h];
            F = T.pend[h];
            T.pend[h] = 0;
            const uint64_t Fp = F;
            uint64_t rest = 0;
            Row rr = row_ref<DIR, MODEL, SLICE>(g, co, x, word, rs);
            if (TASK == TASK_INIT && flists) {
                rest = pick_rows<DIR, SLICE>(g, co, x, word, F, rr);
                if (rest) {  // the other bits are expanded when x is popped again
                    T.pend[h] = rest;
                    T.queue[atomicAdd(&T.ctr[0], 1) & (C - 1)] = (unsigned short)h;
                }
                if (rr.heavy >= 3 && F) lel += (unsigned long long)rr.vdeg;
            }
            base = rr.base;
            vdeg = F ? rr.vdeg : 0;
            heavy = rr.heavy;
            rtm1 = rr.rtm1;
            live = rr.live;
            if (TASK == TASK_INIT) tedges += (unsigned long long)__popcll(Fp & ~rest) * (unsigned long long)rr.deg;
        }
        qhead += nb;
        __syncwarp();
        int incl = vdeg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - vdeg;
        if (lane == 1) wk += (unsigned long long)total;
        for (int abase = 0; abase < total; abase += 32) {
            const int j = abase + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = lo + step;
                const int ex = __shfl_sync(FULL, excl, cand & 31);
                if (cand < nb && ex <= j) lo = cand;
            }
            const long long ib = __shfl_sync(FULL, base, lo);
            const int iex = __shfl_sync(FULL, excl, lo);
            const int ih = __shfl_sync(FULL, heavy, lo);
            // forward rows share the uniform threshold; only initial gains
            // use one-arc lists
            const uint32_t itm1 = DIR == DIR_FWD ? co.uic_tm1 : __shfl_sync(FULL, rtm1, lo);
            const uint64_t iF = __shfl_sync(FULL, F, lo);
            const uint64_t ilive = TASK == TASK_INIT ? __shfl_sync(FULL, live, lo) : 0ull;
            if (j < total) {
                int y;
                uint64_t ml = elem<DIR, MODEL, SLICE>(g, co, ib, ih, itm1, j - iex, iF, rs, y, ilive);
                // nodes reaching v* in this snapshot were settled by the ancestor pass
                if (TASK == TASK_REVT && ml && ((__ldg(a.anc + (size_t)word * g.n + y) >> (rs & 63u)) & 1ull))
                    ml = 0;
                if (TASK == TASK_INIT) ml = lmk_filter<true>(a, word, y, ml, T.xbits, xany);
                if (ml) {
                    const int h = table_slot<LOGC>(T, y, LIMIT);
                    if (h >= 0) {
                        const uint64_t old = atomicOr(&T.vis[h], (unsigned long long)ml);
                        const uint64_t nw = ml & ~old;
                        if (nw) {
                            const uint64_t oldp = atomicOr(&T.pend[h], (unsigned long long)nw);
                            if (oldp == 0) {
                                const int pos = atomicAdd(&T.ctr[0], 1);
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
    const int ovf = *(volatile int *)&T.ctr[2];
    const int nt = *(volatile int *)&T.ctr[1];
    if (lane == 0) wk += (unsigned long long)nt;  // lane 0: keys, lane 1: elements
    uint64_t xb[MAX_LMK];
#pragma unroll
    for (int i = 0; i < MAX_LMK; ++i) xb[i] = (TASK == TASK_INIT && i < a.lmk_k) ? *(volatile unsigned long long *)&T.xbits[i] : 0ull;
    long long cnt = 0;
    unsigned long long redges = 0;
    for (int i = lane; i < nt; i += 32) {
        const int h = T.touched[i];
        if (!ovf) {
            const int u = T.key[h];
            if (TASK == TASK_INIT) {
                const uint64_t v = T.vis[h];
                if (u != x0) {
                    cnt += __popcll(v);  // arrivals passed the landmark filter
                } else {
                    // the source's seeded bits inside a credited landmark
                    // set are credited by the landmark instead
                    const uint64_t ve = lmk_effective(a, word, u, v, xb);
                    cnt += __popcll(ve);
                    if (ve != v)
                        tedges -= (unsigned long long)__popcll(v & ~ve) *
                                  (unsigned long long)(__ldg(g.rp + u + 1) - __ldg(g.rp + u));
                }
            } else {
                const int c = __popcll(T.vis[h]);
                atomicAdd((unsigned long long *)&a.s[u], (unsigned long long)(-(long long)c));
                redges += (unsigned long long)c * (unsigned long long)(__ldg(g.crp + u + 1) - __ldg(g.crp + u));
            }
        }
        T.key[h] = EMPTY_KEY;
        T.vis[h] = 0;
        T.pend[h] = 0;
    }
    if (TASK == TASK_INIT) {
        cnt = warp_sum(cnt);
        if (lane == 0 && !ovf) {
            unsigned long long e = 0;
            lmk_totals(a, word, xb, cnt, e);
            tedges += e;
        }
    }
    if (!ovf) edges_acc += TASK == TASK_INIT ? tedges : redges;
    __syncwarp();
    if (lane == 0) {
        if (!ovf && TASK == TASK_INIT) atomicAdd((unsigned long long *)&a.s[x0], (unsigned long long)cnt);
        T.ctr[0] = 0;
        T.ctr[1] = 0;
        T.ctr[2] = 0;
    }
    __syncwarp();
    if (!ovf) return 0;
    // a task that overflowed with a large frontier still to expand is sent
    // straight to the dense tier
    return (a.t1_direct > 0 && left >= a.t1_direct) ? 2 : 1;
}

// Tier 1: tasks [0, ntasks) by dynamic chunks, one warp per task with a
// shared-memory table; tasks that overflow it are listed for tier 2.
template <int LOGC, int DIR, int MODEL, int TASK>
__global__ void __launch_bounds__(WE_THREADS) warp_engine_kernel(EngineArgs a, int chunk)
{
    constexpr int C = 1 << LOGC;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const WTab T = tab_at<LOGC>(smem_raw + (size_t)wib * tab_bytes<LOGC>());
    for (int i = lane; i < C; i += 32) {
        T.key[i] = EMPTY_KEY;
        T.vis[i] = 0;
        T.pend[i] = 0;
    }
    if (lane == 0) {
        T.ctr[0] = 0;
        T.ctr[1] = 0;
        T.ctr[2] = 0;
    }
    __syncwarp();
    Ctl *ctl = a.ctl;
    const long long ntasks = TASK == TASK_INIT ? a.ntasks : *(volatile long long *)&ctl->du_total;
    unsigned long long edges = 0, wk = 0, lel = 0;
    while (true) {
        long long base = 0;
        if (lane == 0) base = (long long)atomicAdd(&ctl->t1_next, (unsigned long long)chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= ntasks) break;
        const long long tend = min(base + (long long)chunk, ntasks);
        for (long long t = base; t < tend; ++t) {
            const int ovf = warp_task<LOGC, DIR, MODEL, TASK>(a, T, t, lane, edges, wk, lel);
            if (ovf == 1 && lane == 0) a.list1[atomicAdd(&ctl->l1_count, 1ull)] = (int32_t)t;
            if (ovf == 2 && lane == 0) a.list2[atomicAdd(&ctl->l2_count, 1ull)] = (int32_t)t;
        }
    }
    edges = warp_sum(edges);
    if (lane == 0 && edges) atomicAdd(TASK == TASK_INIT ? &ctl->init_edges : &ctl->rev_edges, edges);
    if (TASK == TASK_INIT) {
        lel = warp_sum(lel);
        if (lane == 0 && lel) atomicAdd(&ctl->list_elems[0], lel);
    }
    if (lane < 2 && wk)
        atomicAdd(lane == 0 ? &ctl->work_keys[TASK == TASK_INIT ? 0 : 1][0] : &ctl->work_elems[TASK == TASK_INIT ? 0 : 1][0],
                  wk);
}

// ============================================================= CTA engine

constexpr int BT = 512;  // threads of the CTA engine
constexpr int BW = BT / 32;

struct CtaShared {
    unsigned long long F[BT];
    unsigned long long live[BT];
    long long base[BT];
    int ex[BT];
    int heavy[BT];
    uint32_t tm1[BT];
    int wsum[BW];
    int qlen, qnext, ntouch, ndu, total;
    long long red_ll[BW];
    unsigned long long red_ull[BW];
    int bcnt[64], boff[64], bcur[64];
};

// Block-wide exclusive scan of v; *total receives the sum.
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
        const int w = lane < BW ? S.wsum[lane] : 0;
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

struct CtaState {
    unsigned long long *vis;
    unsigned long long *pend;
    int32_t *qa;
    int32_t *qb;
    int32_t *touched;           // TASK_INIT / TASK_REVT / TASK_ANC
    unsigned long long *nbits;  // TASK_FWD / TASK_LMK
    int32_t *du_x;              // TASK_FWD / TASK_LMK: the word's list of nodes gaining bits
    int32_t *ndu;               // ... and its length (global, shared by the word's blocks)
    unsigned long long gm;      // snapshot bits this block owns (several blocks may share a word)
    long long *cnt_out;               // TASK_SPREAD: reached (node, snapshot) pairs are added here
    unsigned long long *edges_out;    // TASK_SPREAD: snapshot-edge count
    unsigned long long *fr = nullptr;  // bottom-up levels: the level's frontier bits per node (zero between
                                       // levels; shared by the word's blocks, bit-disjoint); NULL: top-down only
};

// Bottom-up level of a level-synchronous walk (direction-optimising BFS,
// Beamer, Asanovic and Patterson, SC 2012), bit-sliced: the frontier's state
// bits go into w.fr; then every node y still missing some of the block's
// snapshot bits scans its arcs from the walk's other side (in-arcs of a
// forward walk, out-arcs of a reverse walk) and takes
//     new(y) = OR over arcs e = (x, y) of (fr[x] & live(e)) & ~vis(y),
// stopping once no bit is missing.  The same set of (node, bit) pairs is
// reached as by a top-down level; the snapshot-edge counters count the
// frontier's expansions as a top-down level would.
template <int DIR, int MODEL, int TASK, size_t VS>
__device__ void bu_level(const EngineArgs &a, const CtaState &w, int word, uint32_t rs, int L, const int32_t *cur,
                         int32_t *nxt, long long &cnt, unsigned long long &edges, CtaShared &S)
{
    constexpr int BDIR = DIR == DIR_FWD ? DIR_REV : DIR_FWD;
    const GraphView &g = a.g;
    const Coins &co = a.co;
    const int tid = threadIdx.x;
    const unsigned long long *lm = BDIR == DIR_FWD ? g.lm_out : g.lm_in;
    for (int i = tid; i < L; i += BT) {
        const int x = cur[i];
        const uint64_t F = w.gm == ~0ull ? atomicExch(&w.pend[x], 0ull) : (atomicAnd(&w.pend[x], ~w.gm) & w.gm);
        if (!F) continue;
        atomicOr(&w.fr[x], (unsigned long long)F);
        if (TASK == TASK_FWD || TASK == TASK_SPREAD)
            edges += (unsigned long long)__popcll(F) * (unsigned long long)(__ldg(g.rp + x + 1) - __ldg(g.rp + x));
    }
    __syncthreads();
    const uint64_t wm = word_mask(word, co.R) & w.gm;
    for (long long yl = tid; yl < g.n; yl += BT) {
        const int y = (int)yl;
        uint64_t miss = ~*(volatile unsigned long long *)&w.vis[(size_t)y * VS] & wm;
        if (!miss) continue;
        const Row rr = row_ref<BDIR, MODEL, SLICE_SNAP>(g, co, y, word, rs);
        uint64_t acc = 0;
        for (int j = 0; j < rr.vdeg && miss; ++j) {
            const long long q = rr.base + j;
            int x;
            uint64_t mk = ~0ull;
            uint32_t eid = 0, tm1 = 0;
            bool hashed = false;
            if (rr.heavy) {
                const HeavyView &hv = BDIR == DIR_FWD ? g.hout : g.hin;
                x = __ldg(hv.hnbr + q);
                mk = __ldg(hv.hmask + q);
            } else if (lm) {
                x = BDIR == DIR_FWD ? __ldg(g.col + q) : __ldg(&g.cin[q].x);
                mk = __ldg(lm + (long long)((int)(rs >> 6) - g.lm_w0) * g.m + q);
            } else {
                arc_at<BDIR, MODEL>(g, (int)q, rr.rtm1, x, eid, tm1);
                hashed = true;
            }
            uint64_t f = *(volatile unsigned long long *)&w.fr[x] & miss & mk;
            if (!f) continue;
            if (hashed) f = live_bits(co, eid, rs, f, tm1);
            acc |= f;
            miss &= ~f;
        }
        if (!acc) continue;
        const uint64_t old = atomicOr(&w.vis[(size_t)y * VS], (unsigned long long)acc);
        const uint64_t nw = acc & ~old;
        if (!nw) continue;
        if (TASK == TASK_SPREAD) cnt += __popcll(nw);
        if (TASK == TASK_ANC && (old & w.gm) == 0) w.touched[atomicAdd(&S.ntouch, 1)] = y;
        if ((TASK == TASK_FWD || TASK == TASK_LMK) && w.du_x) {
            const uint64_t ob = atomicOr(&w.nbits[y], (unsigned long long)nw);
            if (ob == 0) w.du_x[atomicAdd(w.ndu, 1)] = y;
        }
        const uint64_t op = atomicOr(&w.pend[y], (unsigned long long)nw);
        if ((op & w.gm) == 0) nxt[atomicAdd(&S.qnext, 1)] = y;
    }
    __syncthreads();
    for (int i = tid; i < L; i += BT) {
        const int x = cur[i];
        if (w.gm == ~0ull) w.fr[x] = 0;
        else atomicAnd(&w.fr[x], ~w.gm);
    }
    __syncthreads();
}

// One traversal by the whole block over dense arrays, level-synchronous.
// TASK_INIT / TASK_REVT: vis/pend are a zeroed slot and are zero again on
// return.  TASK_FWD: vis is the word's coverage bitset; every node gaining
// bits is listed once, its merged new bits left in nbits.  TASK_ANC:
// reverse walk from v* over the snapshots where v* newly covers nodes; vis
// (the word's ancestor bits) is kept, and every ancestor u loses
// sum over its bits r of |N_r| (= ncov[r]) from its gain.
// TASK_SPREAD: multi-source walk from tgt[0..ntgt) with bits M0 over a
// zeroed vis; the reached (node, snapshot) pairs and their out-degrees are
// added to cnt_out / edges_out.
// Seeds: INIT, FWD, ANC: x0 with bits M0 (FWD: minus what is covered);
// REVT: the targets tgt[0..ntgt) with one bit each.
template <int DIR, int MODEL, int TASK>
__device__ void cta_bfs(const EngineArgs &a, CtaState w, int x0, uint64_t M0, int word, uint32_t rs,
                        const int32_t *tgt, int ntgt, const int *ncov, CtaShared &S)
{
    constexpr int SLICE = TASK == TASK_REVT ? SLICE_TGT : SLICE_SNAP;
    // landmark walks write one word of each node's 8-word landmark record
    constexpr size_t VS = TASK == TASK_LMK ? (size_t)MAX_LMK : 1;
    const GraphView &g = a.g;
    const Coins &co = a.co;
    const int tid = threadIdx.x;
    long long cnt = 0;
    if (tid == 0) {
        S.qlen = 0;
        S.qnext = 0;
        S.ntouch = 0;
        S.ndu = 0;
    }
    __syncthreads();
    if (TASK == TASK_REVT) {
        for (int j = tid; j < ntgt; j += BT) {
            const int x = tgt[j];
            w.vis[x] = 1ull << j;
            w.pend[x] = 1ull << j;
            w.qa[j] = x;
            w.touched[j] = x;
        }
        if (tid == 0) {
            S.qlen = ntgt;
            S.ntouch = ntgt;
        }
    } else if (TASK == TASK_SPREAD) {
        for (int j = tid; j < ntgt; j += BT) {
            const int x = tgt[j];
            const uint64_t M = M0 & ~atomicOr(&w.vis[x], (unsigned long long)M0);  // repeated sources count once
            if (M) {
                atomicOr(&w.pend[x], (unsigned long long)M);
                w.qa[atomicAdd(&S.qlen, 1)] = x;
                cnt += __popcll(M);
            }
        }
    } else if (tid == 0) {
        uint64_t M = M0;
        if (TASK == TASK_FWD || TASK == TASK_LMK) {
            M &= w.gm;
            M &= ~atomicOr(&w.vis[(size_t)x0 * VS], (unsigned long long)M);
            if (M) {
                atomicOr(&w.pend[x0], (unsigned long long)M);
                w.qa[0] = x0;
                S.qlen = 1;
                if (w.du_x && atomicOr(&w.nbits[x0], (unsigned long long)M) == 0) w.du_x[atomicAdd(w.ndu, 1)] = x0;
            }
        } else if (TASK == TASK_ANC) {
            // the word's groups walk their own bits of the shared words
            M &= w.gm;
            if (M) {
                atomicOr(&w.vis[x0], (unsigned long long)M);
                atomicOr(&w.pend[x0], (unsigned long long)M);
                w.qa[0] = x0;
                S.qlen = 1;
                w.touched[0] = x0;
                S.ntouch = 1;
            }
        } else if (M) {
            w.vis[x0] |= M;
            w.pend[x0] = M;
            w.qa[0] = x0;
            S.qlen = 1;
            {
                w.touched[0] = x0;
                S.ntouch = 1;
                if (TASK == TASK_INIT) cnt = __popcll(M);
            }
        }
    }
    unsigned long long edges = 0;
    int32_t *cur = w.qa, *nxt = w.qb;
    const bool flists = DIR == DIR_FWD && (TASK == TASK_FWD || TASK == TASK_LMK || TASK == TASK_SPREAD) && g.fsoff &&
                        __ldg(g.fsvalid);
    __syncthreads();
    int level = 0;
    while (true) {
        const int L = S.qlen;
        if (L == 0) break;
        // Direction-optimising step: once the frontier is a large part of
        // the graph, a level is cheaper pulled from the unreached side.
        constexpr bool CAN_BU = TASK == TASK_FWD || TASK == TASK_LMK || TASK == TASK_SPREAD || TASK == TASK_ANC;
        const bool bu = CAN_BU && w.fr && level > 0 &&
                        (a.bu_mode == 2 || (a.bu_mode == 1 && (long long)L * a.bu_div > (long long)g.n));
        ++level;
        if (bu) {
            bu_level<DIR, MODEL, TASK, VS>(a, w, word, rs, L, cur, nxt, cnt, edges, S);
            if (tid == 0) {
                S.qlen = S.qnext;
                S.qnext = 0;
            }
            int32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
            __syncthreads();
            continue;
        }
        for (int cbase = 0; cbase < L; cbase += BT) {
            const int i = cbase + tid;
            int vd = 0;
            if (i < L) {
                const int x = cur[i];
                uint64_t F = w.gm == ~0ull ? atomicExch(&w.pend[x], 0ull)
                                           : (atomicAnd(&w.pend[x], ~w.gm) & w.gm);
                const uint64_t Fp = F;
                uint64_t rest = 0;
                Row rr = row_ref<DIR, MODEL, SLICE>(g, co, x, word, rs);
                if (flists) {
                    // sparse state: one snapshot's live out-arcs now, the
                    // other bits at the next level (reachability only)
                    rest = pick_rows<DIR, SLICE>(g, co, x, word, F, rr);
                    if (rest && (atomicOr(&w.pend[x], (unsigned long long)rest) & w.gm) == 0ull)
                        nxt[atomicAdd(&S.qnext, 1)] = x;
                }
                vd = F ? rr.vdeg : 0;
                S.F[tid] = F;
                S.base[tid] = rr.base;
                S.heavy[tid] = rr.heavy;
                S.tm1[tid] = rr.rtm1;
                S.live[tid] = rr.live;
                if (TASK == TASK_INIT || TASK == TASK_FWD || TASK == TASK_SPREAD)
                    edges += (unsigned long long)__popcll(Fp & ~rest) * (unsigned long long)rr.deg;
            }
            int total;
            const int ex = block_excl_scan(vd, S, &total);
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
                    uint64_t ml = elem<DIR, MODEL, SLICE>(g, co, S.base[lo], S.heavy[lo], S.tm1[lo], j - S.ex[lo],
                                                          S.F[lo], rs, y, S.live[lo]);
                    if (TASK == TASK_REVT && ml && ((__ldg(a.anc + (size_t)word * g.n + y) >> (rs & 63u)) & 1ull))
                        ml = 0;
                    if (ml) {
                        const uint64_t old = atomicOr(&w.vis[(size_t)y * VS], (unsigned long long)ml);
                        const uint64_t nw = ml & ~old;
                        if (nw) {
                            if (TASK == TASK_INIT || TASK == TASK_SPREAD) cnt += __popcll(nw);
                            if (TASK != TASK_FWD && TASK != TASK_LMK && TASK != TASK_SPREAD && (old & w.gm) == 0)
                                w.touched[atomicAdd(&S.ntouch, 1)] = y;
                            if ((TASK == TASK_FWD || TASK == TASK_LMK) && w.du_x) {
                                const uint64_t ob = atomicOr(&w.nbits[y], (unsigned long long)nw);
                                if (ob == 0) w.du_x[atomicAdd(w.ndu, 1)] = y;
                            }
                            const uint64_t op = atomicOr(&w.pend[y], (unsigned long long)nw);
                            if ((op & w.gm) == 0) nxt[atomicAdd(&S.qnext, 1)] = y;
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
    if (TASK == TASK_INIT || TASK == TASK_REVT) {
        const int nt = S.ntouch;
        for (int i = tid; i < nt; i += BT) {
            const int y = w.touched[i];
            if (TASK == TASK_REVT) {
                const int c = __popcll(w.vis[y]);
                atomicAdd((unsigned long long *)&a.s[y], (unsigned long long)(-(long long)c));
                edges += (unsigned long long)c * (unsigned long long)(__ldg(g.crp + y + 1) - __ldg(g.crp + y));
            }
            w.vis[y] = 0;
        }
    } else if (TASK == TASK_ANC) {
        const int nt = S.ntouch;
        for (int i = tid; i < nt; i += BT) {
            const int y = w.touched[i];
            uint64_t b = w.vis[y] & w.gm;
            long long d = 0;
            while (b) {
                const int k = __ffsll((long long)b) - 1;
                b &= b - 1;
                d += ncov[k];
            }
            atomicAdd((unsigned long long *)&a.s[y], (unsigned long long)(-d));
            edges += (unsigned long long)d * (unsigned long long)(__ldg(g.crp + y + 1) - __ldg(g.crp + y));
        }
    }
    const unsigned long long e_tot = block_sum(edges, S.red_ull);
    if (TASK == TASK_INIT || TASK == TASK_SPREAD) {
        const long long c_tot = block_sum(cnt, S.red_ll);
        if (tid == 0 && c_tot)
            atomicAdd((unsigned long long *)(TASK == TASK_INIT ? &a.s[x0] : w.cnt_out), (unsigned long long)c_tot);
    }
    if (TASK == TASK_SPREAD) {
        if (tid == 0 && e_tot) atomicAdd(w.edges_out, e_tot);
    } else if (tid == 0 && e_tot) {
        unsigned long long *dst = TASK == TASK_INIT ? &a.ctl->init_edges
                                  : (TASK == TASK_FWD ? &a.ctl->fwd_edges : &a.ctl->rev_edges);
        atomicAdd(dst, e_tot);
    }
    __syncthreads();
}

struct SlotArgs {
    unsigned long long *vis, *pend;
    int32_t *qa, *touched;
    int qmask;  // tier-3 queue: per-slot ring of qmask+1 entries
};

// ===================================================== cooperative engine
//
// One block per task: its warps share one visited/pending table and one
// ring queue of frontier entries (block shapes below).  A warp claims up to 32
// queued entries at a time (CAS on the queue head), expands them with the
// same load-balanced arc split as the warp engine and pushes the nodes that
// gain new bits; there are no level barriers.  The traversal ends when the
// queue is empty and no warp holds claimed entries.  Every spin (waiting
// for work, waiting for a pushed entry to land) is bounded; on expiry the
// block records an error flag instead of waiting on.
//   TAB_HASH   hash table in shared memory (tier 2; a task that grows
//              past the key limit moves on to tier 3)
//   TAB_DENSE  dense per-block arrays in global memory indexed by node
//              (tier 3; never overflows)

// Block shapes.  Shared-memory tables take 24 bytes per slot: 2048-slot
// tables run in four 256-thread blocks per SM, 4096-slot tables in two
// 512-thread blocks.  Tasks are deep and narrow walks, so tasks in flight
// per SM set the throughput more than threads per task.  The dense tier
// (LOGC selects its shape: 0 initial gains, 1 reverse tasks) runs four
// 384-thread blocks per SM for initial gains and twelve 128-thread blocks
// for the smaller reverse tasks (40 registers either way): a reverse
// task's frontier rarely keeps more than four warps busy, so more tasks in
// flight pay (six 256-thread blocks: 26 ms more per R-MAT 20 select),
// while initial-gain tasks lose with fewer warps each.
constexpr int CO_LOGC = 12;  // the largest shared-memory table
constexpr unsigned short QE16 = 0xFFFF;
enum { TAB_HASH = 0, TAB_DENSE = 1 };
template <int TAB, int LOGC>
struct CoopShape {
    static constexpr int T = LOGC <= 11 ? 256 : (LOGC == 12 ? 512 : 1024);
    static constexpr int MINB = LOGC <= 11 ? 4 : (LOGC == 12 ? 2 : 1);
};
template <int LOGC>
struct CoopShape<TAB_DENSE, LOGC> {
    static constexpr int T = LOGC == 0 ? SG_DENSE_INIT_THREADS : SG_DENSE_REV_THREADS;
    static constexpr int MINB = LOGC == 0 ? SG_DENSE_INIT_BLOCKS : SG_DENSE_REV_BLOCKS;
    static constexpr int SQ = LOGC == 0 ? SG_DENSE_INIT_SQ : SG_DENSE_REV_SQ;  // shared-memory queue entries
};

struct CoopCtl {
    int head, tail, busy, nkeys, overflow, err;
    unsigned long long xbits[MAX_LMK];  // initial gains: snapshots in which the task reached each landmark
};

template <int TAB, int LOGC>
struct CoopTab;

template <int LOGC>
struct CoopTab<TAB_HASH, LOGC> {
    static constexpr int C = 1 << LOGC;
    unsigned long long *vis, *pend;
    int *key;
    unsigned short *queue, *touched;

    __device__ __forceinline__ static size_t bytes() { return (size_t)C * 24; }
    __device__ __forceinline__ unsigned long long &visr(int idx) { return vis[idx]; }
    __device__ __forceinline__ unsigned long long &pendr(int idx) { return pend[idx]; }
    __device__ __forceinline__ void bind(unsigned char *p)
    {
        vis = reinterpret_cast<unsigned long long *>(p);
        pend = vis + C;
        key = reinterpret_cast<int *>(pend + C);
        queue = reinterpret_cast<unsigned short *>(key + C);
        touched = queue + C;
    }
    // slot of y, inserting it; -1 (and overflow) past `limit` keys
    __device__ __forceinline__ int slot(int y, int limit, CoopCtl &c)
    {
        uint32_t h = ((uint32_t)y * 2654435761u) >> (32 - LOGC);
        volatile int *keys = key;
        for (int probe = 0; probe < C; ++probe) {
            const int k = keys[h];
            if (k == y) return (int)h;
            if (k == EMPTY_KEY) {
                if (*(volatile int *)&c.nkeys >= limit) {
                    c.overflow = 1;
                    return -1;
                }
                const int old = atomicCAS(&key[h], EMPTY_KEY, y);
                if (old == EMPTY_KEY) {
                    touched[atomicAdd(&c.nkeys, 1)] = (unsigned short)h;
                    return (int)h;
                }
                if (old == y) return (int)h;
            }
            h = (h + 1) & (C - 1);
        }
        c.overflow = 1;
        return -1;
    }
    __device__ __forceinline__ void note_new(int, CoopCtl &) {}
    __device__ __forceinline__ int node(int idx) const { return key[idx]; }
    __device__ __forceinline__ void put(int pos, int idx) { *(volatile unsigned short *)&queue[pos & (C - 1)] = (unsigned short)idx; }
    __device__ __forceinline__ int take(int pos, CoopCtl &c, long long spin)
    {
        volatile unsigned short *q = &queue[pos & (C - 1)];
        for (long long i = 0; i < spin; ++i) {
            const unsigned short v = *q;
            if (v != QE16) {
                *q = QE16;
                return v;
            }
            __nanosleep(32);
        }
        c.err = 1;
        return -1;
    }
    __device__ __forceinline__ void clear_slot(int idx)
    {
        key[idx] = EMPTY_KEY;
        vis[idx] = 0;
        pend[idx] = 0;
    }
    __device__ __forceinline__ int touched_at(int i) const { return touched[i]; }
    __device__ __forceinline__ void clear_queue(int, int)
    {
        for (int i = threadIdx.x; i < C; i += blockDim.x) queue[i] = QE16;
    }
};

template <int LOGC>
struct CoopTab<TAB_DENSE, LOGC> {
    // vis(y) and pend(y) share one 16-byte record: st[2y], st[2y + 1]
    unsigned long long *st;
    int *queue, *touched;
    int qmask;
    // queue positions below scap live in shared memory (sq), the rest in
    // the global ring: most tasks push fewer entries than scap, so their
    // producer-to-consumer hand-off stays on the SM
    int *sq;
    int scap;
    __device__ __forceinline__ volatile int *qref(int pos)
    {
        return pos < scap ? (volatile int *)&sq[pos] : (volatile int *)&queue[pos & qmask];
    }

    __device__ __forceinline__ unsigned long long &visr(int idx) { return st[2 * (size_t)idx]; }
    __device__ __forceinline__ unsigned long long &pendr(int idx) { return st[2 * (size_t)idx + 1]; }
    __device__ __forceinline__ int slot(int y, int, CoopCtl &) { return y; }
    __device__ __forceinline__ void note_new(int y, CoopCtl &c) { touched[atomicAdd(&c.nkeys, 1)] = y; }
    __device__ __forceinline__ int node(int idx) const { return idx; }
    __device__ __forceinline__ void put(int pos, int idx) { *qref(pos) = idx; }
    __device__ __forceinline__ int take(int pos, CoopCtl &c, long long spin)
    {
        volatile int *q = qref(pos);
        for (long long i = 0; i < spin; ++i) {
            const int v = *q;
            if (v != EMPTY_KEY) {
                *q = EMPTY_KEY;
                return v;
            }
            __nanosleep(32);
        }
        c.err = 1;
        return -1;
    }
    __device__ __forceinline__ void clear_slot(int idx)
    {
        visr(idx) = 0;
        pendr(idx) = 0;
    }
    __device__ __forceinline__ int touched_at(int i) const { return touched[i]; }
    __device__ __forceinline__ void clear_queue(int head, int tail)
    {
        for (int i = head + (int)threadIdx.x; i < tail; i += blockDim.x) *qref(i) = EMPTY_KEY;
    }
};

// Seed: entry `idx` carries bits M (vis and pend), queued.
template <int TAB, int LOGC>
__device__ __forceinline__ void coop_seed(CoopTab<TAB, LOGC> &T, CoopCtl &c, int y, uint64_t M, int limit)
{
    const int idx = T.slot(y, limit, c);
    if (idx < 0) return;
    if (TAB == TAB_DENSE) T.note_new(y, c);
    T.visr(idx) = M;
    T.pendr(idx) = M;
    T.put(atomicAdd(&c.tail, 1), idx);
}

// The block's warps expand the task's frontier until nothing is queued or
// claimed.
template <int TAB, int DIR, int MODEL, int TASK, int LOGC>
__device__ __forceinline__ unsigned long long coop_expand(const EngineArgs &a, CoopTab<TAB, LOGC> &T, CoopCtl &c, int word,
                                                          uint32_t rs, int limit, unsigned long long &elems,
                                                          unsigned long long &lel, long long &acnt)
{
    constexpr int SLICE = TASK == TASK_REVT ? SLICE_TGT : SLICE_SNAP;
    const GraphView &g = a.g;
    const Coins &co = a.co;
    const int lane = threadIdx.x & 31;
    unsigned long long tedges = 0;
    long long idle = 0;
    uint64_t xany = 0;  // snapshots credited through some landmark (fixed for the task)
    if (TASK == TASK_INIT)
        for (int i = 0; i < a.lmk_k; ++i) xany |= c.xbits[i];
    const bool flists = TASK == TASK_INIT && g.fsoff && __ldg(g.fsvalid);
    while (true) {
        int nb = 0, qb = 0;
        if (lane == 0) {
            // announce intent (busy) only when there is something to claim,
            // so that idle polling never hides quiescence from other warps
            if (*(volatile int *)&c.head < *(volatile int *)&c.tail && !*(volatile int *)&c.overflow) {
                atomicAdd(&c.busy, 1);
                __threadfence_block();
                int h = *(volatile int *)&c.head;
                while (true) {
                    const int t = *(volatile int *)&c.tail;
                    if (h >= t) break;
                    const int want = min(32, t - h);
                    const int old = atomicCAS(&c.head, h, h + want);
                    if (old == h) {
                        nb = want;
                        qb = h;
                        break;
                    }
                    h = old;
                }
                if (nb == 0) {
                    __threadfence_block();
                    atomicSub(&c.busy, 1);
                }
            }
        }
        nb = __shfl_sync(FULL, nb, 0);
        qb = __shfl_sync(FULL, qb, 0);
        if (nb == 0) {
            int done = 0;
            if (lane == 0) {
                const int h = *(volatile int *)&c.head;
                const int t = *(volatile int *)&c.tail;
                __threadfence_block();
                const int b = *(volatile int *)&c.busy;
                done = *(volatile int *)&c.overflow || *(volatile int *)&c.err || (h >= t && b == 0);
            }
            done = __shfl_sync(FULL, done, 0);
            if (done) break;
            if (++idle > a.spin) {
                if (lane == 0) c.err = 1;
                break;
            }
            // idle warps back off: 64 ns doubling up to SG_IDLE_NS_MAX (1 us)
            __nanosleep((unsigned)min((long long)SG_IDLE_NS_MAX, 64ll << min(idle - 1, 10ll)));
            continue;
        }
        idle = 0;
        long long base = 0;
        int vdeg = 0, heavy = 0;
        uint32_t rtm1 = 0;
        uint64_t F = 0, live = 0;
        if (lane < nb) {
            const int idx = T.take(qb + lane, c, a.spin);
            if (idx >= 0) {
                F = atomicExch(&T.pendr(idx), 0ull);
                Row rr = row_ref<DIR, MODEL, SLICE>(g, co, T.node(idx), word, rs);
                const uint64_t Fp = F;
                uint64_t rest = 0;
                if (TASK == TASK_INIT && flists) {
                    rest = pick_rows<DIR, SLICE>(g, co, T.node(idx), word, F, rr);
                    // the other bits go back to pending; re-queue unless an
                    // arrival already did
                    if (rest && atomicOr(&T.pendr(idx), (unsigned long long)rest) == 0ull)
                        T.put(atomicAdd(&c.tail, 1), idx);
                    if (rr.heavy >= 3 && F) lel += (unsigned long long)rr.vdeg;
                }
                base = rr.base;
                vdeg = F ? rr.vdeg : 0;
                heavy = rr.heavy;
                rtm1 = rr.rtm1;
                live = rr.live;
                if (TASK == TASK_INIT)
                    tedges += (unsigned long long)__popcll(Fp & ~rest) * (unsigned long long)rr.deg;
            }
        }
        // The arrival filters: ancestors already credited (reverse tasks),
        // landmark sets (initial gains).
        auto keep = [&](int y, uint64_t ml) -> uint64_t {
            if (TASK == TASK_REVT && ml && ((__ldg(a.anc + (size_t)word * g.n + y) >> (rs & 63u)) & 1ull))
                return 0ull;
            if (TASK == TASK_INIT) ml = lmk_filter<TAB == TAB_HASH>(a, word, y, ml, c.xbits, xany);
            return ml;
        };
        // After the visited-word atomic at idx returned old: record the new
        // bits, count them (initial gains count (node, snapshot) pairs as
        // they are first reached) and queue the node unless it is pending.
        auto settle = [&](int y, int idx, uint64_t ml, uint64_t old) {
            const uint64_t nw = ml & ~old;
            if (!nw) return;
            if (TASK == TASK_INIT) acnt += __popcll(nw);
            if (TAB == TAB_DENSE && old == 0) T.note_new(y, c);
            const uint64_t oldp = atomicOr(&T.pendr(idx), (unsigned long long)nw);
            if (oldp == 0) T.put(atomicAdd(&c.tail, 1), idx);
        };
        int incl = vdeg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - vdeg;
        if (lane == 0) elems += (unsigned long long)total;
        // Element j of the batch: its neighbour y and the state bits it
        // carries there (0 when j is past the end or nothing is live).
        // Warp-collective (shuffles): every lane calls it with its own j.
        auto fetch = [&](int j, int &y) -> uint64_t {
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = lo + step;
                const int ex = __shfl_sync(FULL, excl, cand & 31);
                if (cand < nb && ex <= j) lo = cand;
            }
            const long long ib = __shfl_sync(FULL, base, lo);
            const int iex = __shfl_sync(FULL, excl, lo);
            const int ih = __shfl_sync(FULL, heavy, lo);
            // forward rows share the uniform threshold; only initial gains
            // use one-arc lists
            const uint32_t itm1 = DIR == DIR_FWD ? co.uic_tm1 : __shfl_sync(FULL, rtm1, lo);
            const uint64_t iF = __shfl_sync(FULL, F, lo);
            const uint64_t ilive = TASK == TASK_INIT ? __shfl_sync(FULL, live, lo) : 0ull;
            y = 0;
            if (j >= total) return 0ull;
            return elem<DIR, MODEL, SLICE>(g, co, ib, ih, itm1, j - iex, iF, rs, y, ilive);
        };
        for (int abase = 0; abase < total; abase += 32) {
            int y;
            const uint64_t raw = fetch(abase + lane, y);
            const uint64_t ml = keep(y, raw);
            if (ml) {
                const int idx = T.slot(y, limit, c);
                if (idx >= 0) settle(y, idx, ml, atomicOr(&T.visr(idx), (unsigned long long)ml));
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicSub(&c.busy, 1);
        }
    }
    return tedges;
}

// The tasks of one stage: read from `in` (count *in_count, claimed through
// *next); a task that outgrows the table goes to `out` (count *out_count).
// stat: 1 counts the stage's tasks as tier-2 tasks, 2 as tier-3 tasks.
struct StageIO {
    const int32_t *in;
    unsigned long long *in_count;
    unsigned long long *next;
    int32_t *out;
    unsigned long long *out_count;
    int stat;
};

// Tier 2 (TAB_HASH, one stage per table size) and tier 3 (TAB_DENSE).
template <int TAB, int DIR, int MODEL, int TASK, int LOGC>
__global__ void __launch_bounds__(CoopShape<TAB, LOGC>::T, CoopShape<TAB, LOGC>::MINB)
    coop_engine_kernel(EngineArgs a, SlotArgs sl, StageIO io)
{
    constexpr int CO_T = CoopShape<TAB, LOGC>::T;
    constexpr int CO_W = CO_T / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CoopCtl c;
    __shared__ long long sh_t;
    __shared__ long long red_ll[CO_W];
    __shared__ unsigned long long red_ull[CO_W];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int wid = tid >> 5;
    const GraphView &g = a.g;
    Ctl *ctl = a.ctl;
    CoopTab<TAB, LOGC> T;
    int limit = 0x7fffffff;
    if constexpr (TAB == TAB_HASH) {
        T.bind(smem_raw);
        for (int i = tid; i < CoopTab<TAB_HASH, LOGC>::C; i += CO_T) {
            T.key[i] = EMPTY_KEY;
            T.vis[i] = 0;
            T.pend[i] = 0;
            T.queue[i] = QE16;
        }
        limit = a.limit;
    } else {
        const size_t so = (size_t)blockIdx.x * (size_t)g.n;
        T.st = sl.vis + 2 * so;
        T.touched = sl.touched + so;
        T.queue = sl.qa + (size_t)blockIdx.x * (size_t)(sl.qmask + 1);
        T.qmask = sl.qmask;
        T.sq = reinterpret_cast<int *>(smem_raw);
        T.scap = CoopShape<TAB, LOGC>::SQ;
        for (int i = tid; i < T.scap; i += CO_T) T.sq[i] = EMPTY_KEY;
    }
    const long long count = (long long)*(volatile unsigned long long *)io.in_count;
    unsigned long long *next = io.next;
    const int32_t *list = io.in;
    unsigned long long edges = 0, wk_keys = 0, wk_elems = 0, lel = 0;
    __syncthreads();
    while (true) {
        if (tid == 0) sh_t = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long k = sh_t;
        if (k >= count) break;
        const long long t = list[k];
        int x0 = 0, word;
        uint32_t rs;
        if (tid == 0) {
            c.head = 0;
            c.tail = 0;
            c.busy = 0;
            c.nkeys = 0;
            c.overflow = 0;
            c.err = 0;
        }
        __syncthreads();
        if (TASK == TASK_INIT) {
            init_task(a, t, x0, word);
            rs = (uint32_t)word * 64u;
            if (tid < MAX_LMK)
                c.xbits[tid] = tid < a.lmk_k ? lmk_reaches(a, word, x0, tid) & word_mask(word, a.co.R) : 0ull;
            if (tid == 0) coop_seed<TAB, LOGC>(T, c, x0, word_mask(word, a.co.R) & ~lmk_scc_bits(a, word, x0), limit);
        } else {
            const int r = find_off(a.coff, 64 * a.co.W, t);
            const long long ci = t - a.coff[r];
            word = r >> 6;
            rs = (uint32_t)r;
            const long long b0 = a.toff[r] + (long long)REV_GROUP * ci;
            const int cnt = (int)min((long long)REV_GROUP, (long long)a.tcnt[r] - (long long)REV_GROUP * ci);
            if (tid < cnt) coop_seed<TAB, LOGC>(T, c, a.tl[b0 + tid], 1ull << tid, limit);
        }
        __syncthreads();
        long long cnt = 0;
        unsigned long long tedges =
            coop_expand<TAB, DIR, MODEL, TASK, LOGC>(a, T, c, word, rs, limit, wk_elems, lel, cnt);
        __syncthreads();
        const int ovf = c.overflow | c.err;
        const int nt = c.nkeys;
        uint64_t xb[MAX_LMK];
#pragma unroll
        for (int i = 0; i < MAX_LMK; ++i) xb[i] = (TASK == TASK_INIT && i < a.lmk_k) ? c.xbits[i] : 0ull;
        if (TASK == TASK_INIT && tid == 0 && !ovf) {
            // Every bit recorded by an arrival passed the landmark filter and
            // was counted then; only the source's own seeded bits can lie in
            // a credited landmark set (x0 in R(G'_r, x_i) for a reached x_i):
            // those are credited by the landmark instead.
            const uint64_t M0 = word_mask(word, a.co.R) & ~lmk_scc_bits(a, word, x0);  // the seeded bits
            const uint64_t ve = lmk_effective(a, word, x0, M0, xb);
            cnt += __popcll(ve);
            if (ve != M0)
                tedges -= (unsigned long long)__popcll(M0 & ~ve) *
                          (unsigned long long)(__ldg(g.rp + x0 + 1) - __ldg(g.rp + x0));
        }
        unsigned long long redges = 0;
        for (int i = tid; i < nt; i += CO_T) {
            const int idx = T.touched_at(i);
            if (!ovf) {
                const int u = T.node(idx);
                if (TASK == TASK_INIT) {
                    // counted on arrival; the slot only needs clearing
                } else {
                    const int cc = __popcll(T.visr(idx));
                    atomicAdd((unsigned long long *)&a.s[u], (unsigned long long)(-(long long)cc));
                    redges += (unsigned long long)cc * (unsigned long long)(__ldg(g.crp + u + 1) - __ldg(g.crp + u));
                }
            }
            T.clear_slot(idx);
        }
        if (ovf) T.clear_queue(c.head, c.tail);
        if (!ovf) edges += (TASK == TASK_INIT ? tedges : 0) + redges;
        if (tid == 0) wk_keys += (unsigned long long)nt;
        if (TASK == TASK_INIT) {
            cnt = warp_sum(cnt);
            if (lane == 0) red_ll[wid] = cnt;
        }
        __syncthreads();
        if (tid == 0) {
            if (c.err) atomicOr(&ctl->flags, 2);
            if (ovf && !c.err) {
                if (io.out) io.out[atomicAdd(io.out_count, 1ull)] = (int32_t)t;
            } else if (!ovf && TASK == TASK_INIT) {
                long long tot = 0;
                for (int w = 0; w < CO_W; ++w) tot += red_ll[w];
                unsigned long long e = 0;
                lmk_totals(a, word, xb, tot, e);
                edges += e;
                atomicAdd((unsigned long long *)&a.s[x0], (unsigned long long)tot);
            }
        }
        __syncthreads();
    }
    edges = warp_sum(edges);
    wk_elems = warp_sum(wk_elems);
    if (TASK == TASK_INIT) {
        lel = warp_sum(lel);
        if (lane == 0 && lel) atomicAdd(&ctl->list_elems[TAB == TAB_HASH ? 1 : 2], lel);
    }
    if (lane == 0) red_ull[wid] = edges;
    if (lane == 0) red_ll[wid] = (long long)wk_elems;
    __syncthreads();
    if (tid == 0) {
        unsigned long long tot = 0, el = 0;
        for (int w = 0; w < CO_W; ++w) {
            tot += red_ull[w];
            el += (unsigned long long)red_ll[w];
        }
        const int tr = TAB == TAB_HASH ? 1 : 2;
        atomicAdd(&ctl->work_keys[TASK == TASK_INIT ? 0 : 1][tr], wk_keys);
        atomicAdd(&ctl->work_elems[TASK == TASK_INIT ? 0 : 1][tr], el);
        if (tot) atomicAdd(TASK == TASK_INIT ? &ctl->init_edges : &ctl->rev_edges, tot);
        if (blockIdx.x == 0) {
            if (io.stat == 1) {
                if (TASK == TASK_INIT) ctl->init_t2 += (unsigned long long)count;
                else ctl->rev_t2 += (unsigned long long)count;
            } else if (io.stat == 2) {
                if (TASK == TASK_INIT) ctl->init_t3 += (unsigned long long)count;
                else ctl->rev_t3 += (unsigned long long)count;
            }
        }
    }
}

size_t coop_hash_smem(int logc) { return (size_t)(1 << logc) * 24; }

// ========================================================== forward DU

struct FwdArgs {
    unsigned long long *cov, *nbits, *pendf, *anc;
    int32_t *fq_a, *fq_b, *du_x, *du_cnt, *tl, *anc_list, *anc_cnt;
    long long *toff, *coff;
    int32_t *tcnt;
    long long tcap;  // per-word capacity of tl
    int groups;      // blocks per word of the forward walk (8, 16, 32 or 64)
    unsigned long long *frw;  // [W][n] bottom-up frontier bits (zero between levels)
};

constexpr int FWD_GROUPS = 8;  // blocks per 64-snapshot word in the forward walk

// Forward DU, walk (Algorithm 2, inner loops): block (word, group) walks
// from v* over the live arcs of the 64/FWD_GROUPS snapshots it owns, with
// the word's coverage bitset as the visited set, so that N_r = R(G'_r, v*)
// minus what earlier seeds cover is marked in cov and nbits; every node of
// the word gaining bits is listed once.
template <int MODEL>
__global__ void __launch_bounds__(BT) fwd_walk_kernel(EngineArgs a, FwdArgs f)
{
    __shared__ CtaShared S;
    const int n = a.g.n;
    const int word = blockIdx.x / f.groups;
    const int grp = blockIdx.x - word * f.groups;
    const int vstar = *(volatile int32_t *)&a.ctl->vstar;
    if (vstar < 0) return;
    const int GB = 64 / f.groups;
    const size_t so = (size_t)word * (size_t)n;
    const size_t qo = (size_t)blockIdx.x * (size_t)n;
    CtaState w;
    w.vis = f.cov + so;
    w.pend = f.pendf + so;
    w.qa = f.fq_a + qo;
    w.qb = f.fq_b + qo;
    w.touched = nullptr;
    w.nbits = f.nbits + so;
    w.du_x = f.du_x + so;
    w.ndu = f.du_cnt + word;
    w.gm = (GB == 64 ? ~0ull : ((1ull << GB) - 1ull)) << (grp * GB);
    w.fr = f.frw ? f.frw + so : nullptr;
    cta_bfs<DIR_FWD, MODEL, TASK_FWD>(a, w, vstar, word_mask(word, a.co.R), word, (uint32_t)word * 64u, nullptr, 0,
                                      nullptr, S);
}

// Forward DU after the walk, in three launches:
//  fwd_anc_kernel    per (word, group) -- the walk's groups, 64/G snapshot
//                    bits each (bit-disjoint atomics on the shared words):
//                    clears the group's bits of the previous round's
//                    ancestor marks; |N_r| for its snapshots; then walks back
//                    from v* over live in-arcs: every u reaching v* in
//                    snapshot r reaches all of N_r (N_r lies inside
//                    R(G'_r, v*)), so s_u drops by |N_r| at once, and u is
//                    marked an ancestor;
//  fwd_lists_kernel  per (word, 8-bit group, slice of the word's new
//                    entries): per-snapshot lists of the remaining targets
//                    (N_r minus the ancestors), one fixed region of n
//                    entries per snapshot, for the target-sliced reverse
//                    tasks, which never enter a marked node (a path through
//                    one would make its start an ancestor); the last block
//                    turns the counts into the reverse tasks' offsets;
//  fwd_clear_kernel  clears the round's new-bit words.
constexpr int FPB = 64 / FWD_GROUPS;  // snapshot bits per list group
constexpr int LIST_SLICES = 4;       // blocks per (word, list group)

__device__ __forceinline__ uint64_t group_mask(int grp, int gb)
{
    return (gb == 64 ? ~0ull : ((1ull << gb) - 1ull)) << (grp * gb);
}

template <int MODEL>
__global__ void __launch_bounds__(BT) fwd_anc_kernel(EngineArgs a, FwdArgs f)
{
    __shared__ CtaShared S;
    const int n = a.g.n;
    const int word = blockIdx.x / f.groups;
    const int grp = blockIdx.x - word * f.groups;
    const int gb = 64 / f.groups;  // at most 8
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t gm = group_mask(grp, gb);
    const int vstar = *(volatile int32_t *)&a.ctl->vstar;
    const size_t so = (size_t)word * (size_t)n;
    unsigned long long *ancw = f.anc + so;
    int32_t *anclw = f.anc_list + (size_t)blockIdx.x * (size_t)n;
    {
        // this group's bits of the previous round's marks (other groups
        // clear theirs of the same words at the same time)
        const int na = f.anc_cnt[blockIdx.x];
        for (int i = tid; i < na; i += BT) atomicAnd(&ancw[anclw[i]], ~gm);
    }
    if (tid < 64) S.boff[tid] = 0;
    if (tid < gb) f.tcnt[64 * word + grp * gb + tid] = 0;  // the target lists' counters (fwd_lists_kernel)
    __syncthreads();
    const int nd = vstar >= 0 ? *(volatile int32_t *)&f.du_cnt[word] : 0;
    const int32_t *dux = f.du_x + so;
    const unsigned long long *nb = f.nbits + so;
    // |N_r| for the group's snapshots: ballots over 32 entries at a time
    int c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = 0;
    for (int base = (tid >> 5) * 32; base < nd; base += BT) {
        const int i = base + lane;
        const uint64_t M = i < nd ? (__ldg(nb + dux[i]) & gm) >> (grp * gb) : 0ull;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < gb) c[j] += __popc(__ballot_sync(FULL, (M >> j) & 1ull));
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < gb && c[j]) atomicAdd(&S.boff[grp * gb + j], c[j]);
    __syncthreads();
    const uint64_t mv = vstar >= 0 ? nb[vstar] & gm : 0ull;  // bits v* newly covers
    int nanc = 0;
    if (mv) {
        CtaState w;
        w.vis = ancw;
        w.pend = f.pendf + so;
        w.qa = f.fq_a + (size_t)blockIdx.x * (size_t)n;
        w.qb = f.fq_b + (size_t)blockIdx.x * (size_t)n;
        w.touched = anclw;
        w.nbits = nullptr;
        w.du_x = nullptr;
        w.ndu = nullptr;
        w.gm = gm;
        w.fr = f.frw ? f.frw + so : nullptr;
        cta_bfs<DIR_REV, MODEL, TASK_ANC>(a, w, vstar, mv, word, (uint32_t)word * 64u, nullptr, 0, S.boff, S);
        nanc = S.ntouch;
    }
    if (tid == 0) f.anc_cnt[blockIdx.x] = nanc;
}

__global__ void __launch_bounds__(BT) fwd_lists_kernel(FwdArgs f, Ctl *ctl, int n)
{
    __shared__ CtaShared S;
    __shared__ int sh_last;
    constexpr int PER_WORD = FWD_GROUPS * LIST_SLICES;
    const int word = blockIdx.x / PER_WORD;
    const int rem = blockIdx.x - word * PER_WORD;
    const int grp = rem / LIST_SLICES, slice = rem - grp * LIST_SLICES;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t gm = group_mask(grp, FPB);
    const int vstar = *(volatile int32_t *)&ctl->vstar;
    const size_t so = (size_t)word * (size_t)n;
    const int nd = vstar >= 0 ? *(volatile int32_t *)&f.du_cnt[word] : 0;
    const int32_t *dux = f.du_x + so;
    const unsigned long long *nb = f.nbits + so, *ancw = f.anc + so;
    int32_t *tlw = f.tl + (size_t)word * (size_t)f.tcap;
    int32_t *cnt = f.tcnt + 64 * word + grp * FPB;  // zeroed by fwd_anc_kernel
    const unsigned lt = (1u << lane) - 1u;
    // whole warps take 32 entries at a time (every lane joins the ballots);
    // the slices of one (word, group) share its counters
    for (int base = ((tid >> 5) + BW * slice) * 32; base < nd; base += BT * LIST_SLICES) {
        const int i = base + lane;
        int y = 0;
        uint64_t T = 0;
        if (i < nd) {
            y = dux[i];
            T = ((nb[y] & ~ancw[y]) & gm) >> (grp * FPB);
        }
#pragma unroll
        for (int j = 0; j < FPB; ++j) {
            const unsigned bal = __ballot_sync(FULL, (T >> j) & 1ull);
            if (!bal) continue;
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&cnt[j], __popc(bal));
            pos = __shfl_sync(FULL, pos, 0);
            if ((T >> j) & 1ull) tlw[(size_t)(grp * FPB + j) * (size_t)n + pos + __popc(bal & lt)] = y;
        }
    }
    if (slice == 0 && tid < FPB) {
        const int b = grp * FPB + tid;
        f.toff[64 * word + b] = (long long)word * f.tcap + (long long)b * n;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->fwd_arrivals, 1u);
        sh_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // last block: chunk-task offsets over every snapshot
    const int W = gridDim.x / PER_WORD;
    const int NS = 64 * W;
    long long carry = 0;
    for (int base = 0; base < NS; base += BT) {
        const int i = base + tid;
        const int v = i < NS ? (*(volatile int32_t *)&f.tcnt[i] + REV_GROUP - 1) / REV_GROUP : 0;
        int total;
        const int ex = block_excl_scan(v, S, &total);
        if (i < NS) f.coff[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    long long entries = 0;
    for (int i = tid; i < W; i += BT) entries += *(volatile int32_t *)&f.du_cnt[i];
    entries = block_sum(entries, S.red_ll);
    if (tid == 0) {
        f.coff[NS] = carry;
        ctl->du_total = carry;
        ctl->rev_tasks += (unsigned long long)carry;
        ctl->du_entries += (unsigned long long)entries;
        ctl->fwd_arrivals = 0;
    }
}

// The round's new-bit words back to zero (the next walk lists a node when
// its word goes from zero to nonzero).
__global__ void __launch_bounds__(256) fwd_clear_kernel(FwdArgs f, Ctl *ctl, int n, int W)
{
    if (*(volatile int32_t *)&ctl->vstar < 0) return;
    for (int word = 0; word < W; ++word) {
        const int nd = *(volatile int32_t *)&f.du_cnt[word];
        const size_t so = (size_t)word * (size_t)n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd;
             i += (long long)gridDim.x * blockDim.x)
            f.nbits[so + f.du_x[so + i]] = 0;
    }
}


// Landmark reach sets (initial gains).  landmark_walk_kernel: block
// (word, group) walks from landmark i over the live arcs (DIR_FWD) or the
// reversed live arcs (DIR_REV) of the snapshots it owns, into word i of
// every node's landmark record (zero on entry): R(G'_r, x_i) into rx,
// U(G'_r, x_i) into ux.
struct LmkArgs {
    unsigned long long *rx, *ux, *any, *pendf, *E, *HE;
    int32_t *fq_a, *fq_b, *U, *H;
    int groups;  // blocks per word (8, 16, 32 or 64)
    unsigned long long *frw;  // [W][n] bottom-up frontier bits (zero between levels)
};

template <int DIR, int MODEL>
__global__ void __launch_bounds__(BT) landmark_walk_kernel(EngineArgs a, LmkArgs l, int i)
{
    __shared__ CtaShared S;
    const int n = a.g.n;
    const int word = blockIdx.x / l.groups;
    const int grp = blockIdx.x - word * l.groups;
    const int GB = 64 / l.groups;
    const size_t qo = (size_t)blockIdx.x * (size_t)n;
    CtaState w;
    w.vis = (DIR == DIR_FWD ? l.rx : l.ux) + (((size_t)word * (size_t)n) << 3) + i;
    w.pend = l.pendf + (size_t)word * (size_t)n;
    w.qa = l.fq_a + qo;
    w.qb = l.fq_b + qo;
    w.touched = nullptr;
    w.nbits = nullptr;
    w.du_x = nullptr;
    w.ndu = nullptr;
    w.gm = (GB == 64 ? ~0ull : ((1ull << GB) - 1ull)) << (grp * GB);
    w.fr = l.frw ? l.frw + (size_t)word * (size_t)n : nullptr;
    // In a snapshot where x_i and an earlier landmark x_j reach each other
    // (one strongly connected component), R(x_i) = R(x_j) and U(x_i) =
    // U(x_j): copy those bits of word j instead of walking them.
    uint64_t M = word_mask(word, a.co.R) & w.gm;
    const unsigned long long *ri = l.rx + (((size_t)word * (size_t)n + (size_t)a.lmk_x[i]) << 3);
    const unsigned long long *ui = l.ux + (((size_t)word * (size_t)n + (size_t)a.lmk_x[i]) << 3);
    for (int j = 0; j < i && M; ++j) {
        const uint64_t same = M & ri[j] & ui[j];
        if (!same) continue;
        M &= ~same;
        unsigned long long *base = (DIR == DIR_FWD ? l.rx : l.ux) + (((size_t)word * (size_t)n) << 3);
        for (int y = threadIdx.x; y < n; y += BT) {
            const uint64_t v = base[((size_t)y << 3) + j] & same;
            if (v) atomicOr(&base[((size_t)y << 3) + i], (unsigned long long)v);
        }
    }
    cta_bfs<DIR, MODEL, TASK_LMK>(a, w, a.lmk_x[i], M, word, (uint32_t)word * 64u, nullptr,
                                      0, nullptr, S);
}

// Multi-source walk over the snapshots of words w0 .. w0 + gridDim.x /
// groups - 1: block b walks word w0 + b / groups, owning 64 / groups of its
// snapshot bits (the word's blocks share vis and pend, bit-disjoint), from
// every node of S.  vis holds the nodes to leave out (zero, or a copy of
// the coverage) and gains the reached bits; the newly reached (node,
// snapshot) pairs and their out-degree sum are added to total / edges.
struct SpreadArgs {
    unsigned long long *vis, *pend;  // [words][n]; pend zero on entry
    int32_t *qa, *qb;                // [words * groups][n]
    const int32_t *S;
    int ns;
    int w0;
    int groups;                      // 1, 2, 4 or 8
    long long *total;
    unsigned long long *edges;
    unsigned long long *fr;          // [words][n] bottom-up frontier bits, zero on entry (NULL: top-down only)
};

template <int MODEL>
__global__ void __launch_bounds__(BT) spread_kernel(EngineArgs a, SpreadArgs sp)
{
    __shared__ CtaShared S;
    const size_t n = (size_t)a.g.n;
    const int wi = blockIdx.x / sp.groups, grp = blockIdx.x - wi * sp.groups;
    const int word = sp.w0 + wi;
    const int gb = 64 / sp.groups;
    CtaState w;
    w.vis = sp.vis + (size_t)wi * n;
    w.pend = sp.pend + (size_t)wi * n;
    w.qa = sp.qa + blockIdx.x * n;
    w.qb = sp.qb + blockIdx.x * n;
    w.touched = nullptr;
    w.nbits = nullptr;
    w.du_x = nullptr;
    w.ndu = nullptr;
    w.gm = gb == 64 ? ~0ull : (((1ull << gb) - 1ull) << (grp * gb));
    w.cnt_out = sp.total;
    w.edges_out = sp.edges;
    w.fr = sp.fr ? sp.fr + (size_t)wi * n : nullptr;
    cta_bfs<DIR_FWD, MODEL, TASK_SPREAD>(a, w, -1, word_mask(word, a.co.R) & w.gm, word, (uint32_t)word * 64u, sp.S,
                                         sp.ns, nullptr, S);
}

// Histogram, per snapshot r, of the landmark-membership mask
// m_r(y) = {i : y in R(G'_r, x_i)} over the nodes with m_r(y) nonempty
// (count and out-degree sum), in H / HE [(r << K) + m]; any[w][y] = the
// OR of y's eight R(x_i) words.
__global__ void __launch_bounds__(256) landmark_hist_kernel(EngineArgs a, LmkArgs l)
{
    const int n = a.g.n, K = a.lmk_k, W = a.co.W;
    const long long total = (long long)W * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int word = (int)(t / n);
        const int y = (int)(t - (long long)word * n);
        uint64_t rx[MAX_LMK];
        uint64_t any = 0;
        const unsigned long long *rec = l.rx + (((size_t)word * (size_t)n + (size_t)y) << 3);
#pragma unroll
        for (int i = 0; i < MAX_LMK; ++i) {
            rx[i] = i < K ? rec[i] : 0ull;
            any |= rx[i];
        }
        l.any[t] = any;
        if (!any) continue;
        const unsigned long long d = (unsigned long long)(__ldg(a.g.rp + y + 1) - __ldg(a.g.rp + y));
        while (any) {
            const int b = __ffsll((long long)any) - 1;
            any &= any - 1;
            int m = 0;
#pragma unroll
            for (int i = 0; i < MAX_LMK; ++i) m |= (int)((rx[i] >> b) & 1ull) << i;
            const long long q = ((long long)(64 * word + b) << K) + m;
            atomicAdd(&l.H[q], 1);
            atomicAdd(&l.HE[q], d);
        }
    }
}

// Per snapshot (one block each, 2^K threads): subset sums over the
// histogram, Z[J] = sum over m within J of H[m]; the union of the sets of
// the landmarks in I holds every node whose mask meets I, i.e.
// U[I] = Z[all] - Z[all minus I].
__global__ void landmark_union_kernel(int K, LmkArgs l)
{
    __shared__ long long zc[1 << MAX_LMK];
    __shared__ unsigned long long ze[1 << MAX_LMK];
    const int r = blockIdx.x;
    const int S = 1 << K;
    const int J = threadIdx.x;
    const long long base = (long long)r << K;
    if (J < S) {
        zc[J] = l.H[base + J];
        ze[J] = l.HE[base + J];
    }
    __syncthreads();
    for (int i = 0; i < K; ++i) {
        long long c = 0;
        unsigned long long e = 0;
        const bool has = J < S && ((J >> i) & 1);
        if (has) {
            c = zc[J ^ (1 << i)];
            e = ze[J ^ (1 << i)];
        }
        __syncthreads();
        if (has) {
            zc[J] += c;
            ze[J] += e;
        }
        __syncthreads();
    }
    if (J < S) {
        const int all = S - 1;
        l.U[base + J] = (int32_t)(zc[all] - zc[all ^ J]);
        l.E[base + J] = ze[all] - ze[all ^ J];
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
                                                      int32_t *out_seeds, long long *out_gains, int round,
                                                      int32_t *du_cnt, int W)
{
    __shared__ long long sg[AM_T / 32];
    __shared__ int si[AM_T / 32];
    __shared__ int sh_last;
    long long bg = -1;
    int bi = -1;
    // 64-bit index: n may lie within one grid stride of 2^31
    for (long long v = (long long)blockIdx.x * AM_T + threadIdx.x; v < n; v += (long long)gridDim.x * AM_T) {
        const long long x = s[v];
        if (x > bg) {
            bg = x;
            bi = (int)v;
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
    for (int w = threadIdx.x; w < W; w += AM_T) du_cnt[w] = 0;
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
        ctl->t1_next = 0;
        ctl->l1_count = 0;
        ctl->l1_next = 0;
        ctl->l2_count = 0;
        ctl->l2_next = 0;
    }
}

// ======================================================== heavy live index

// The heavy live index, one lane per arc: warp k takes the 32 consecutive
// CSR (or CSC) positions 32k .. 32k + 31, whatever rows they fall in, and
// computes each arc's live mask for every word (64 coin hashes per arc and
// word).  A warp per row segment left most lanes idle on short rows: 36.9
// against 26.5 ms for both directions of the R-MAT 20 index.  Each lane
// finds its row by binary search on the row offsets; lanes of one row are
// grouped (match) and append their nonzero masks to the (row, word) segment
// with one atomic per group, so the order within a segment is arbitrary
// (every reader treats a segment as a set).  Arcs of light rows are
// skipped.  hcnt must be zero on entry.
template <int DIR, int MODEL>
__global__ void __launch_bounds__(256) heavy_index_kernel(GraphView g, Coins co, const int32_t *hid,
                                                               int32_t *hcnt, int32_t *hnbr,
                                                               unsigned long long *hmask, const long long *hpref)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t *rp = DIR == DIR_FWD ? g.rp : g.crp;
    const long long nck = (g.m + 31) / 32;
    const long long gw0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long ck = gw0; ck < nck; ck += nwarps) {
        const long long e = ck * 32 + lane;
        int x = -1, h = -1, deg = 0, y = 0;
        uint32_t eid = 0, tm1 = 0;
        if (e < g.m) {
            int lo = 0, hi = g.n;  // the row x with rp[x] <= e < rp[x + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if ((long long)__ldg(rp + mid) <= e) lo = mid;
                else hi = mid;
            }
            x = lo;
            h = __ldg(hid + x);
            if (h >= 0) {
                deg = __ldg(rp + x + 1) - __ldg(rp + x);
                const uint32_t rtm1 = (MODEL == MODEL_WIC && DIR == DIR_REV) ? __ldg(g.tmi + x) : co.uic_tm1;
                arc_at<DIR, MODEL>(g, (int)e, rtm1, y, eid, tm1);
            }
        }
        const unsigned grp = __match_any_sync(FULL, x);
        const long long hp = h >= 0 ? __ldg(hpref + h) * co.W : 0;
        for (int word = 0; word < co.W; ++word) {
            const uint64_t mk = h >= 0 ? live_bits(co, eid, (uint32_t)word * 64u, word_mask(word, co.R), tm1) : 0ull;
            const unsigned nz = __ballot_sync(FULL, mk != 0) & grp;
            const int first = nz ? __ffs(nz) - 1 : lane;
            int pos0 = 0;
            if (mk && lane == first) pos0 = atomicAdd(&hcnt[(long long)h * co.W + word], __popc(nz));
            pos0 = __shfl_sync(FULL, pos0, first);
            if (mk) {
                const long long q = hp + (long long)word * deg + pos0 + __popc(nz & lt);
                hnbr[q] = y;
                hmask[q] = mk;
            }
        }
    }
}

// ------------------------------------------- per-snapshot heavy in-lists
// From the per-word index of heavy in-rows: count the live in-arcs of every
// (heavy row, snapshot), scan, and fill.  mode 0 writes the counts into
// scnt, mode 1 fills snbr from the offsets soff (scnt unused).
// by_node 0: lists indexed by heavy-row ordinal h (q = h*64W + r), nq =
// nh*64W; by_node 1: indexed by the row's node (q = x*64W + r), nq = n*64W.
// rp holds the row offsets of the index's direction (for the degree).
__global__ void __launch_bounds__(256) snapshot_lists_kernel(Coins co, int nh, const int32_t *hcnt,
                                                             const int32_t *hnbr, const unsigned long long *hmask,
                                                             const long long *hpref, const int32_t *crp,
                                                             const int32_t *hrow, long long *scnt,
                                                             const long long *soff, int32_t *snbr,
                                                             long long cap, int32_t *svalid, int mode,
                                                             int by_node, long long nq)
{
    // One warp owns each (row, word) segment and so its 64 (row, snapshot)
    // lists: counts and ranks come from warp ballots, no atomics; lane l
    // keeps the counters (or cursors) of snapshot bits l and l + 32.
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long nseg = (long long)nh * co.W;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int R64 = 64 * co.W;
    for (long long sg = ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5); sg < nseg; sg += nwarps) {
        const int h = (int)(sg / co.W);
        const int w = (int)(sg - (long long)h * co.W);
        const int x = hrow[h];
        const int deg = crp[x + 1] - crp[x];
        const long long seg = hpref[h] * co.W + (long long)w * deg;
        const int cnt = hcnt[sg];
        const long long q0 = (long long)(by_node ? x : h) * R64 + 64 * w;  // list of snapshot 64w + b at q0 + b
        long long acc0 = 0, acc1 = 0;  // counts (mode 0) or list cursors (mode 1) of bits lane, lane + 32
        if (mode == 1) {
            acc0 = soff[q0 + lane];
            acc1 = soff[q0 + 32 + lane];
        }
        for (int j0 = 0; j0 < cnt; j0 += 32) {
            const int j = j0 + lane;
            const uint64_t M = j < cnt ? hmask[seg + j] : 0ull;
            const int y = j < cnt ? hnbr[seg + j] : 0;
#pragma unroll 4
            for (int b = 0; b < 64; ++b) {
                const bool has = (M >> b) & 1ull;
                const unsigned bal = __ballot_sync(FULL, has);
                if (!bal) continue;
                if (mode == 1) {
                    const long long cur = __shfl_sync(FULL, b < 32 ? acc0 : acc1, b & 31);
                    if (has) {
                        const long long pos = cur + __popc(bal & lt);
                        if (pos < cap) snbr[pos] = y;
                    }
                }
                if (lane == (b & 31)) {
                    if (b < 32) acc0 += __popc(bal);
                    else acc1 += __popc(bal);
                }
            }
        }
        if (mode == 0) {
            scnt[q0 + lane] = acc0;
            scnt[q0 + 32 + lane] = acc1;
        }
    }
    if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) *svalid = soff[nq] <= cap ? 1 : 0;
}

// Exclusive scan of int64 counts (in place into `out`), three phases.
constexpr int SC_T = 1024;
__global__ void __launch_bounds__(SC_T) scan_blocks_kernel(const long long *in, long long *out, long long n,
                                                           long long *sums)
{
    __shared__ long long sh[SC_T];
    const long long i = blockIdx.x * (long long)SC_T + threadIdx.x;
    const long long v = i < n ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SC_T; o <<= 1) {
        const long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == SC_T - 1) sums[blockIdx.x] = sh[SC_T - 1];
}

__global__ void __launch_bounds__(SC_T) scan_sums_kernel(long long *sums, long long nb, long long *total)
{
    __shared__ long long sh[SC_T];
    long long carry = 0;
    for (long long base = 0; base < nb; base += SC_T) {
        const long long i = base + threadIdx.x;
        const long long v = i < nb ? sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < SC_T; o <<= 1) {
            const long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
        const long long add = sh[SC_T - 1];
        __syncthreads();
        carry += add;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_add_kernel(long long *out, long long n, const long long *sums)
{
    const long long i = blockIdx.x * (long long)SC_T + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

// ============================================================== live masks

// cid (undirected variant, else null): the arc id each coin hashes.
__global__ void live_masks_kernel(Coins co, long long m, const uint2 *fw, uint32_t uic_tm1, int wic,
                                  const int32_t *cid, unsigned long long *out)
{
    const long long total = m * co.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / co.W;
        const int word = (int)(i - e * co.W);
        const uint32_t tm1 = wic ? fw[e].y : uic_tm1;
        const uint32_t id = cid ? (uint32_t)__ldg(cid + e) : (uint32_t)e;
        out[i] = live_bits(co, id, (uint32_t)word * 64u, word_mask(word, co.R), tm1);
    }
}

// ================================================== forward row descriptors

// One warp per (word, node).  With the forward lists, the word's 65 list
// offsets of an indexed row give its live mask (nonempty lists), its list
// base and whether every nonempty list holds one arc.
// Live-edge linear threshold coins (Kempe, Kleinberg and Tardos 2003, weights
// 1/indeg): node v's draw in snapshot r is coin_hi32(seed ^ v, r); its
// in-arcs, in CSC order (sources ascending), own consecutive intervals of
// width w_v = floor(2^32 / indeg(v)) = tmi[v] + 1, and the arc whose
// interval holds the draw is live in r (none when the draw is past d_v w_v).
// One thread per (node, word) of words [w0, w0 + words): it alone writes the
// masks of v's in-arcs for that word (zero on entry), so no atomics.
// Outputs (each may be NULL): lm_in / lm_out [word - w0][m] in CSC / CSR
// order, arc-major [e][aW] (sg_live_masks' layout).
__global__ void __launch_bounds__(256) lt_masks_kernel(Coins co, int n, long long m, int w0, int words,
                                                       const int32_t *crp, const int2 *cin, const uint32_t *tmi,
                                                       unsigned long long *lm_in, unsigned long long *lm_out,
                                                       unsigned long long *arc_major, int aW)
{
    const long long total = (long long)words * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int wi = (int)(t / n);
        const int v = (int)(t - (long long)wi * n);
        const int word = w0 + wi;
        const int beg = __ldg(crp + v), d = __ldg(crp + v + 1) - beg;
        if (d == 0) continue;
        const uint64_t w = (uint64_t)__ldg(tmi + v) + 1ull;
        const uint64_t base = co.seed ^ (uint64_t)(uint32_t)v;
        const uint64_t wm = word_mask(word, co.R);
        int cj = -1;
        uint64_t cm = 0;
        auto flush = [&]() {
            if (cj < 0) return;
            const long long q = beg + cj;
            const long long e = __ldg(&cin[q].y);
            if (lm_in) lm_in[(long long)wi * m + q] |= cm;
            if (lm_out) lm_out[(long long)wi * m + e] |= cm;
            if (arc_major) arc_major[e * aW + word] |= cm;
        };
        for (int b = 0; b < 64; ++b) {
            if (!((wm >> b) & 1ull)) break;
            const uint64_t j = (uint64_t)coin_hi32(base, (uint32_t)word * 64u + (uint32_t)b) / w;
            if (j >= (uint64_t)d) continue;
            if ((int)j != cj) {
                flush();
                cj = (int)j;
                cm = 0;
            }
            cm |= 1ull << b;
        }
        flush();
    }
}

__global__ void __launch_bounds__(256) row_desc_kernel(GraphView g, int W, const long long *fsoff, int4 *out)
{
    const int lane = threadIdx.x & 31;
    const long long total = (long long)W * g.n;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; i < total; i += nwarps) {
        const int word = (int)(i / g.n);
        const int x = (int)(i - (long long)word * g.n);
        const int beg = __ldg(g.rp + x), deg = __ldg(g.rp + x + 1) - beg;
        const int h = __ldg(g.hout.hid + x);
        long long base = beg;
        int vdeg = deg, heavy = 0;
        if (h >= 0) {
            base = __ldg(g.hout.hpref + h) * W + (long long)word * deg;
            vdeg = __ldg(g.hout.hcnt + (long long)h * W + word);
            heavy = 1;
        }
        unsigned long long live = ~0ull, lb = 0;
        int single = 0;
        if (h >= 0 && fsoff) {
            // offsets of lists 64x*W + 64w + b for b = 0..64 (the last is
            // the end of list 63)
            const long long *o = fsoff + (long long)x * 64 * W + 64LL * word;
            const long long a0 = __ldg(o + lane), a1 = __ldg(o + lane + 1);
            const long long b0 = __ldg(o + 32 + lane), b1 = __ldg(o + 33 + lane);
            const unsigned lo = __ballot_sync(FULL, a1 > a0), hi = __ballot_sync(FULL, b1 > b0);
            live = ((unsigned long long)hi << 32) | lo;
            const long long first = __shfl_sync(FULL, a0, 0), end = __shfl_sync(FULL, b1, 31);
            lb = (unsigned long long)first;
            single = (end - first == (long long)__popcll(live)) && first < (1LL << 62) ? 1 : 0;
        }
        if (lane == 0) {
            out[2 * i] = make_int4((int)(unsigned)(unsigned long long)base,
                                   (int)(unsigned)((unsigned long long)base >> 32), vdeg, deg | (heavy << 31));
            out[2 * i + 1] = make_int4((int)(unsigned)live, (int)(unsigned)(live >> 32), (int)(unsigned)lb,
                                       (int)((unsigned)(lb >> 32) | ((unsigned)single << 31)));
        }
    }
}

// ========================================================= live-mask cache

// lm_out[w*m + e] = live bits of arc e in the snapshots of word w.
template <int MODEL>
__global__ void __launch_bounds__(256) mask_cache_kernel(Coins co, long long m, const uint2 *fw,
                                                         unsigned long long *lm_out)
{
    const long long total = m * co.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int word = (int)(i / m);
        const long long e = i - (long long)word * m;
        const uint32_t tm1 = MODEL == MODEL_WIC ? __ldg(&fw[e].y) : co.uic_tm1;
        lm_out[i] = live_bits(co, (uint32_t)e, (uint32_t)word * 64u, word_mask(word, co.R), tm1);
    }
}

// lm_in[w*m + j] = lm_out[w*m + eid(j)] for CSC position j.
__global__ void __launch_bounds__(256) mask_cache_csc_kernel(int W, long long m, const int2 *cin,
                                                             const unsigned long long *lm_out,
                                                             unsigned long long *lm_in)
{
    const long long total = m * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int word = (int)(i / m);
        const long long j = i - (long long)word * m;
        lm_in[i] = __ldg(lm_out + (long long)word * m + __ldg(&cin[j].y));
    }
}

// ================================================================ launches

EngineArgs engine_args(sg_graph *g, sg_workspace &ws, const Coins &co, int heavy_on)
{
    EngineArgs a;
    a.g = view_of(g, ws, heavy_on);
    a.co = co;
    a.ctl = ws.ctl.p;
    a.s = ws.s.p;
    a.tl = ws.tl.p;
    a.toff = ws.toff.p;
    a.tcnt = ws.tcnt.p;
    a.coff = ws.coff.p;
    a.list1 = ws.list1.p;
    a.list2 = ws.list2.p;
    a.anc = ws.anc.p;
    a.lmk_k = 0;
    for (int i = 0; i < MAX_LMK; ++i) a.lmk_x[i] = -1;
    a.lmk_rx = ws.lmk_rx.p;
    a.lmk_ux = ws.lmk_ux.p;
    a.lmk_any = ws.lmk_any.p;
    a.lmk_U = ws.lmk_U.p;
    a.lmk_E = ws.lmk_E.p;
    a.ntasks = 0;
    a.limit = 1;
    a.spin = g_wait_polls;
    const Knobs kn = knobs();
    a.bu_mode = kn.bu_mode;
    a.bu_div = kn.bu_div;
    a.scc = kn.scc;
    a.word_major = kn.word_major;
    a.t1_direct = kn.t1_direct;
    return a;
}

SlotArgs slot_args(sg_workspace &ws)
{
    SlotArgs s;
    s.vis = ws.slot_vis.p;
    s.pend = nullptr;
    s.qa = ws.slot_qa.p;
    s.touched = ws.slot_touched.p;
    s.qmask = ws.slot_qmask;
    return s;
}

// tier 1 -> tier 2 -> tier 3 for one task family
// One shared-memory stage of tier 2: 2^LOGC-slot tables, blocks per SM
// from CoopShape.
template <int DIR, int MODEL, int TASK, int LOGC>
sg_status launch_stage(sg_graph *g, sg_workspace &ws, EngineArgs a, int limit, StageIO io, cudaStream_t st)
{
    a.limit = limit;
    auto kern = coop_engine_kernel<TAB_HASH, DIR, MODEL, TASK, LOGC>;
    const size_t smem = coop_hash_smem(LOGC);
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<g->num_sms * CoopShape<TAB_HASH, LOGC>::MINB, CoopShape<TAB_HASH, LOGC>::T, smem, st>>>(a, slot_args(ws), io);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

template <int DIR, int MODEL, int TASK>
sg_status launch_tiers(sg_graph *g, sg_workspace &ws, const EngineArgs &a0, cudaStream_t st, const TierEvents *ev)
{
    if (ev && ev->start) SG_CUDA_TRY(cudaEventRecord(ev->start, st));
    EngineArgs a = a0;
    {
        a.limit = std::max(1, std::min(knobs().t1_keys, (1 << T1_LOGC) / 2));
        auto kern = warp_engine_kernel<T1_LOGC, DIR, MODEL, TASK>;
        const size_t smem = (WE_THREADS / 32) * tab_bytes<T1_LOGC>();
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WE_THREADS, smem));
        if (per_sm < 1) per_sm = 1;
        kern<<<g->num_sms * per_sm, WE_THREADS, smem, st>>>(a, 8);
        SG_CUDA_TRY(cudaGetLastError());
        ++g_launches;
    }
    if (ev && ev->t1) SG_CUDA_TRY(cudaEventRecord(ev->t1, st));
    {
        // Tier 2: one shared-memory stage.  Initial-gain tasks run in
        // 2048-slot tables, four per SM (a 4096-slot second stage for their
        // 1-2 K-node tasks was slower than sending those to tier 3); so do
        // reverse tasks by default (4096-slot tables, two per SM, measured
        // 34 ms slower per select with the dense tier's reverse blocks).
        const int lim1 = std::max(1, std::min(knobs().t1_keys, (1 << T1_LOGC) / 2));
        const int t2 = std::max(1, std::min(knobs().t2_keys, (1 << CO_LOGC) / 2));
        Ctl *ctl = ws.ctl.p;
        const StageIO io{ws.list1.p, &ctl->l1_count, &ctl->l1_next, ws.list2.p, &ctl->l2_count, 1};
        if (TASK == TASK_INIT)
            SG_TRY((launch_stage<DIR, MODEL, TASK, 11>(g, ws, a, std::max(lim1, std::min(1 << 10, t2)), io, st)));
        else
            SG_TRY((launch_stage<DIR, MODEL, TASK, SG_REV_T2_LOGC>(
                g, ws, a, std::max(lim1, std::min((1 << SG_REV_T2_LOGC) / 2, t2)), io, st)));
    }
    if (ev && ev->t2) SG_CUDA_TRY(cudaEventRecord(ev->t2, st));
    {
        constexpr int DV = TASK == TASK_INIT ? 0 : 1;  // dense shape by task kind
        const int blocks = std::min(ws.nslots, g->num_sms * CoopShape<TAB_DENSE, DV>::MINB);
        constexpr size_t sqb = (size_t)CoopShape<TAB_DENSE, DV>::SQ * sizeof(int);
        if (sqb)
            SG_CUDA_TRY(cudaFuncSetAttribute(coop_engine_kernel<TAB_DENSE, DIR, MODEL, TASK, DV>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sqb));
        coop_engine_kernel<TAB_DENSE, DIR, MODEL, TASK, DV><<<blocks, CoopShape<TAB_DENSE, DV>::T, sqb, st>>>(
            a, slot_args(ws), StageIO{ws.list2.p, &ws.ctl.p->l2_count, &ws.ctl.p->l2_next, nullptr, nullptr, 2});
    }
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    if (ev && ev->t3) SG_CUDA_TRY(cudaEventRecord(ev->t3, st));
    return SG_OK;
}

template <int DIR, int MODEL>
sg_status launch_index(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    const bool fwd = DIR == DIR_FWD;
    const int nh = fwd ? g->nh_out : g->nh_in;
    if (nh == 0) return SG_OK;
    int32_t *hcnt = fwd ? ws.hcnt_out.p : ws.hcnt_in.p;
    SG_CUDA_TRY(cudaMemsetAsync(hcnt, 0, (size_t)nh * co.W * sizeof(int32_t), st));
heavy_index_kernel<DIR, MODEL><<<g->num_sms * 8, 256, 0, st>>>(
        view_of(g, ws, 1), co, fwd ? g->hid_out.p : g->hid_in.p, hcnt, fwd ? ws.hnbr_out.p : ws.hnbr_in.p,
        fwd ? ws.hmask_out.p : ws.hmask_in.p, fwd ? g->hpref_out.p : g->hpref_in.p);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

template <int MODEL>
sg_status init_gains_t(sg_graph *g, sg_workspace &ws, const Coins &co, int heavy_on, cudaStream_t st,
                       const TierEvents *ev)
{
    EngineArgs a = engine_args(g, ws, co, heavy_on);
    a.ntasks = (long long)g->n * co.W;
    const int K = std::min(std::min(knobs().landmarks, g->lmk_count), MAX_LMK);
    if (K > 0) {
        a.lmk_k = K;
        for (int i = 0; i < K; ++i) a.lmk_x[i] = g->lmk_nodes[i];
        const size_t nw = (size_t)g->n * co.W;
        SG_CUDA_TRY(cudaMemsetAsync(ws.lmk_rx.p, 0, nw * 8 * MAX_LMK, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.lmk_ux.p, 0, nw * 8 * MAX_LMK, st));
        LmkArgs l;
        l.rx = ws.lmk_rx.p;
        l.ux = ws.lmk_ux.p;
        l.any = ws.lmk_any.p;
        l.pendf = ws.pendf.p;
        l.fq_a = ws.fq_a.p;
        l.fq_b = ws.fq_b.p;
        l.U = ws.lmk_U.p;
        l.E = ws.lmk_E.p;
        l.H = ws.lmk_H.p;
        l.HE = ws.lmk_HE.p;
        l.groups = ws.walk_groups;
        l.frw = ws.frw.p;
        for (int i = 0; i < K; ++i) {
            landmark_walk_kernel<DIR_FWD, MODEL><<<co.W * l.groups, BT, 0, st>>>(a, l, i);
            SG_CUDA_TRY(cudaGetLastError());
            landmark_walk_kernel<DIR_REV, MODEL><<<co.W * l.groups, BT, 0, st>>>(a, l, i);
            SG_CUDA_TRY(cudaGetLastError());
        }
        const size_t nq = ((size_t)64 * co.W) << K;
        SG_CUDA_TRY(cudaMemsetAsync(ws.lmk_H.p, 0, nq * 4, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.lmk_HE.p, 0, nq * 8, st));
        const int blocks = (int)std::min<long long>(((long long)nw + 255) / 256, (long long)g->num_sms * 16);
        landmark_hist_kernel<<<blocks, 256, 0, st>>>(a, l);
        SG_CUDA_TRY(cudaGetLastError());
        landmark_union_kernel<<<64 * co.W, 1 << MAX_LMK, 0, st>>>(K, l);
        SG_CUDA_TRY(cudaGetLastError());
        g_launches += 2 * K + 2;
    }
    return launch_tiers<DIR_FWD, MODEL, TASK_INIT>(g, ws, a, st, ev);
}

sg_status launch_argmax(sg_graph *g, sg_workspace &ws, const Coins &co, int32_t round, cudaStream_t st)
{
    argmax_kernel<<<ws.am_blocks, AM_T, 0, st>>>(ws.s.p, (int)g->n, ws.ctl.p, ws.am_gain.p, ws.am_id.p,
                                                 ws.out_seeds.p, ws.out_gains.p, round, ws.du_cnt.p, co.W);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

template <int MODEL>
sg_status round_t(sg_graph *g, sg_workspace &ws, const Coins &co, int heavy_on, int32_t round, cudaStream_t st,
                  cudaEvent_t after_fwd)
{
    argmax_kernel<<<ws.am_blocks, AM_T, 0, st>>>(ws.s.p, (int)g->n, ws.ctl.p, ws.am_gain.p, ws.am_id.p,
                                                 ws.out_seeds.p, ws.out_gains.p, round, ws.du_cnt.p, co.W);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    EngineArgs a = engine_args(g, ws, co, heavy_on);
    FwdArgs f;
    f.cov = ws.cov.p;
    f.nbits = ws.nbits.p;
    f.pendf = ws.pendf.p;
    f.fq_a = ws.fq_a.p;
    f.fq_b = ws.fq_b.p;
    f.du_x = ws.du_x.p;
    f.du_cnt = ws.du_cnt.p;
    f.tl = ws.tl.p;
    f.toff = ws.toff.p;
    f.coff = ws.coff.p;
    f.tcnt = ws.tcnt.p;
    f.tcap = 64 * g->n;
    f.anc = ws.anc.p;
    f.anc_list = ws.anc_list.p;
    f.anc_cnt = ws.anc_cnt.p;
    f.groups = ws.walk_groups;
    f.frw = ws.frw.p;
    fwd_walk_kernel<MODEL><<<co.W * f.groups, BT, 0, st>>>(a, f);
    SG_CUDA_TRY(cudaGetLastError());
    fwd_anc_kernel<MODEL><<<co.W * f.groups, BT, 0, st>>>(a, f);
    SG_CUDA_TRY(cudaGetLastError());
    fwd_lists_kernel<<<co.W * FWD_GROUPS * LIST_SLICES, BT, 0, st>>>(f, ws.ctl.p, (int)g->n);
    SG_CUDA_TRY(cudaGetLastError());
    fwd_clear_kernel<<<g->num_sms * 2, 256, 0, st>>>(f, ws.ctl.p, (int)g->n, co.W);
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 4;
    if (after_fwd) SG_CUDA_TRY(cudaEventRecord(after_fwd, st));
    return launch_tiers<DIR_REV, MODEL, TASK_REVT>(g, ws, a, st, nullptr);
}

}  // namespace

thread_local int g_launches = 0;
long long g_wait_polls = WAIT_POLLS_DEFAULT;
int g_bu_mode = 1;
int g_bu_div = 4;
int g_scc = 1;
thread_local const Knobs *t_knobs = nullptr;
// tier-1 tables hand tasks on at 64 keys (of at most 256): measured on R-MAT
// 20, 64 keys 528.9 ms per select, 32 529.3, 128 534.5, 256 547.4
int g_tier_limit[2] = {64, (1 << CO_LOGC) / 2};
int g_landmarks = 8;

sg_status run_heavy_index(sg_graph *g, sg_workspace &ws, const Coins &co, int model, cudaStream_t st)
{
    if (model == MODEL_WIC) {
        SG_TRY((launch_index<DIR_FWD, MODEL_WIC>(g, ws, co, st)));
        return launch_index<DIR_REV, MODEL_WIC>(g, ws, co, st);
    }
    SG_TRY((launch_index<DIR_FWD, MODEL_UIC>(g, ws, co, st)));
    return launch_index<DIR_REV, MODEL_UIC>(g, ws, co, st);
}

sg_status run_lt_masks(sg_graph *g, const Coins &co, int w0, int words, unsigned long long *lm_in,
                       unsigned long long *lm_out, unsigned long long *arc_major, int aW, cudaStream_t st)
{
    const long long total = (long long)words * g->n;
    if (total == 0 || g->m == 0) return SG_OK;
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)g->num_sms * 16);
    lt_masks_kernel<<<blocks, 256, 0, st>>>(co, (int)g->n, g->m, w0, words, g->crp.p, g->cin.p, g->tmi.p, lm_in,
                                            lm_out, arc_major, aW);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

sg_status run_mask_cache(sg_graph *g, sg_workspace &ws, const Coins &co, int model, cudaStream_t st)
{
    const long long total = g->m * co.W;
    if (total == 0) return SG_OK;
    if (co.lt) {
        // per-node draws: every word's masks in both arc orders
        SG_CUDA_TRY(cudaMemsetAsync(ws.lm_in.p, 0, (size_t)total * 8, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.lm_out.p, 0, (size_t)total * 8, st));
        return run_lt_masks(g, co, 0, co.W, ws.lm_in.p, ws.lm_out.p, nullptr, 0, st);
    }
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)g->num_sms * 16);
    if (model == MODEL_WIC)
        mask_cache_kernel<MODEL_WIC><<<blocks, 256, 0, st>>>(co, g->m, g->fw.p, ws.lm_out.p);
    else
        mask_cache_kernel<MODEL_UIC><<<blocks, 256, 0, st>>>(co, g->m, g->fw.p, ws.lm_out.p);
    SG_CUDA_TRY(cudaGetLastError());
    mask_cache_csc_kernel<<<blocks, 256, 0, st>>>(co.W, g->m, g->cin.p, ws.lm_out.p, ws.lm_in.p);
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 2;
    return SG_OK;
}

sg_status run_row_desc(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    const long long total = g->n * co.W;
    const int blocks = (int)std::min<long long>((total * 32 + 255) / 256, (long long)g->num_sms * 16);
    GraphView v = view_of(g, ws, 1);
    v.rdesc = nullptr;
    row_desc_kernel<<<blocks, 256, 0, st>>>(v, co.W, ws.fl_on ? ws.fsoff.p : nullptr, ws.rdesc.p);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

sg_status run_spread(sg_graph *g, const Coins &co, int model, const int32_t *d_S, int32_t ns, long long *d_total,
                     unsigned long long *d_edges, cudaStream_t st)
{
    const size_t n = (size_t)g->n;
    // words per launch: dense vis/pend (8 B each) and two level queues (4 B
    // each) per node and word (LT: both orders of the chunk's live-mask
    // cache as well), within 8 GiB, split into launches of equal size (one
    // block per word: a short last launch would leave SMs idle).  The spread
    // walks stay top-down: they hash coins in registers, and a bottom-up
    // level would hash every in-arc of every node not yet reached (measured
    // on R-MAT 20, 20,000 snapshots: 7.97 s against 0.69 s top-down).
    const size_t per_word = n * 24 + (co.lt ? (size_t)g->m * 16 : 0);
    const int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)co.W, ((size_t)8 << 30) / per_word));
    const int nl = (co.W + cap - 1) / cap;
    const int wc = (co.W + nl - 1) / nl;
    DBuf<unsigned long long> vis, pend, lmc;
    DBuf<int32_t> qa, qb;
    sg_status rc = SG_OK;
    if (co.lt && (rc = dbuf_alloc(lmc, (size_t)wc * (size_t)g->m * 2, st)) != SG_OK) return rc;
    if ((rc = dbuf_alloc(vis, (size_t)wc * n, st)) != SG_OK || (rc = dbuf_alloc(pend, (size_t)wc * n, st)) != SG_OK ||
        (rc = dbuf_alloc(qa, (size_t)wc * n, st)) != SG_OK || (rc = dbuf_alloc(qb, (size_t)wc * n, st)) != SG_OK) {
        dbuf_free(vis, st);
        dbuf_free(pend, st);
        dbuf_free(qa, st);
        dbuf_free(qb, st);
        dbuf_free(lmc, st);
        return rc;
    }
    EngineArgs a{};
    a.spin = g_wait_polls;
    a.bu_mode = knobs().bu_mode;
    a.bu_div = knobs().bu_div;
    a.g = view_of(g, g->ws, 0);
    a.g.lm_out = nullptr;  // caches belong to another query's snapshots
    a.g.lm_in = nullptr;
    a.g.rdesc = nullptr;
    a.co = co;
    a.lmk_k = 0;
    for (int w0 = 0; w0 < co.W && rc == SG_OK; w0 += wc) {
        const int words = std::min(wc, co.W - w0);
        if (cudaMemsetAsync(vis.p, 0, (size_t)words * n * 8, st) != cudaSuccess ||
            cudaMemsetAsync(pend.p, 0, (size_t)words * n * 8, st) != cudaSuccess) {
            set_error("sg_spread: memset failed");
            rc = SG_ECUDA;
            break;
        }
        if (co.lt) {
            const size_t cm = (size_t)words * (size_t)g->m;
            if (cudaMemsetAsync(lmc.p, 0, cm * 16, st) != cudaSuccess) {
                set_error("sg_spread: memset failed");
                rc = SG_ECUDA;
                break;
            }
            if ((rc = run_lt_masks(g, co, w0, words, lmc.p + cm, lmc.p, nullptr, 0, st)) != SG_OK) break;
            a.g.lm_out = lmc.p;
            a.g.lm_in = lmc.p + cm;
            a.g.lm_w0 = w0;
        }
        SpreadArgs sp{vis.p, pend.p, qa.p, qb.p, d_S, ns, w0, 1, d_total, d_edges, nullptr};
        if (model == MODEL_WIC) spread_kernel<MODEL_WIC><<<words, BT, 0, st>>>(a, sp);
        else spread_kernel<MODEL_UIC><<<words, BT, 0, st>>>(a, sp);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("sg_spread: launch failed");
            rc = SG_ECUDA;
        }
        ++g_launches;
    }
    dbuf_free(vis, st);
    dbuf_free(pend, st);
    dbuf_free(qa, st);
    dbuf_free(qb, st);
    dbuf_free(lmc, st);
    return rc;
}

sg_status run_walk(sg_graph *g, const sg_workspace &ws, const Coins &co, int model, int heavy_on,
                   const int32_t *d_S, int32_t ns, unsigned long long *vis, unsigned long long *pend, int32_t *qa,
                   int32_t *qb, long long *d_total, unsigned long long *d_edges, cudaStream_t st)
{
    EngineArgs a{};
    a.spin = g_wait_polls;
    a.bu_mode = 0;  // the marginal-gain walks get no frontier array
    a.bu_div = 1;
    a.g = view_of(g, ws, heavy_on);
    a.co = co;
    a.lmk_k = 0;
    SpreadArgs sp{vis, pend, qa, qb, d_S, ns, 0, FWD_GROUPS, d_total, d_edges, nullptr};
    if (model == MODEL_WIC) spread_kernel<MODEL_WIC><<<co.W * FWD_GROUPS, BT, 0, st>>>(a, sp);
    else spread_kernel<MODEL_UIC><<<co.W * FWD_GROUPS, BT, 0, st>>>(a, sp);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

sg_status run_fwd_lists(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    const int nh = g->nh_out;
    const long long nq = g->n * 64LL * co.W;
    const long long n1 = nq + 1;
    const long long nb = (n1 + SC_T - 1) / SC_T;
    long long *cnt = ws.fscan.p, *sums = ws.fscan.p + n1;
    const int grid = g->num_sms * 8;
    SG_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)n1 * 8, st));
    snapshot_lists_kernel<<<grid, 256, 0, st>>>(co, nh, ws.hcnt_out.p, ws.hnbr_out.p, ws.hmask_out.p, g->hpref_out.p,
                                                g->rp.p, g->hrow_out.p, cnt, nullptr, nullptr, 0, nullptr, 0, 1, nq);
    SG_CUDA_TRY(cudaGetLastError());
    scan_blocks_kernel<<<(unsigned)nb, SC_T, 0, st>>>(cnt, ws.fsoff.p, n1, sums);
    scan_sums_kernel<<<1, SC_T, 0, st>>>(sums, nb, sums + nb);
    scan_add_kernel<<<(unsigned)nb, SC_T, 0, st>>>(ws.fsoff.p, n1, sums);
    SG_CUDA_TRY(cudaGetLastError());
    // the fill keeps its list cursors in registers (no counters to clear)
    snapshot_lists_kernel<<<grid, 256, 0, st>>>(co, nh, ws.hcnt_out.p, ws.hnbr_out.p, ws.hmask_out.p, g->hpref_out.p,
                                                g->rp.p, g->hrow_out.p, cnt, ws.fsoff.p, ws.fsnbr.p,
                                                (long long)ws.fsnbr_cap, ws.fsvalid.p, 1, 1, nq);
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 5;
    return SG_OK;
}

sg_status run_snapshot_lists(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st)
{
    const int nh = g->nh_in;
    const long long nq = (long long)nh * 64 * co.W;
    // counts
    SG_CUDA_TRY(cudaMemsetAsync(ws.scan_tmp.p, 0, (size_t)(nq + 1) * 8, st));
    const int grid = g->num_sms * 8;
    snapshot_lists_kernel<<<grid, 256, 0, st>>>(co, nh, ws.hcnt_in.p, ws.hnbr_in.p, ws.hmask_in.p, g->hpref_in.p,
                                                g->crp.p, g->hrow_in.p, ws.scan_tmp.p, nullptr, nullptr, 0, nullptr,
                                                0, 0, nq);
    SG_CUDA_TRY(cudaGetLastError());
    // offsets: soff[0..nq] = exclusive scan of counts (nq+1 entries, last = total)
    const long long n1 = nq + 1;
    const long long nb = (n1 + SC_T - 1) / SC_T;
    long long *sums = ws.scan_tmp.p + n1;
    scan_blocks_kernel<<<(unsigned)nb, SC_T, 0, st>>>(ws.scan_tmp.p, ws.soff.p, n1, sums);
    scan_sums_kernel<<<1, SC_T, 0, st>>>(sums, nb, sums + nb);
    scan_add_kernel<<<(unsigned)nb, SC_T, 0, st>>>(ws.soff.p, n1, sums);
    SG_CUDA_TRY(cudaGetLastError());
    // fill (list cursors in registers)
    snapshot_lists_kernel<<<grid, 256, 0, st>>>(co, nh, ws.hcnt_in.p, ws.hnbr_in.p, ws.hmask_in.p, g->hpref_in.p,
                                                g->crp.p, g->hrow_in.p, ws.scan_tmp.p, ws.soff.p, ws.snbr.p,
                                                (long long)ws.snbr_cap, ws.svalid.p, 1, 0, nq);
    SG_CUDA_TRY(cudaGetLastError());
    g_launches += 5;
    return SG_OK;
}

sg_status run_init_gains(sg_graph *g, sg_workspace &ws, const Coins &co, int model, int heavy_on, cudaStream_t st,
                         const TierEvents *ev)
{
    return model == MODEL_WIC ? init_gains_t<MODEL_WIC>(g, ws, co, heavy_on, st, ev)
                              : init_gains_t<MODEL_UIC>(g, ws, co, heavy_on, st, ev);
}

sg_status run_round(sg_graph *g, sg_workspace &ws, const Coins &co, int model, int heavy_on, int32_t round,
                    cudaStream_t st, cudaEvent_t after_fwd)
{
    return model == MODEL_WIC ? round_t<MODEL_WIC>(g, ws, co, heavy_on, round, st, after_fwd)
                              : round_t<MODEL_UIC>(g, ws, co, heavy_on, round, st, after_fwd);
}

sg_status run_argmax(sg_graph *g, sg_workspace &ws, const Coins &co, int32_t round, cudaStream_t st)
{
    return launch_argmax(g, ws, co, round, st);
}

sg_status run_live_masks(sg_graph *g, const Coins &co, int model, uint64_t *out, cudaStream_t st,
                         const int32_t *cid)
{
    const long long total = g->m * co.W;
    if (total == 0) return SG_OK;
    if (co.lt) {
        SG_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)total * 8, st));
        return run_lt_masks(g, co, 0, co.W, nullptr, nullptr, reinterpret_cast<unsigned long long *>(out), co.W, st);
    }
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)g->num_sms * 16);
    live_masks_kernel<<<blocks, 256, 0, st>>>(co, g->m, g->fw.p, co.uic_tm1, model == MODEL_WIC, cid,
                                              reinterpret_cast<unsigned long long *>(out));
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

}  // namespace sgi
