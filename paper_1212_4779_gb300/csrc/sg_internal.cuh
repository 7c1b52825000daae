// sg_internal.cuh -- shared declarations of the GB300 StaticGreedy-DU library.
//
// Device data layout (resident in HBM for the life of a graph handle):
//   rp   int32[n+1]  canonical CSR row offsets (arcs sorted by (src, dst))
//   col  int32[m]    CSR destinations; canonical arc id e = CSR position
//   fw   uint2[m]    WIC only: (dst, thr-1) per arc, interleaved so that one
//                    8-byte coalesced load gives both (built on first WIC use)
//   crp  int32[n+1]  CSC row offsets (in-arcs of each node)
//   cin  int2[m]     CSC entries (src, canonical arc id)
//   tmi  uint32[n]   WIC threshold-1 of every in-arc of the node
//                    (floor(2^32 / indeg) - 1; in-arcs of one node share it)
//   heavy rows (degree >= heavy threshold), per direction:
//     hid   int32[n]     ordinal of the node's heavy row, or -1
//     hrow  int32[nh]    node of each heavy row
//     hpref int64[nh+1]  prefix sum of heavy-row degrees
// Per-query state (workspace, reused across calls; zero between calls):
//   s     int64[n]        marginal gains (Algorithm 2's s_v)
//   cov   uint64[W][n]    coverage bitsets: bit b of cov[w][v] = v is
//                         reached from the seed set in snapshot 64w+b
//   nbits uint64[W][n]    bits newly covered in the current round
//   pendf uint64[W][n]    forward-DU frontier bits not yet expanded
//   du_x [W][n]           nodes gaining coverage bits this round, per word
//   tl    int32[W][64n]   newly covered nodes of the round, per snapshot,
//                         minus those that reach the round's seed
//   anc   uint64[W][n]    bit b: the node reaches the round's seed in snapshot 64w+b
//   lm_out / lm_in uint64[W][m]  optional live-mask cache: the live bits of
//                         every arc for each 64-snapshot word, in CSR and in
//                         CSC order (built once per query from the hash)
//   heavy live index, per direction: for heavy row h and word w the
//     nonzero 64-snapshot live masks of its arcs, compacted in arc order:
//     hcnt[h*W+w] entries at hnbr/hmask[hpref[h]*W + w*deg(h) ...]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sg.h"

// Dense (tier-3) engine block shapes: threads per block (the warps sharing
// one task) and resident blocks per SM, for initial-gain and for reverse
// tasks; the workspace holds slots for the larger count per SM.
#ifndef SG_DENSE_INIT_THREADS
#define SG_DENSE_INIT_THREADS 384
#endif
#ifndef SG_DENSE_INIT_BLOCKS
#define SG_DENSE_INIT_BLOCKS 4
#endif
#ifndef SG_DENSE_REV_THREADS
#define SG_DENSE_REV_THREADS 128
#endif
#ifndef SG_DENSE_REV_BLOCKS
#define SG_DENSE_REV_BLOCKS 12
#endif
#define SG_DENSE_BLOCKS (SG_DENSE_INIT_BLOCKS > SG_DENSE_REV_BLOCKS ? SG_DENSE_INIT_BLOCKS : SG_DENSE_REV_BLOCKS)
// Dense-engine queue entries held in shared memory per block (the first
// positions of each task's queue; the rest go to the global ring).  Initial
// gains: 4096 (16 KB; the R-MAT 20 dense launch 267.0 -> 260.7 ms, 8192:
// 261.2 ms); reverse tasks none (2048 made the selection rounds 5 ms
// slower: twelve blocks' carve-out leaves less L1 to a kernel whose
// scattered accesses keep the L1 data pipe the busiest unit).
#ifndef SG_DENSE_INIT_SQ
#define SG_DENSE_INIT_SQ 4096
#endif
#ifndef SG_DENSE_REV_SQ
#define SG_DENSE_REV_SQ 0
#endif
// log2 of the shared-memory table slots of the reverse tasks' block-shared
// tier (11: 2048-slot tables, four 256-thread blocks per SM, tasks past 1024
// keys go on to the dense tier; 12: 4096-slot tables, two 512-thread blocks)
#ifndef SG_REV_T2_LOGC
#define SG_REV_T2_LOGC 11
#endif
#ifndef SG_IDLE_NS_MAX
#define SG_IDLE_NS_MAX 1024
#endif


namespace sgi {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

#define SG_CUDA_TRY(call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            sgi::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                           __LINE__);                                                      \
            return SG_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

#define SG_TRY(expr)                      \
    do {                                  \
        sg_status s_ = (expr);            \
        if (s_ != SG_OK) return s_;       \
    } while (0)

// ------------------------------------------------------------------ memory
// nonzero: this thread allocates with cudaMallocAsync even when hooks are set
extern thread_local int g_builtin_alloc;
void *dalloc(size_t bytes, cudaStream_t st);
void dfree(void *p, size_t bytes, cudaStream_t st);

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t bytes = 0;
};

template <class T>
sg_status dbuf_alloc(DBuf<T> &b, size_t count, cudaStream_t st)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    b.p = static_cast<T *>(dalloc(bytes, st));
    if (!b.p) {
        set_error("device allocation of %zu bytes failed", bytes);
        return SG_ENOMEM;
    }
    b.bytes = bytes;
    return SG_OK;
}

template <class T>
void dbuf_free(DBuf<T> &b, cudaStream_t st)
{
    if (b.p) dfree(b.p, b.bytes, st);
    b.p = nullptr;
    b.bytes = 0;
}

// ----------------------------------------------------------- device views
enum Model { MODEL_UIC = 0, MODEL_WIC = 1 };

// Coin parameters of one query (hash-defined snapshots).
struct Coins {
    uint64_t seed;
    uint32_t uic_tm1;  // UIC: thr - 1 (thr = floor(p 2^32) >= 1)
    int32_t none_live; // UIC with thr = 0: no arc is ever live
    int32_t R;
    int32_t W;         // ceil(R / 64)
    int32_t lt;        // linear threshold model: coins come from the live-mask cache (per-node draws)
};

// High 32 bits of splitmix64(base ^ (r << 40)) (Steele, Lea, Flood 2014,
// with Stafford's Mix13 finaliser), base = seed ^ e: arc e is live in
// snapshot r iff this is at most thr(e) - 1 (Section 3.1's snapshot, with
// the coin drawn from a counter-based hash).
__device__ __forceinline__ uint32_t coin_hi32(uint64_t base, uint32_t r)
{
    uint64_t z = (base ^ ((uint64_t)r << 40)) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    const uint32_t hi = (uint32_t)(z >> 32);
    return hi ^ (hi >> 31);
}

// Heavy rows of one direction and the query's live index over them.
struct HeavyView {
    const int32_t *hid;
    const long long *hpref;
    const int32_t *hcnt;
    const int32_t *hnbr;
    const unsigned long long *hmask;
    // per-snapshot live lists (reverse direction only): the live in-arcs of
    // heavy row h in snapshot r are snbr[soff[h*64W + r] .. soff[h*64W + r + 1])
    const long long *soff;
    const int32_t *snbr;
    const int32_t *svalid;  // device flag: 1 if the lists were built completely
};

struct GraphView {
    int32_t n;
    int64_t m;
    const int32_t *rp;
    const int32_t *col;
    const uint2 *fw;
    const int32_t *crp;
    const int2 *cin;
    const uint32_t *tmi;
    HeavyView hout;  // heavy CSR rows (forward traversals)
    HeavyView hin;   // heavy CSC rows (reverse traversals)
    int32_t heavy_on;
    // live-mask cache (null when off): lm_out[w*m + e] = live bits of arc e
    // (CSR position) in snapshots 64w..64w+63; lm_in[w*m + j] the same for
    // the arc at CSC position j
    const unsigned long long *lm_out;
    const unsigned long long *lm_in;
    int32_t lm_w0;  // word of the cache's first block (a cache may hold a range of words)
    // forward row descriptors (null when the heavy-row index is off), two
    // int4 (one 32-byte sector) per (w, x):
    // rdesc[2(w*n + x)]     = {segment base (lo, hi), elements to expand for
    //                          word w, out-degree | (indexed << 31)}
    // rdesc[2(w*n + x) + 1] = {live (lo, hi), list base (lo, hi | single << 31)}
    // live: bit b set iff x has a live out-arc in snapshot 64w+b (all ones
    // without the forward lists); single: every nonempty list of the word
    // holds one arc, the lists of the word start at the list base
    const int4 *rdesc;
    // forward per-snapshot live lists (null when off): the live out-arcs of
    // node x in snapshot r are fsnbr[fsoff[x*64W + r] .. fsoff[x*64W + r + 1])
    // for every indexed row x; *fsvalid = 1 once built completely
    const long long *fsoff;
    const int32_t *fsnbr;
    const int32_t *fsvalid;
};

// Counters kept on the device during one call (zeroed at the start).
struct Ctl {
    unsigned long long init_edges;
    unsigned long long fwd_edges;
    unsigned long long rev_edges;
    unsigned long long init_t2, init_t3;  // initial-gain tasks run by tier 2 / tier 3
    unsigned long long rev_t2, rev_t3;    // reverse tasks run by tier 2 / tier 3
    unsigned long long du_entries;
    unsigned long long rev_tasks;         // target-sliced reverse tasks, all rounds
    unsigned long long work_keys[2][3];   // [init, reverse][tier]: nodes held in task tables
    unsigned long long work_elems[2][3];  // [init, reverse][tier]: arcs / index entries expanded
    unsigned long long list_elems[3];     // initial gains, per tier: of those, per-snapshot list entries
    unsigned long long t1_next;   // dynamic task counter, tier 1
    unsigned long long l1_count;  // tasks handed from tier 1 to tier 2
    unsigned long long l1_next;
    unsigned long long l2_count;  // tasks handed from tier 2 to tier 3
    unsigned long long l2_next;
    unsigned int argmax_arrivals;
    unsigned int fwd_arrivals;
    int32_t vstar;
    int32_t flags;
    long long du_total;   // reverse tasks of the current round
};

}  // namespace sgi

// Workspace owned by a graph handle and reused by every call on it.
struct sg_workspace {
    int64_t owner_n = -1;  // node count of the graph it was created for (explicit workspaces)
    int device = 0;
    int64_t n = 0;
    int32_t wcap = 0;     // words of capacity of the [W][n] arrays
    int32_t nslots = 0;   // tier-3 (CTA engine) slots
    int32_t fq_groups = 0;    // forward-walk blocks per word the queues fq_a/fq_b were sized for
    int32_t walk_groups = 8;  // forward/landmark walk blocks per word for the current query
    sgi::DBuf<long long> s;
    sgi::DBuf<unsigned long long> cov, nbits, pendf;
    sgi::DBuf<int32_t> fq_a, fq_b, du_x, list1, list2, tl;
    sgi::DBuf<long long> toff, coff;     // per snapshot: target list offset, chunk-task offset [64W+1]
    sgi::DBuf<int32_t> tcnt;             // per snapshot: newly covered count [64W]
    sgi::DBuf<int32_t> du_cnt;           // [W] entries per word
    sgi::DBuf<unsigned long long> anc;   // [W][n] ancestors of the round's seed, per snapshot bit
    sgi::DBuf<unsigned long long> frw;   // [W][n] bottom-up frontier bits of the walks (zero between levels)
    sgi::DBuf<int32_t> anc_list;         // [W][G][n] nodes given ancestor bits, per (word, walk group)
    sgi::DBuf<int32_t> anc_cnt;          // [W][G]
    sgi::DBuf<unsigned long long> lmk_rx;    // [W][n][8] landmark reach bits (R(x_i) membership)
    sgi::DBuf<unsigned long long> lmk_ux;    // [W][n][8] ... and which landmarks the node reaches
    sgi::DBuf<unsigned long long> lmk_any;   // [W][n] OR over the landmarks of the R(x_i) bits
    sgi::DBuf<int32_t> lmk_U, lmk_H;         // [64W << K] union sizes / membership histogram
    sgi::DBuf<unsigned long long> lmk_E, lmk_HE;  // ... their out-degree sums
    sgi::DBuf<unsigned long long> slot_vis;  // tier-3 slots: [slot][n][2] visited / pending words
    sgi::DBuf<int32_t> slot_qa, slot_touched;
    int32_t slot_qmask = 0;              // tier-3 per-slot queue: ring of slot_qmask+1 entries (in slot_qa)
    sgi::DBuf<sgi::Ctl> ctl;
    sgi::DBuf<long long> am_gain;        // argmax per-block partials
    sgi::DBuf<int32_t> am_id;
    sgi::DBuf<int32_t> out_seeds;
    sgi::DBuf<long long> out_gains;
    // heavy live index (per direction) for the current W
    sgi::DBuf<int32_t> hcnt_out, hnbr_out, hcnt_in, hnbr_in;
    sgi::DBuf<unsigned long long> hmask_out, hmask_in;
    int32_t hw_cap = 0;   // W the heavy index was sized for
    // per-snapshot live in-lists of heavy rows
    sgi::DBuf<long long> soff;
    sgi::DBuf<int32_t> snbr, svalid;
    sgi::DBuf<long long> scan_tmp;
    size_t soff_cap = 0, snbr_cap = 0;
    int32_t slists_on = 0;    // built for the current query
    sgi::DBuf<int4> rdesc;    // [W][n][2] forward row descriptors (with the heavy-row index)
    // forward per-snapshot live lists of indexed rows, node-indexed
    sgi::DBuf<long long> fsoff, fscan;
    sgi::DBuf<int32_t> fsnbr, fsvalid;
    size_t fsoff_cap = 0, fsnbr_cap = 0;
    int32_t fl_on = 0;        // built for the current query
    int32_t rd_cap = 0;
    int32_t rd_on = 0;
    // live-mask cache, [W][m] per direction (optional)
    sgi::DBuf<unsigned long long> lm_out, lm_in;
    int32_t lm_cap = 0;       // words the cache was sized for
    // undirected variant: per-snapshot component labels, sizes, degree sums,
    // covered flags [R][n]; the round's roots and new sizes [2R]
    sgi::DBuf<int32_t> cc_lab, cc_size, cc_root;
    sgi::DBuf<long long> cc_deg;
    sgi::DBuf<uint8_t> cc_cov;
    size_t cc_cap = 0;
    int32_t cc_rcap = 0;
    int32_t lm_on = 0;        // built for the current query
    int32_t kcap = 0;
    int32_t am_blocks = 0;
};

struct sg_graph {
    int64_t n = 0;
    int64_t m = 0;
    int device = 0;
    int num_sms = 0;
    sgi::DBuf<int32_t> rp, col, crp;
    sgi::DBuf<int2> cin;
    sgi::DBuf<uint32_t> tmi;
    sgi::DBuf<uint2> fw;      // built on first WIC query
    int32_t lmk_nodes[8] = {-1, -1, -1, -1, -1, -1, -1, -1};  // landmarks: largest out-degrees (>= 32)
    int32_t lmk_count = 0;
    // heavy rows (static)
    int32_t heavy_min_deg = 0;
    int32_t nh_out = 0, nh_in = 0;
    long long hsum_out = 0, hsum_in = 0;   // sum of heavy-row degrees
    double hlive_out_wic = 0;              // sum over heavy out-rows' arcs of 1 / indeg(destination)
    // undirected variant: -1 not checked, 0 not symmetric, 1 symmetric; the
    // source of every arc and min(arc id, reverse arc id)
    int32_t cc_sym = -1;
    sgi::DBuf<int32_t> cc_esrc, cc_pmin;
    sgi::DBuf<int32_t> hid_out, hrow_out, hid_in, hrow_in;
    sgi::DBuf<long long> hpref_out, hpref_in;
    sg_workspace ws;
};

namespace sgi {

GraphView view_of(const sg_graph *g, const sg_workspace &ws, int heavy_on);
sg_status ensure_wic(sg_graph *g, cudaStream_t st);
sg_status ensure_workspace(sg_graph *g, sg_workspace &ws, int32_t W, int32_t k, cudaStream_t st);
sg_status ensure_heavy_index(sg_graph *g, sg_workspace &ws, int32_t W, cudaStream_t st);
void free_workspace(sg_workspace &ws, cudaStream_t st);
sg_status make_coins(const sg_cascade &c, uint64_t seed, int32_t R, Coins *out);
bool heavy_index_enabled(const sg_graph *g, int32_t W);


// kernels launched by this thread since the counter was last reset
extern thread_local int g_launches;
// keys a tier-1 / tier-2 warp table may hold (clamped to half its slots)
extern int g_tier_limit[2];
// landmark nodes used for the initial gains (0 .. 8)
extern int g_landmarks;
// blocks per 64-snapshot word of the level-synchronous forward and landmark
// walks (8, 16, 32 or 64; each owns 64/groups snapshot bits)
extern int g_walk_groups;
// direction-optimising switch of the level-synchronous walks: mode 0
// top-down only, 1 bottom-up once a level's frontier holds more than
// n / g_bu_div nodes, 2 bottom-up from the second level on
extern int g_bu_mode;
extern int g_bu_div;
// nonzero: initial-gain sources inside a landmark's strongly connected
// component skip those snapshots' walks (the landmark credit counts them)
extern int g_scc;
extern int g_word_major;
extern int g_t1_direct;
// The tunable knobs one query runs with (none changes a result).
struct Knobs {
    int walk_groups;  // blocks per word of the forward and landmark walks
    int bu_mode;      // direction-optimising switch of the walks
    int bu_div;
    int t1_keys;      // tier-1 / tier-2 key limits of the traversal engines
    int t2_keys;
    int landmarks;    // landmarks for the initial gains (0 .. 8)
    int scc;          // SCC condensation of initial-gain sources
    int fwd_lists;    // forward per-snapshot live lists
    int word_major;   // initial-gain tasks numbered word-major (1) or source-major (0)
    int t1_direct;    // warp-tier overflows with this many frontier entries left skip tier 2 (0: never)
};
// The calling thread's current query knobs: the per-query tuning it was
// given (t_knobs, set for the duration of one query) or else the
// process-wide values of the sg_set_* calls.
extern thread_local const Knobs *t_knobs;
Knobs knobs();
// Applies a query's tuning (NULL: none) to the calling thread for its
// lifetime.
struct KnobScope {
    explicit KnobScope(const sg_tuning *t);
    ~KnobScope();
    KnobScope(const KnobScope &) = delete;
    KnobScope &operator=(const KnobScope &) = delete;

  private:
    const Knobs *prev_ = nullptr;
    Knobs own_{};
};
sg_status check_query_tuning(const sg_tuning *t);
// polls a bounded device-side wait of the traversal engines makes before it
// gives up (default 2^22; a testing hook can shorten it)
extern long long g_wait_polls;
constexpr long long WAIT_POLLS_DEFAULT = 1LL << 22;
// per-snapshot live in-lists of heavy rows for the reverse update (0 or 1)
extern int g_snapshot_lists;
// nonzero: queries build and use the live-mask cache when it fits
extern int g_mask_cache;
// nonzero: queries build and use forward per-snapshot live lists when they fit
extern int g_fwd_lists;

// kernels (sg_kernels.cu)
sg_status run_heavy_index(sg_graph *g, sg_workspace &ws, const Coins &co, int model, cudaStream_t st);
sg_status run_snapshot_lists(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status run_mask_cache(sg_graph *g, sg_workspace &ws, const Coins &co, int model, cudaStream_t st);
sg_status run_argmax(sg_graph *g, sg_workspace &ws, const Coins &co, int32_t round, cudaStream_t st);
// undirected variant (sg_cc.cu)
sg_status cc_prepare_graph(sg_graph *g, cudaStream_t st);
size_t cc_workspace_bytes(const sg_graph *g, int32_t R);
sg_status cc_ensure(sg_graph *g, sg_workspace &ws, int32_t R, cudaStream_t st);
sg_status cc_init_gains(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status cc_round(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status cc_clear_cover(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status cc_spread(sg_graph *g, sg_workspace &ws, const Coins &co, const int32_t *d_S, int32_t ns, long long *d_total,
                    unsigned long long *d_edges, cudaStream_t st);
sg_status run_row_desc(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status run_fwd_lists(sg_graph *g, sg_workspace &ws, const Coins &co, cudaStream_t st);
sg_status ensure_fwd_lists(sg_graph *g, sg_workspace &ws, const Coins &co, double p_uic, int model, cudaStream_t st);
sg_status run_spread(sg_graph *g, const Coins &co, int model, const int32_t *d_S, int32_t ns, long long *d_total,
                     unsigned long long *d_edges, cudaStream_t st);
// Walk from d_S over all W words (FWD_GROUPS blocks per word) on the query's
// coins (heavy-row index and caches of ws when heavy_on): vis [W][n] holds
// the nodes to leave out and gains the reached bits; pend [W][n] zero;
// qa/qb [W * 8][n]; new (node, snapshot) pairs / out-degrees added to
// d_total / d_edges.
sg_status run_walk(sg_graph *g, const sg_workspace &ws, const Coins &co, int model, int heavy_on,
                   const int32_t *d_S, int32_t ns, unsigned long long *vis, unsigned long long *pend, int32_t *qa,
                   int32_t *qb, long long *d_total, unsigned long long *d_edges, cudaStream_t st);
sg_status ensure_mask_cache(sg_graph *g, sg_workspace &ws, int32_t W, cudaStream_t st, bool required = false);
size_t mask_cache_bytes(const sg_graph *g, int32_t W);
sg_status ensure_snapshot_lists(sg_graph *g, sg_workspace &ws, const Coins &co, double p_uic, int model,
                                cudaStream_t st);
// events recorded around the initial-gain tier launches (any may be null)
struct TierEvents {
    cudaEvent_t start = nullptr, t1 = nullptr, t2 = nullptr, t3 = nullptr;
};
sg_status run_init_gains(sg_graph *g, sg_workspace &ws, const Coins &co, int model, int heavy_on, cudaStream_t st,
                         const TierEvents *ev = nullptr);
sg_status run_round(sg_graph *g, sg_workspace &ws, const Coins &co, int model, int heavy_on, int32_t round,
                    cudaStream_t st, cudaEvent_t after_fwd = nullptr);
sg_status run_live_masks(sg_graph *g, const Coins &co, int model, uint64_t *out, cudaStream_t st,
                         const int32_t *cid = nullptr);

// host driver (sg_host.cu)
// Device flags (Ctl::flags) a query can leave: FLAG_NO_CANDIDATE, the argmax
// found no candidate; FLAG_WAIT, a bounded device-side wait gave up;
// FLAG_UNION_FIND, the union-find ran out of hooking retries.
enum { FLAG_NO_CANDIDATE = 1, FLAG_WAIT = 2, FLAG_UNION_FIND = 8 };
// SG_OK for flags 0; SG_ETIMEOUT when FLAG_WAIT is set; SG_EINTERNAL for
// any other flag.  Sets the thread's error text on failure.
sg_status flags_status(int32_t flags);
// Testing hook (sg_debug_inject_flags): OR the flags set aside for the next
// query into ws's device flags, as a failing device step would.
sg_status plant_injected_flags(sg_workspace &ws, cudaStream_t st);
// When ws's device flags are set: seeds[0..count) = -1 (if seeds) and
// vals[0..count) = -flags, so that outputs of an asynchronous call carry
// the failure.  Nothing is written otherwise.
sg_status run_poison(const sg_graph *g, sg_workspace &ws, int32_t *seeds, long long *vals, long long count,
                     cudaStream_t st);
sg_status select_impl(sg_graph *g, sg_workspace &ws, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                      int32_t *out_seeds, int64_t *out_gains, sg_stats *stats, bool prepare_only);
sg_status check_query(const sg_graph *g, int32_t R, int32_t k);
size_t workspace_bytes(const sg_graph *g, int32_t W, int32_t k);

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};


}  // namespace sgi
