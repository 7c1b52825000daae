/*
 * sg.h -- C ABI of the GB300 StaticGreedy-DU library (libsg.so).
 *
 * StaticGreedy (Cheng, Shen, Huang, Zhang, Cheng, CIKM 2013) picks k seed
 * nodes of an independent-cascade graph (Section 3.1) greedily on R static
 * live-edge snapshots (Section 3.3, Algorithm 1); StaticGreedyDU keeps
 * every candidate's marginal gain current with the dynamic update of
 * Section 4 (Algorithm 2).  This library runs that path on one GPU:
 *   - snapshot sampling: arc e is live in snapshot r iff
 *       hi32(splitmix64(seed ^ (r << 40) ^ e)) < thr(e),
 *     thr = floor(p * 2^32) (uniform cascade, UIC) or
 *     thr(u->v) = floor(2^32 / indeg(v)) (weighted cascade, WIC,
 *     p(u,v) = 1/d_v of Section 3.4.1); snapshots are never stored;
 *   - initial gains s_v = sum_r |R(G'_r, v)| (Algorithm 2, first loop),
 *     where R(G'_r, v) includes v itself;
 *   - k rounds of: v* = argmax over non-seeds of s_v, lowest id on ties;
 *     forward BFS from v* marking the nodes it newly covers in each
 *     snapshot; reverse BFS from each newly covered node subtracting one
 *     from the gain of every node that reaches it (Algorithm 2, inner loops).
 * All arithmetic is exact integer, so results are bit-identical to any
 * correct implementation of the same definition.
 *
 * Conventions for every entry point:
 *   - return an sg_status; never abort, trap or print.  On failure
 *     sg_last_error() returns a thread-local message.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it in stream order.
 *   - node ids are int32 in [0, n); arcs are directed u -> v.
 *   - device-side failures: every device-side wait is bounded and every
 *     device step checks its invariants; a failure sets the query's device
 *     flags (a wait that gave up: SG_ETIMEOUT; a failed check:
 *     SG_EINTERNAL).  A call that returns after the stream has finished
 *     (stats requested or pageable host outputs) returns that status.  A
 *     call that returns once the work is enqueued cannot; its outputs carry
 *     the failure instead: every seed reads -1 and every gain (or initial
 *     gain) reads -flags, where flag 2 marks a wait that gave up.  Valid
 *     outputs are never negative.  The CUDA context stays usable.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,    /* an argument is out of range or malformed */
    SG_ENOMEM = 2,    /* a device or host allocation failed */
    SG_ECUDA = 3,     /* a CUDA runtime call failed */
    SG_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    SG_EBUSY = 5,     /* the object is in use (e.g. server slots full) */
    SG_EINTERNAL = 6  /* a device-side consistency check failed */
} sg_status;

/* SG_UIC: every arc live with probability p, one coin per arc.
 * SG_WIC: arc u->v live with probability 1 / indeg(v).
 * SG_UIC_UNDIRECTED: the undirected variant -- a symmetric graph (every
 *   arc's reverse present) with one coin per undirected edge: both arcs use
 *   the coin of the lower of their two canonical arc ids, so each snapshot
 *   is undirected and reach sets are connected components.  sg_select,
 *   sg_init_gains, sg_spread, sg_live_masks, batches and the server accept
 *   it (sg_select runs it by per-snapshot union-find); sg_select_celf does
 *   not.  A graph that is not symmetric gives SG_EINVAL.
 * SG_LT: the linear threshold model in its live-edge form (Kempe, Kleinberg
 *   and Tardos 2003; the paper's Section 3.4.2 and Section 7 name the LT
 *   generalisation), weights 1/indeg(v): in each snapshot every node v
 *   keeps at most one in-arc.  v's draw in snapshot r is
 *   hi32(splitmix64(seed ^ (r << 40) ^ v)); its in-arcs, sources ascending,
 *   own the intervals [j w, (j+1) w), w = floor(2^32 / indeg(v)), and the
 *   arc whose interval holds the draw is live (none when the draw is past
 *   indeg(v) w).  p is ignored.  Every entry point accepts it; the coins are
 *   materialised once per query into the live-mask cache (2 x W x m x 8
 *   bytes, at most 16 GiB, else SG_ENOMEM) and the heavy-row index is not
 *   used. */
typedef enum { SG_UIC = 0, SG_WIC = 1, SG_UIC_UNDIRECTED = 2, SG_LT = 3 } sg_model;

/* Cascade model: UIC uses p in [0, 1] for every arc; WIC ignores p and uses
 * 1/indeg(v) for every arc u -> v (Section 3.4.1 and Section 5.1). */
typedef struct {
    int32_t model; /* sg_model */
    double p;      /* UIC only */
} sg_cascade;

/* Counters and timings of one sg_select call.  The three snapshot-edge
 * counts are implementation independent:
 *   init_edges = sum over (v, r) and u in R(G'_r, v) of outdeg(u)
 *   fwd_edges  = sum over newly covered (u, r) of outdeg(u)
 *   rev_edges  = sum over newly covered (w, r) and u in U(G'_r, w) of indeg(u)
 * (outdeg / indeg of the canonical graph, live or not).  The other fields
 * describe how this implementation ran (tiers, task counts, device times). */
typedef struct {
    uint64_t init_edges;
    uint64_t fwd_edges;
    uint64_t rev_edges;
    uint64_t init_tier2_tasks;  /* initial-gain tasks that outgrew the shared-memory table */
    uint64_t init_tier3_tasks;  /* ... and the global-memory table */
    uint64_t rev_tier2_tasks;   /* same for reverse (dynamic-update) tasks */
    uint64_t rev_tier3_tasks;
    uint64_t rev_tasks;         /* reverse tasks (one snapshot, <= 64 targets), all rounds */
    uint64_t du_entries;        /* (node, 64-snapshot word) pairs newly covered, all rounds */
    float ms_index;             /* device time building the heavy-row live index and lists */
    float ms_init;              /* device time of the initial gains (index included) */
    float ms_init_tier1;        /* device time of the initial-gain tier-1 launch */
    float ms_rounds;            /* device time of the k selection rounds */
    float ms_fwd;               /* ... of which argmax + forward update, summed */
    float ms_total;             /* device time of the whole call */
    int32_t status_flags;       /* device flags: 1 no argmax candidate, 2 a bounded wait gave up, 8 union-find out of retries */
    int32_t kernel_launches;    /* kernels this call launched */
    int32_t heavy_index;        /* 1 if the heavy-row live index was used */
    int32_t mask_cache;         /* 1 if the live-mask cache was used */
    uint64_t work_keys[2][3];   /* [initial, reverse][tier 1..3]: nodes held in task tables */
    uint64_t work_elems[2][3];  /* [initial, reverse][tier 1..3]: arcs / index entries expanded */
    float ms_landmarks;         /* device time of the landmark reach sets */
    float ms_init_tier2;        /* device time of the initial-gain tier-2 launch */
    float ms_init_tier3;        /* device time of the initial-gain tier-3 launch */
    int32_t reserved2;
    uint64_t list_elems[3];     /* initial gains, tier 1..3: of work_elems, per-snapshot live-list entries */
} sg_stats;

/* Opaque graph handle; owns its device memory until sg_free_graph. */
typedef struct sg_graph sg_graph;

/* Device memory hooks.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); release returns it.  Without
 * hooks the library uses cudaMallocAsync / cudaFreeAsync.  Passing NULL
 * functions restores the default.  Not thread-safe with concurrent calls. */
typedef void *(*sg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*sg_release_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
sg_status sg_set_allocator(sg_alloc_fn alloc, sg_release_fn release, void *ctx);

/* Load a graph given in CSR form (Section 3.1 graph G).
 *   n        number of nodes, 1 <= n < 2^31
 *   m        number of arcs in col, 0 <= m < 2^31
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      int32[m], destinations in [0, n)
 *   is_device_ptr  0: row_ptr/col are host memory; 1: device memory
 * The graph is canonicalised: self-loops are dropped and repeated arcs
 * merged (the paper merges parallel edges, Section 5.1), rows sorted by
 * destination; canonical arc ids are CSR positions of that graph.  The
 * caller keeps ownership of its arrays; the library copies them.
 * Errors: SG_EINVAL for any violated bound above.  The handle is written
 * to *out only on SG_OK. */
sg_status sg_load_graph(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                        int is_device_ptr, void *stream, sg_graph **out);

/* Degree at or above which a row gets a per-query live index in graphs
 * loaded after this call: for each such row and 64-snapshot word the
 * nonzero live masks of its arcs are computed once per query (from the
 * same hash) instead of on every expansion, and the reverse pass reads the
 * live in-arcs of such rows per snapshot.  0 disables the index; the
 * default is 2 (every row with two or more arcs; the index is skipped when
 * it would pass 8 GiB).  Results do not depend on it.
 * Errors: SG_EINVAL if < 0. */
sg_status sg_set_heavy_threshold(int32_t min_degree);

/* Traversal-engine limits: a task whose visited set grows past tier1_keys
 * nodes leaves its warp's shared-memory table (tier 1) for a block-shared
 * shared-memory table (tier 2: 2048-slot tables, four blocks per SM,
 * holding up to min(1024, tier2_keys / 2) nodes), and past that for the
 * engine with dense per-slot arrays in global memory (tier 3).  A task
 * that leaves tier 1 with a large frontier still to expand may go straight
 * to tier 3 (sg_tuning.tier1_direct).  Values are clamped to 256 and
 * 2048; the defaults are 64 and 2048.  A tuning and testing knob:
 * results do not depend on it.  Applies to later calls.
 * Errors: SG_EINVAL if either is < 1. */
sg_status sg_set_engine_limits(int32_t tier1_keys, int32_t tier2_keys);

/* Landmarks for the initial gains: the reach sets of the `count` nodes of
 * largest out-degree (default 8, at most 8, degree >= 32) are computed once
 * per snapshot, together with the size of the union of every subset of
 * them; a source that reaches some landmarks in a snapshot is credited with
 * the union of their sets instead of traversing them again.  0 disables
 * it.  Results do not depend on it.  Applies to later calls.
 * Errors: SG_EINVAL unless 0 <= count <= 8. */
sg_status sg_set_landmarks(int32_t count);

/* Per-snapshot live in-arc lists of heavy rows for the reverse (dynamic
 * update) pass: 1 (the default) builds them per query from the heavy-row
 * index so that a reverse step over one snapshot reads only that
 * snapshot's live in-arcs of a hub; 0 disables.  Results do not depend on
 * it.  Applies to later calls.  Errors: SG_EINVAL unless 0 or 1. */
sg_status sg_set_snapshot_lists(int32_t enable);

/* Forward per-snapshot live lists for the initial gains and the forward
 * walks: 1 (the default) builds, per query, each indexed row's live
 * out-arcs per snapshot (from the heavy-row index).  With them, state bits
 * of snapshots in which a node has no live out-arc are finished without a
 * read; a node whose nonempty lists in a word hold one arc each expands
 * one list entry per state bit; another node reached in at most 4 of a
 * word's snapshots is expanded through those lists one snapshot at a time
 * instead of scanning all its index entries.  0 disables.  Skipped when
 * the lists would pass 8 GiB.  Results do not depend on it.  Applies to
 * later calls.  Errors: SG_EINVAL unless 0 or 1. */
sg_status sg_set_forward_lists(int32_t enable);

/* Per-snapshot SCC condensation of the initial-gain sources: 1 (the default)
 * or 0.  The landmarks serve as pivots: a landmark's strongly connected
 * component in snapshot r is R(G'_r, x_i) intersected with U(G'_r, x_i)
 * (forward-backward from the pivot, exact), and every member v has
 * R(G'_r, v) = R(G'_r, x_i).  A source inside such a component skips its
 * walk for that snapshot and is credited the pivot's reach through the
 * landmark union (which already counts it); without the switch the walk
 * runs and all it finds is filtered out.  Needs landmarks (sg_set_landmarks
 * > 0).  Results and counters do not depend on it.  Applies to later
 * calls.  Errors: SG_EINVAL unless 0 or 1. */
sg_status sg_set_scc_condensation(int32_t enable);

/* Direction-optimising switch of the level-synchronous walks (the forward
 * dynamic update's walk from each new seed, its walk back over the seed's
 * ancestors, and the landmark walks of the initial gains; sg_spread's
 * walks, which hash their coins in registers, stay top-down).  A
 * top-down level expands every frontier node's arcs; a bottom-up level
 * instead lets every node still missing some snapshot bits scan its arcs
 * from the other side (in-arcs of a forward walk) for frontier nodes with
 * live arcs, stopping once nothing is missing -- cheaper once the frontier
 * is a large part of the graph (Beamer et al., SC 2012).
 *   mode 0: top-down only; 1 (default): a level runs bottom-up when its
 *   frontier holds more than n / divisor nodes (default divisor 4); 2:
 *   every level after the first runs bottom-up (for testing).
 * Results and the snapshot-edge counters do not depend on it.  Applies to
 * later calls.  Errors: SG_EINVAL unless 0 <= mode <= 2 and divisor >= 1. */
sg_status sg_set_direction(int32_t mode, int32_t divisor);

/* Blocks per 64-snapshot word of the level-synchronous walks (the forward
 * dynamic update's walk from each new seed and the landmark walks of the
 * initial gains): each block owns 64/groups of the word's snapshot bits.
 * 8, 16, 32 or 64 (default 64: one snapshot bit per block); more blocks
 * spread one walk over more SMs.
 * Workspaces size their level queues for max(8, groups) at creation (4
 * bytes per node, word and block, twice); a query on an older workspace
 * uses at most what it was sized for.  Results do not depend on it.
 * Applies to later calls.  Errors: SG_EINVAL for any other value. */
sg_status sg_set_walk_groups(int32_t groups);

/* Live-mask cache: 1 makes each later query first evaluate every arc's coin
 * for all R snapshots once (the hash of Section 3.1's snapshot definition,
 * 64 snapshots per 64-bit word) into a per-workspace table of 2 x W x m
 * words (CSR and CSC order), which the traversals then read instead of
 * hashing in registers; 0 (the default) hashes in registers.  The table
 * is a cache of the same function, so results do not depend on it.  It is
 * skipped (in-register hashing) when it would pass 16 GiB.  Its bytes are
 * included in sg_workspace_bytes while it is enabled.  Applies to later
 * calls.  Errors: SG_EINVAL unless 0 or 1. */
sg_status sg_set_mask_cache(int32_t enable);

/* StaticGreedyCELF (Section 6): the same seeds and gains as sg_select,
 * found with lazy forward evaluation (CELF, Section 2) over the static
 * snapshots instead of the dynamic update.  After the initial gains (the
 * same kernels as sg_select) the candidates wait in a host priority queue
 * ordered by (bound descending, id ascending); a head whose bound is from
 * the current round is the seed, otherwise its marginal gain
 * sum_r |R(G'_r, v) minus the covered nodes| is computed on the GPU and it
 * is queued again.  *out_evals (may be NULL) receives the number of such
 * evaluations (the initial gains not counted).  Outputs as sg_select (host
 * or device); stats (may be NULL): init and forward snapshot-edge counts
 * (reverse 0), ms_init, ms_rounds, ms_total.  Synchronises `stream` once per
 * evaluation and per round (not capturable).  Uses the graph's default
 * workspace, like sg_select.  Errors: as sg_select. */
sg_status sg_select_celf(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                         int32_t *out_seeds, int64_t *out_gains, int64_t *out_evals, sg_stats *stats);

/* Seed-set spread on fresh snapshots (Section 3.1's snapshot estimate of
 * the influence spread; Section 6 rates seed sets by Monte Carlo
 * simulation): *out_total = sum over the R snapshots of hash seed `seed`
 * of |R(G'_r, S)|, the nodes reachable from S = S[0..s_count) including
 * S; the spread estimate is *out_total / R.  Repeated seeds count once;
 * s_count = 0 gives 0.  *out_edges (may be NULL) gets the snapshot-edge
 * count, the out-degree sum over the reached (node, snapshot) pairs.
 * A multi-source bit-sliced traversal, one 64-snapshot word per block, with
 * the coins hashed in registers (no per-query cache is used).  S: host or
 * device int32[s_count]; out_total: host or device int64; out_edges: host.
 * Synchronises `stream` before returning; uses up to ~8 GiB of scratch.
 * Errors: SG_EINVAL for a NULL graph/output, s_count < 0, a seed outside
 * [0, n), R outside [1, 2^24) or an invalid cascade; SG_ENOMEM; SG_ECUDA. */
sg_status sg_spread(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, const int32_t *S, int32_t s_count,
                    void *stream, int64_t *out_total, uint64_t *out_edges);

/* Same as sg_load_graph from an arc list src[i] -> dst[i], i < m.
 * src/dst are host memory when is_device_ptr is 0, device memory when 1. */
sg_status sg_load_graph_coo(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            int is_device_ptr, void *stream, sg_graph **out);

/* Release the device memory of the graph's own workspace (the one
 * sg_select, sg_init_gains, sg_select_celf and sg_spread use); the graph
 * itself stays resident and the next such call sizes the workspace again.
 * Explicit workspaces (sg_workspace_create) are not affected.  Waits for
 * the device.  Errors: SG_EINVAL for a NULL graph. */
sg_status sg_graph_trim(sg_graph *g);

/* Node count and canonical arc count. */
sg_status sg_graph_info(const sg_graph *g, int64_t *n, int64_t *m_canonical);

/* Select k seeds with StaticGreedyDU (Algorithm 2) on R hash-defined
 * snapshots of g under cascade c.
 *   R      1 <= R < 2^24 snapshots (64 per bit-sliced word; the last word
 *          is masked to R mod 64 snapshots)
 *   k      1 <= k <= n
 *   seed   64-bit hash seed of the snapshots
 *   out_seeds int32[k]: seed i (0-based round order)
 *   out_gains int64[k]: gain_i = f(S_i) - f(S_{i-1}) with
 *             f(S) = sum_r |R(G'_r, S)|; the spread estimate of S_k is
 *             sum(gains) / R.
 *   stats  optional (NULL allowed); filling it synchronises the stream.
 * Outputs may be device memory, pinned host memory or pageable host
 * memory; with pageable host memory or stats the call returns after the
 * stream has finished, otherwise it returns once the work is enqueued.
 * Ties in the argmax go to the lowest node id among non-seeds, also when
 * every remaining gain is 0; seeds are never re-picked.
 * Errors: SG_EINVAL (bounds above, p outside [0,1] or NaN, unknown model),
 * SG_ENOMEM, SG_ECUDA; SG_ETIMEOUT / SG_EINTERNAL for a device-side failure
 * (see the conventions above). */
sg_status sg_select(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                    int32_t *out_seeds, int64_t *out_gains, sg_stats *stats);

/* sg_select, then the state Algorithm 2 maintains after its k rounds, for
 * checking its invariant (Section 4):
 *   out_s   int64[n]: for every non-seed u the marginal gain
 *           f(S ∪ {u}) − f(S) of the k seeds S (the s_u of Algorithm 2 after
 *           the last round's update); seeds hold a negative marker
 *   out_cov uint64[ceil(R/64) * n]: bit b of out_cov[w*n + u] is set iff u
 *           is reached from S in snapshot 64w + b (the coverage of S)
 * Outputs are host or device memory; the call synchronises `stream`.
 * Cascades SG_UIC, SG_WIC and SG_LT (the undirected variant keeps its
 * state as per-snapshot components).  Errors: as sg_select, and SG_EINVAL
 * for NULL outputs or the undirected variant. */
sg_status sg_select_state(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                          int32_t *out_seeds, int64_t *out_gains, int64_t *out_s, uint64_t *out_cov);

/* Per-query device state (gains, coverage bitsets, task lists, caches).
 * sg_select uses one owned by the graph; several queries can run on one
 * graph at the same time only with workspaces of their own.
 * sg_workspace_create sizes one for queries on g with R <= R_max and
 * k <= k_max (device memory taken through the allocator hooks, cleared;
 * synchronises `stream`).  sg_workspace_bytes reports that size without
 * allocating.  A workspace belongs to the graph it was created for until
 * sg_workspace_free (waits for the device). */
typedef struct sg_workspace sg_workspace;
sg_status sg_workspace_create(const sg_graph *g, int32_t R_max, int32_t k_max, void *stream,
                              sg_workspace **out);
sg_status sg_workspace_bytes(const sg_graph *g, int32_t R_max, int32_t k_max, size_t *bytes);
void sg_workspace_free(sg_workspace *ws);

/* sg_select with an explicit workspace (same arguments and results).
 * Calls with different workspaces may run concurrently on different
 * streams; one workspace serves one call at a time. */
sg_status sg_select_ws(sg_graph *g, sg_workspace *ws, int32_t R, int32_t k, sg_cascade c, uint64_t seed,
                       void *stream, int32_t *out_seeds, int64_t *out_gains, sg_stats *stats);

/* Tuning knobs of a query (no counterpart in the paper; none changes a
 * result, only how the same counts are computed):
 *   walk_groups     blocks per 64-snapshot word of the forward and landmark
 *                   walks (8, 16, 32, 64; see sg_set_walk_groups)
 *   direction_mode, direction_div   the walks' top-down/bottom-up switch
 *                   (see sg_set_direction)
 *   tier1_keys, tier2_keys          engine tier limits (sg_set_engine_limits)
 *   landmarks       0..8 (sg_set_landmarks)
 *   scc             0/1 (sg_set_scc_condensation)
 *   forward_lists   0/1 (sg_set_forward_lists)
 *   word_major      initial-gain task order: 1 (default) all of one 64-snapshot
 *                   word's sources before the next word's, so the tasks in
 *                   flight share that word's caches in L2; 0 source by source
 *   tier1_direct    a task (initial gains or reverse update) that outgrows
 *                   its warp's table with at least this many frontier
 *                   entries still to expand goes straight to the dense tier,
 *                   skipping the block-shared table it would likely outgrow
 *                   too (default 16; 0: never)
 * The slice width is fixed at 64 snapshots (one 64-bit word per node and
 * task) and is not a knob. */
typedef struct {
    int32_t walk_groups;
    int32_t direction_mode;
    int32_t direction_div;
    int32_t tier1_keys;
    int32_t tier2_keys;
    int32_t landmarks;
    int32_t scc;
    int32_t forward_lists;
    int32_t word_major;
    int32_t tier1_direct;
} sg_tuning;

/* The process-wide knobs (what the sg_set_* calls set) / set all of them.
 * Errors: SG_EINVAL for a NULL pointer or a value out of range. */
sg_status sg_get_tuning(sg_tuning *out);
sg_status sg_set_tuning(const sg_tuning *t);

/* Autotuner.  Finds the fastest knobs for one query: times whole
 * selections of (g, R, k, c, seed) on `stream` under candidate settings,
 * one knob at a time (walk groups, direction switch, landmarks, SCC
 * condensation, tier limits, forward lists; each candidate the fastest of
 * two timed runs after one untimed), checks that every candidate returns
 * the same seeds and gains, and keeps a change only when it is at least 1%
 * faster.  *out receives the tuning and *out_ms (may be NULL) its time per
 * selection.  With cache_path (may be NULL) a JSON-lines file is read
 * first -- a line whose key (node and arc counts, largest out-degree,
 * model, UIC probability, word count) matches is returned without timing --
 * and a new result is appended.  The process-wide knobs are not changed:
 * pass *out to sg_set_tuning, or put it in sg_query.tuning.  The graph's
 * own workspace is released and sized again (its queues for 64 walk
 * groups).  Synchronises `stream`; takes about 20 selections' time.
 * Errors: as sg_select; SG_EINTERNAL if two settings gave different
 * results. */
sg_status sg_autotune(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                      const char *cache_path, sg_tuning *out, double *out_ms);

/* One query of a batch. */
typedef struct {
    sg_graph *graph;
    sg_workspace *ws;     /* NULL: the graph's own (then one query per graph in a batch) */
    int32_t R;
    int32_t k;
    sg_cascade cascade;
    uint64_t seed;
    int32_t *out_seeds;   /* int32[k], device or pinned host memory */
    int64_t *out_gains;   /* int64[k], device or pinned host memory */
    sg_status status;     /* written by the call */
    const sg_tuning *tuning;  /* NULL: the process-wide knobs; else this query's (e.g. from sg_autotune);
                                 a workspace's walk queues cap walk_groups at what it was sized for */
} sg_query;

/* Run nq independent queries (different graphs, R, k, cascades) at once:
 * they are spread over `concurrency` internal streams that start after the
 * work already queued on `stream` and that `stream` waits for at the end,
 * so their kernels overlap on the device.  Returns once everything is
 * enqueued.  Results are identical to running each query alone.
 * Errors: SG_EINVAL (bad query; its status says which), others as
 * sg_select.  The first failing status is returned. */
sg_status sg_select_batch(int32_t nq, sg_query *q, int32_t concurrency, void *stream);

/* The same batch recorded once as a CUDA graph (stream capture over the
 * internal streams) and replayed with a single graph launch per
 * sg_batch_launch.  Buffers and parameters are fixed at capture; every
 * query needs its own workspace sized for it, and outputs must be device
 * or pinned host memory.  sg_batch_capture runs nothing on the device. */
typedef struct sg_batch sg_batch;
sg_status sg_batch_capture(int32_t nq, sg_query *q, int32_t concurrency, void *stream, sg_batch **out);
sg_status sg_batch_launch(sg_batch *b, void *stream);
void sg_batch_free(sg_batch *b);

/* Serving loop with continuous batching.  A worker thread keeps up to
 * max_running queries on the device at once, each on its own stream and
 * workspace; queued requests are admitted in arrival order as soon as a
 * slot and device memory (memory_budget bytes for workspaces) allow, so
 * requests arriving while others run overlap with them on the device.
 * Idle workspaces are kept per graph and reused; when memory is short the
 * least recently used idle ones are released.  Graphs must stay loaded
 * while requests on them are pending.  Results are identical to sg_select
 * on the same query.  The worker uses the library's built-in allocator
 * (cudaMallocAsync), not the allocator hooks. */
typedef struct sg_server sg_server;
typedef struct {
    int32_t max_running;   /* >= 1 */
    size_t memory_budget;  /* bytes for workspaces; 0: 80% of free device memory at creation */
    int32_t k_cap;         /* largest k a request may ask for */
} sg_server_cfg;
sg_status sg_server_create(const sg_server_cfg *cfg, sg_server **out);
/* Queue a request; *request_id identifies it.  SG_EINVAL for bad
 * arguments, SG_EBUSY if the server is shutting down. */
sg_status sg_server_submit(sg_server *srv, sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed,
                           int64_t *request_id);
/* *done = 1 and the results (host memory, k entries) once the request has
 * finished; latency_ms = completion minus submission (host clock).
 * *done = 0 while pending; SG_EINVAL for an unknown id.  A finished
 * request is forgotten after its results are returned.  If it failed, its
 * status is returned. */
sg_status sg_server_poll(sg_server *srv, int64_t request_id, int32_t *done, int32_t *out_seeds,
                         int64_t *out_gains, double *latency_ms);
/* Requests queued, running, finished-but-unpolled. */
sg_status sg_server_counts(sg_server *srv, int64_t *queued, int64_t *running, int64_t *finished);
/* Stop accepting, finish everything queued, free every resource. */
void sg_server_destroy(sg_server *srv);

/* Initial gains only (Algorithm 2, first loop): s[v] = sum_r |R(G'_r, v)|
 * for every v, written to out_s (int64[n], device or host memory), and the
 * init snapshot-edge count to *init_edges (NULL allowed; non-NULL
 * synchronises the stream).  Same argument rules as sg_select. */
sg_status sg_init_gains(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, void *stream,
                        int64_t *out_s, uint64_t *init_edges);

/* Live-edge masks of snapshots 0..R-1 as 64-snapshot words:
 * out_masks[e * W + w] bit b = live(e, 64w + b), W = ceil(R/64), bits at
 * or beyond R are 0; e is the canonical arc id.  out_masks: uint64[m*W],
 * device or host memory.  Exposes the snapshot definition for checking. */
sg_status sg_live_masks(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, void *stream,
                        uint64_t *out_masks);

/* Canonical CSR of g into caller buffers (host or device):
 * row_ptr int64[n+1], col int32[m_canonical]. */
sg_status sg_graph_csr(const sg_graph *g, void *stream, int64_t *row_ptr, int32_t *col);

/* Argmax over a gain vector the caller owns, with no device allocation.
 * The paper has no counterpart: this exists for callers that cannot
 * allocate device memory where they need the argmax -- latency-bound
 * serving loops that must not stall on a synchronous allocation, or
 * plug-ins whose host framework owns all device memory through its own
 * pool and hands out only the buffers it manages.
 *   s         int64[n] in device-accessible memory; entries < 0 are
 *             excluded (sg_select marks seeds that way)
 *   n         1 <= n <= 2^31 - 1
 *   out_id    int32 (device-accessible): the lowest v with the largest
 *             s[v] >= 0, or -1 if every entry is negative
 *   out_gain  int64 (device-accessible): s[out_id], or -1
 * Work is enqueued on `stream`; the call returns without waiting.
 * Scratch: one statically sized array of about 12 KB per device (1024
 * block partials and a counter), held until the process exits.  The first
 * call in a CUDA context (normally the device's primary context; with none
 * current, the current device's primary context is bound) looks up that
 * array's address there with cudaGetSymbolAddress and caches it for that
 * context, so make the first call before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  No cudaMalloc,
 * cudaFree or other allocating routine is called.
 * Errors: SG_EINVAL (NULL pointer, n out of range, more than 64 contexts),
 * SG_ECUDA. */
sg_status sg_argmax_noalloc(const int64_t *s, int64_t n, void *stream, int32_t *out_id, int64_t *out_gain);

/* Testing hook (host fault injection): the next query started on any
 * thread (sg_select, sg_select_ws, sg_init_gains, sg_select_celf, a batch
 * or a server request) ORs `flags` into its device flags after its
 * kernels, as a failing device step would, and then reports it as
 * described in the conventions above (flag 2: a bounded wait gave up,
 * SG_ETIMEOUT; flag 1: a failed check, SG_EINTERNAL).  0 clears a pending
 * injection.  No kernel is made to wait, fault or trap.
 * Errors: SG_EINVAL if flags < 0. */
sg_status sg_debug_inject_flags(int32_t flags);

/* Testing hook: the number of polls a bounded device-side wait of the
 * traversal engines makes before it gives up (an idle warp waiting for work
 * in a block-shared queue, a warp waiting for a claimed queue entry to
 * land; a claimed entry's poll sleeps 32 ns, an idle warp's poll sleeps
 * 64 ns doubling up to 1 us).  A wait that runs out sets flag 2 in
 * the query's device flags and returns, and the query reports SG_ETIMEOUT
 * as described in the conventions above; the engine's per-block state is
 * cleaned up so the next query is exact.  0 restores the default (2^22
 * polls: a few seconds at most).  Applies to queries started later, on every
 * thread.  Errors: SG_EINVAL if polls < 0. */
sg_status sg_debug_set_wait_limit(int64_t polls);

/* Free a graph handle (NULL is a no-op).  Waits for the device. */
void sg_free_graph(sg_graph *g);

/* Message describing the last failure on this thread ("" if none). */
const char *sg_last_error(void);

/* Library version string. */
const char *sg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
