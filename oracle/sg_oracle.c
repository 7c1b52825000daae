/*
 * sg_oracle.c -- plain CPU oracle for StaticGreedy and StaticGreedyDU.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes, and exists so that tests and
 * the benchmark's CPU-baseline leg can check and time against it.  Nothing
 * in the product path may include, link or call it, and it includes,
 * links and calls nothing of the product path.
 *
 * Paper: W. Cheng, H. Shen, J. Huang, G. Zhang, X. Cheng, "StaticGreedy:
 * Solving the Scalability-Accuracy Dilemma in Influence Maximization",
 * CIKM 2013 (arXiv:1212.4779).
 *
 * What is computed (all exact integers):
 *   - the independent-cascade graph of Section 3.1, with parallel arcs
 *     merged (Section 5.1, datasets footnote) and self-loops dropped;
 *   - R static snapshots (Section 3.1 "Snapshot", Algorithm 1 sampling
 *     stage): arc e is kept in snapshot r iff
 *         hi32(splitmix64(seed XOR (r << 40) XOR e)) < thr(e)
 *     where thr = floor(p * 2^32) for the uniform cascade and
 *     thr(u->v) = floor(2^32 / indeg(v)) for the weighted cascade
 *     (Section 3.4.1 / 5.1: p(u,v) = 1/d_v);
 *   - greedy selection of k seeds maximising f(S) = sum_r |R(G'_r, S)|
 *     with ties broken towards the lowest node id, by three routes:
 *       OR_LITERAL  Algorithm 1 as stated (recompute |R(G'_r, S u {v})|);
 *       OR_COVER    Algorithm 1 with the marginal gain counted directly as
 *                   |R(G'_r, v) \ R(G'_r, S)|;
 *       OR_DU       Algorithm 2 (dynamic update of Section 4);
 *       OR_CELF     lazy forward evaluation (CELF, Section 2) on the same
 *                   snapshots: StaticGreedyCELF of Section 6.
 *
 * Parity pins and readings of the paper (counted from vertex itself,
 * lowest-id tie break, DU set = newly covered nodes) are stated at each
 * function.  Snapshots are materialised as per-snapshot live out- and
 * in-lists, exactly as the paper's method stores them (Section 3.4.2:
 * space O(R' m')).
 *
 * splitmix64 is the generator of Steele, Lea and Flood, "Fast Splittable
 * Pseudorandom Number Generators" (OOPSLA 2014), with Stafford's Mix13
 * finaliser; written here from that published definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_EINVARIANT -3

enum { OR_UIC = 0, OR_WIC = 1 };
enum { OR_LITERAL = 0, OR_COVER = 1, OR_DU = 2, OR_CELF = 3 };

/* ------------------------------------------------------------------ hash */

/* SplitMix64 output function applied to x (Steele-Lea-Flood 2014). */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Coin of arc e in snapshot r (Section 3.1, "flip all coins a priori"):
 * 1 iff the arc is kept.  thr lies in [0, 2^32]; the compare is 64-bit so
 * thr = 2^32 keeps every arc and thr = 0 keeps none. */
int or_live(uint64_t seed, uint32_t r, uint64_t e, uint64_t thr)
{
    uint64_t x = seed ^ ((uint64_t)r << 40) ^ e;
    uint64_t hi = or_splitmix64(x) >> 32;
    return hi < thr;
}

/* The general form: the hash of `key` in snapshot r keeps the arc iff its
 * high 32 bits fall in [lo, hi).  The cascade models take lo = 0 and
 * key = the arc id (or_live); the linear threshold model hashes the arc's
 * destination and gives each of its in-arcs an interval of its own. */
int or_live_range(uint64_t seed, uint32_t r, uint64_t key, uint64_t lo, uint64_t hi)
{
    uint64_t h = or_splitmix64(seed ^ ((uint64_t)r << 40) ^ key) >> 32;
    return lo <= h && h < hi;
}

/* ------------------------------------------------------------- the graph */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Canonical graph of an arc list (Section 3.1 graph G; Section 5.1
 * footnote: parallel arcs are one arc).  Self-loops are dropped, repeated
 * arcs merged, and arcs ordered by (source, destination).  The canonical
 * arc id e of an arc is its position in that order, i.e. its CSR index.
 * Writes rp[n+1] and col[*m_out]; col must hold m_raw entries. */
int or_canon_coo(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                 int64_t *rp, int32_t *col, int64_t *m_out)
{
    if (n < 1 || m_raw < 0) return OR_EINVAL;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m_raw > 0 ? m_raw : 1));
    if (!key) return OR_ENOMEM;
    int64_t cnt = 0;
    for (int64_t i = 0; i < m_raw; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) { free(key); return OR_EINVAL; }
        if (src[i] == dst[i]) continue;
        key[cnt++] = ((uint64_t)(uint32_t)src[i] << 32) | (uint32_t)dst[i];
    }
    qsort(key, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < cnt; i++)
        if (i == 0 || key[i] != key[i - 1]) key[m++] = key[i];
    for (int64_t v = 0; v <= n; v++) rp[v] = 0;
    for (int64_t i = 0; i < m; i++) {
        rp[(key[i] >> 32) + 1]++;
        col[i] = (int32_t)(key[i] & 0xFFFFFFFFu);
    }
    for (int64_t v = 0; v < n; v++) rp[v + 1] += rp[v];
    *m_out = m;
    free(key);
    return OR_OK;
}

/* Propagation thresholds thr(e) in [0, 2^32] for every canonical arc.
 * UIC (uniform p, Section 5.1): thr = floor(p * 2^32), evaluated in double;
 *   multiplying by a power of two is exact, so floor() is exact too.
 * WIC (p(u,v) = 1/d_v with d_v the in-degree of v, Section 3.4.1):
 *   thr = floor(2^32 / d_v) in integer arithmetic. */
int or_thresholds(int model, double p, int64_t n, const int64_t *rp, const int32_t *col,
                  uint64_t *thr)
{
    int64_t m = rp[n];
    if (model == OR_UIC) {
        if (!(p >= 0.0 && p <= 1.0)) return OR_EINVAL;
        uint64_t t = (uint64_t)floor(p * 4294967296.0);
        for (int64_t e = 0; e < m; e++) thr[e] = t;
        return OR_OK;
    }
    if (model != OR_WIC) return OR_EINVAL;
    int64_t *indeg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!indeg) return OR_ENOMEM;
    for (int64_t e = 0; e < m; e++) indeg[col[e]]++;
    for (int64_t e = 0; e < m; e++) thr[e] = (1ULL << 32) / (uint64_t)indeg[col[e]];
    free(indeg);
    return OR_OK;
}

/* ------------------------------------------------------------- snapshots */

/* Materialised snapshots G'_0 .. G'_{R-1} (Algorithm 1 sampling stage):
 * for each r the kept arcs as out-lists and as in-lists.  Snapshots are
 * numbered from 0 (the paper counts from 1).  snaps_build(r0, R) builds the
 * R snapshots whose absolute indices are r0 .. r0+R-1; entry j of the set
 * is snapshot r0+j. */
typedef struct {
    int64_t n;
    int32_t R;
    int64_t **out_rp;
    int32_t **out_col;
    int64_t **in_rp;
    int32_t **in_col;
} or_snaps;

static void snaps_free(or_snaps *S)
{
    if (!S) return;
    for (int32_t r = 0; r < S->R; r++) {
        if (S->out_rp) free(S->out_rp[r]);
        if (S->out_col) free(S->out_col[r]);
        if (S->in_rp) free(S->in_rp[r]);
        if (S->in_col) free(S->in_col[r]);
    }
    free(S->out_rp); free(S->out_col); free(S->in_rp); free(S->in_col);
    free(S);
}

/* Coupling of a symmetric canonical graph (the undirected variant): cid[e]
 * = the lower of arc e's id and its reverse arc's id, found by binary
 * search in the reverse arc's row.  Returns OR_EINVAL if some arc has no
 * reverse. */
int or_coupled_ids(int64_t n, const int64_t *rp, const int32_t *col, int64_t *cid)
{
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int32_t v = col[e];
            int64_t lo = rp[v], hi = rp[v + 1];
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= rp[v + 1] || col[lo] != u) return OR_EINVAL;
            cid[e] = e < lo ? e : lo;
        }
    return OR_OK;
}

/* The id hashed for arc e's coin: e itself, or cid[e] when a coupling is
 * given (the undirected variant: both arcs of an edge use the lower arc id,
 * so one coin decides the edge in each snapshot, as Section 3.4.1 treats an
 * undirected snapshot). */
static uint64_t coin_of(const int64_t *cid, int64_t e) { return cid ? (uint64_t)cid[e] : (uint64_t)e; }

/* Arc e kept in snapshot r: key coin_of(cid, e), interval [lo[e], thr[e])
 * (lo NULL: [0, thr[e])). */
static int arc_live(uint64_t seed, uint32_t r, int64_t e, const uint64_t *thr, const int64_t *cid,
                    const uint64_t *lo)
{
    return or_live_range(seed, r, coin_of(cid, e), lo ? lo[e] : 0, thr[e]);
}

/* Linear threshold model in its live-edge form (Kempe, Kleinberg and Tardos,
 * KDD 2003): every node v keeps at most one of its in-arcs, arc (u, v) with
 * probability b(u, v), none with probability 1 - sum_u b(u, v); here
 * b(u, v) = 1/d_v with d_v the in-degree, the weights of the weighted
 * cascade (Section 3.4.1).  Discretised like the cascade coins: v's draw in
 * snapshot r is the high 32 bits of splitmix64(seed XOR (r << 40) XOR v);
 * v's in-arcs, in order of source (canonical arc order), own the intervals
 * [j w, (j + 1) w), w = floor(2^32 / d_v), j = 0 .. d_v - 1; the arc whose
 * interval holds the draw is kept (none when the draw is >= d_v w).  Writes
 * key[e] = destination, lo[e] = j w, hi[e] = (j + 1) w. */
int or_lt_intervals(int64_t n, const int64_t *rp, const int32_t *col, int64_t *key, uint64_t *lo, uint64_t *hi)
{
    int64_t m = rp[n];
    int64_t *indeg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *seen = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!indeg || !seen) { free(indeg); free(seen); return OR_ENOMEM; }
    for (int64_t e = 0; e < m; e++) indeg[col[e]]++;
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {  /* sources in increasing order */
            int32_t v = col[e];
            uint64_t w = (1ULL << 32) / (uint64_t)indeg[v];
            int64_t j = seen[v]++;
            key[e] = v;
            lo[e] = (uint64_t)j * w;
            hi[e] = (uint64_t)(j + 1) * w;
        }
    free(indeg); free(seen);
    return OR_OK;
}

static or_snaps *snaps_build(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
                             int32_t r0, int32_t R, uint64_t seed, int nthreads, const int64_t *cid,
                             const uint64_t *lo)
{
    or_snaps *S = (or_snaps *)calloc(1, sizeof(or_snaps));
    if (!S) return NULL;
    S->n = n; S->R = R;
    S->out_rp = (int64_t **)calloc((size_t)R, sizeof(int64_t *));
    S->out_col = (int32_t **)calloc((size_t)R, sizeof(int32_t *));
    S->in_rp = (int64_t **)calloc((size_t)R, sizeof(int64_t *));
    S->in_col = (int32_t **)calloc((size_t)R, sizeof(int32_t *));
    if (!S->out_rp || !S->out_col || !S->in_rp || !S->in_col) { snaps_free(S); return NULL; }
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int32_t r = 0; r < R; r++) {
        int64_t m = rp[n];
        int64_t *orp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        int64_t *irp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        uint8_t *keep = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
        if (!orp || !irp || !keep) { free(orp); free(irp); free(keep); failed = 1; continue; }
        int64_t kept = 0;
        for (int64_t u = 0; u < n; u++)
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                keep[e] = (uint8_t)arc_live(seed, (uint32_t)(r0 + r), e, thr, cid, lo);
                if (keep[e]) { orp[u + 1]++; irp[col[e] + 1]++; kept++; }
            }
        for (int64_t v = 0; v < n; v++) { orp[v + 1] += orp[v]; irp[v + 1] += irp[v]; }
        int32_t *ocol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kept > 0 ? kept : 1));
        int32_t *icol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kept > 0 ? kept : 1));
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        if (!ocol || !icol || !fill) {
            free(orp); free(irp); free(keep); free(ocol); free(icol); free(fill); failed = 1; continue;
        }
        int64_t o = 0;
        for (int64_t v = 0; v < n; v++) fill[v] = irp[v];
        for (int64_t u = 0; u < n; u++)
            for (int64_t e = rp[u]; e < rp[u + 1]; e++)
                if (keep[e]) { ocol[o++] = col[e]; icol[fill[col[e]]++] = (int32_t)u; }
        free(fill); free(keep);
        S->out_rp[r] = orp; S->out_col[r] = ocol; S->in_rp[r] = irp; S->in_col[r] = icol;
    }
    if (failed) { snaps_free(S); return NULL; }
    return S;
}

/* ----------------------------------------------------------- BFS helpers */

/* Per-thread scratch: epoch-stamped visited marks and a FIFO queue. */
typedef struct {
    uint32_t *mark;
    uint32_t epoch;
    int32_t *queue;
} bfs_ws;

static int ws_init(bfs_ws *w, int64_t n)
{
    w->mark = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    w->queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    w->epoch = 0;
    return (w->mark && w->queue) ? 0 : -1;
}

static void ws_free(bfs_ws *w) { free(w->mark); free(w->queue); }

static void ws_next(bfs_ws *w, int64_t n)
{
    if (++w->epoch == 0) { memset(w->mark, 0, sizeof(uint32_t) * (size_t)n); w->epoch = 1; }
}

/* |R(G'_r, sources)| restricted to nodes with blocked[x] == 0 (blocked may
 * be NULL): BFS over kept out-arcs of snapshot r.  A blocked node is
 * neither counted nor expanded.  *edges += sum of canonical out-degree of
 * every expanded node (an implementation-independent work count). */
static int64_t reach_count(const or_snaps *S, int32_t r, const int64_t *rp, int32_t nsrc,
                           const int32_t *src, const uint8_t *blocked, bfs_ws *w,
                           uint64_t *edges)
{
    ws_next(w, S->n);
    const int64_t *orp = S->out_rp[r];
    const int32_t *ocol = S->out_col[r];
    int64_t head = 0, tail = 0;
    for (int32_t i = 0; i < nsrc; i++) {
        int32_t v = src[i];
        if (blocked && blocked[v]) continue;
        if (w->mark[v] == w->epoch) continue;
        w->mark[v] = w->epoch;
        w->queue[tail++] = v;
    }
    while (head < tail) {
        int32_t u = w->queue[head++];
        if (edges) *edges += (uint64_t)(rp[u + 1] - rp[u]);
        for (int64_t j = orp[u]; j < orp[u + 1]; j++) {
            int32_t x = ocol[j];
            if (w->mark[x] == w->epoch) continue;
            if (blocked && blocked[x]) continue;
            w->mark[x] = w->epoch;
            w->queue[tail++] = x;
        }
    }
    return tail;
}

/* --------------------------------------------------------- initial gains */

/* Initial marginal gains s_v = sum_r |R(G'_r, v)| (Algorithm 2, first
 * loop; |R| counts v itself, since a seed is active).  *init_edges is the
 * snapshot-edge count sum_{r,v} sum_{u in R(G'_r,v)} outdeg(u). */
static int init_gains(const or_snaps *S, const int64_t *rp, int nthreads, int64_t *s,
                      uint64_t *init_edges)
{
    int64_t n = S->n;
    uint64_t edges = 0;
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : edges)
#endif
    {
        bfs_ws w;
        if (ws_init(&w, n) != 0) {
            failed = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t v = 0; v < n; v++) {
                int32_t vv = (int32_t)v;
                int64_t acc = 0;
                for (int32_t r = 0; r < S->R; r++)
                    acc += reach_count(S, r, rp, 1, &vv, NULL, &w, &edges);
                s[v] = acc;
            }
        }
        ws_free(&w);
    }
    *init_edges = edges;
    return failed ? OR_ENOMEM : OR_OK;
}

/* argmax over v not in S of s_v; ties go to the lowest id (the paper only
 * says argmax; this reading makes the result unique).  Seeds are excluded
 * even when every remaining gain is 0. */
static int32_t argmax_not_seed(int64_t n, const int64_t *s, const uint8_t *is_seed)
{
    int32_t best = -1;
    for (int64_t v = 0; v < n; v++) {
        if (is_seed[v]) continue;
        if (best < 0 || s[v] > s[best]) best = (int32_t)v;
    }
    return best;
}

/* ------------------------------------------------- CELF priority queue */

/* Binary max-heap of (bound, id, stamp) ordered by bound descending, then
 * id ascending. */
typedef struct {
    int64_t *b;
    int32_t *v, *stamp;
    int64_t size;
} or_heap;

static int heap_before(const or_heap *h, int64_t x, int64_t y)
{
    return h->b[x] > h->b[y] || (h->b[x] == h->b[y] && h->v[x] < h->v[y]);
}

static void heap_swap(or_heap *h, int64_t x, int64_t y)
{
    int64_t tb = h->b[x]; h->b[x] = h->b[y]; h->b[y] = tb;
    int32_t tv = h->v[x]; h->v[x] = h->v[y]; h->v[y] = tv;
    int32_t ts = h->stamp[x]; h->stamp[x] = h->stamp[y]; h->stamp[y] = ts;
}

static int heap_init(or_heap *h, int64_t cap)
{
    h->b = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    h->v = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    h->stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    h->size = 0;
    return (h->b && h->v && h->stamp) ? 0 : -1;
}

static void heap_free(or_heap *h)
{
    free(h->b); free(h->v); free(h->stamp);
    h->b = NULL; h->v = NULL; h->stamp = NULL;
}

static void heap_push(or_heap *h, int64_t b, int32_t v, int32_t stamp)
{
    int64_t i = h->size++;
    h->b[i] = b; h->v[i] = v; h->stamp[i] = stamp;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_before(h, i, p)) break;
        heap_swap(h, i, p);
        i = p;
    }
}

static void heap_pop(or_heap *h, int64_t *b, int32_t *v, int32_t *stamp)
{
    *b = h->b[0]; *v = h->v[0]; *stamp = h->stamp[0];
    h->size--;
    if (h->size > 0) {
        h->b[0] = h->b[h->size]; h->v[0] = h->v[h->size]; h->stamp[0] = h->stamp[h->size];
        int64_t i = 0;
        for (;;) {
            int64_t l = 2 * i + 1, r = l + 1, m = i;
            if (l < h->size && heap_before(h, l, m)) m = l;
            if (r < h->size && heap_before(h, r, m)) m = r;
            if (m == i) break;
            heap_swap(h, i, m);
            i = m;
        }
    }
}

/* ------------------------------------------------------------- selection */

/* Greedy seed selection on static snapshots.
 *   mode OR_LITERAL: Algorithm 1.  Round i: s_v = sum_r |R(G'_r, S u {v})|
 *     for v not in S; v* = argmax; gain_i = s_{v*} - f(S).
 *   mode OR_COVER: Algorithm 1 with s_v = sum_r |R(G'_r, v) \ Cov_r|,
 *     Cov_r = R(G'_r, S): the BFS from v neither counts nor expands covered
 *     nodes, which is exact because everything a covered node reaches is
 *     covered.  gain_i = s_{v*}.
 *   mode OR_DU: Algorithm 2.  s starts at the initial gains; each round
 *     v* = argmax, gain_i = s_{v*}; then for each snapshot r, N_r = the
 *     nodes reached from v* that are not yet covered (the "current" R set
 *     of v*, which excludes nodes earlier seeds already cover); for each
 *     w in N_r, every u in U(G'_r, w) (BFS over kept in-arcs from w, w
 *     included) has s_u decremented by one; then Cov_r gains N_r.  The
 *     reverse BFS must never visit a node covered before this round (such
 *     a node would reach w, so w would already be covered); a visit returns
 *     OR_EINVARIANT.
 *   mode OR_CELF: s starts at the initial gains, which are exact upper
 *     bounds of every later marginal gain (submodularity, Section 3.1).
 *     The candidates sit in a priority queue ordered by (bound descending,
 *     id ascending).  Round i pops the head; if its bound was computed in
 *     round i it is the round's seed (every other candidate's gain is at
 *     most its bound, and an equal bound comes with a larger id), else its
 *     marginal gain sum_r |R(G'_r, v) \ Cov_r| is computed as in OR_COVER
 *     (one evaluation) and it goes back with that bound.  Round 0 uses the
 *     initial gains as computed in round 0.
 * Outputs seeds[k], gains[k].  Optional: s_init[n] (initial gains, DU,
 * COVER and CELF), s_hist[k*n] (the gain vector after each DU round, seeds'
 * entries included), counters[4] = {init, forward, reverse} snapshot-edge
 * counts of the DU route (forward: sum over expanded (u,r) of outdeg(u);
 * reverse: sum over visited (u,w,r) of indeg(u)) and, for OR_CELF, the
 * number of marginal-gain evaluations after the initial gains. */
int or_select(int mode, int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
              int32_t R, int32_t k, uint64_t seed, int nthreads, int32_t *seeds, int64_t *gains,
              int64_t *s_init, int64_t *s_hist, uint64_t *counters, const int64_t *cid, const uint64_t *lo)
{
    if (n < 1 || R < 1 || k < 1 || k > n) return OR_EINVAL;
    or_snaps *S = snaps_build(n, rp, col, thr, 0, R, seed, nthreads, cid, lo);
    if (!S) return OR_ENOMEM;
    int rc = OR_OK;
    int64_t *s = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    uint8_t *is_seed = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *cov = (uint8_t *)calloc((size_t)n * (size_t)R, 1); /* 0 no, 1 old, 2 new */
    int64_t *indeg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    bfs_ws w;
    if (!s || !is_seed || !cov || !indeg || ws_init(&w, n) != 0) {
        free(s); free(is_seed); free(cov); free(indeg); snaps_free(S);
        return OR_ENOMEM;
    }
    for (int64_t e = 0; e < rp[n]; e++) indeg[col[e]]++;
    uint64_t c_init = 0, c_fwd = 0, c_rev = 0;
    int64_t f_S = 0; /* f(S) of the current seed set */

    if (mode == OR_DU || mode == OR_COVER || mode == OR_CELF) {
        rc = init_gains(S, rp, nthreads, s, &c_init);
        if (rc != OR_OK) goto done;
        if (s_init) memcpy(s_init, s, sizeof(int64_t) * (size_t)n);
    }
    uint64_t c_eval = 0;
    or_heap H = {0};
    if (mode == OR_CELF) {
        if (heap_init(&H, n) != 0) { rc = OR_ENOMEM; goto done; }
        for (int64_t v = 0; v < n; v++) heap_push(&H, s[v], (int32_t)v, 0);
    }

    for (int32_t i = 0; i < k; i++) {
        if (mode == OR_LITERAL) {
            int32_t *set = (int32_t *)malloc(sizeof(int32_t) * (size_t)(i + 1));
            if (!set) { rc = OR_ENOMEM; goto done; }
            for (int32_t j = 0; j < i; j++) set[j] = seeds[j];
            for (int64_t v = 0; v < n; v++) {
                if (is_seed[v]) continue;
                set[i] = (int32_t)v;
                int64_t acc = 0;
                for (int32_t r = 0; r < R; r++)
                    acc += reach_count(S, r, rp, i + 1, set, NULL, &w, NULL);
                s[v] = acc;
            }
            free(set);
        } else if (mode == OR_COVER && i > 0) {
            for (int64_t v = 0; v < n; v++) {
                if (is_seed[v]) continue;
                int32_t vv = (int32_t)v;
                int64_t acc = 0;
                for (int32_t r = 0; r < R; r++)
                    acc += reach_count(S, r, rp, 1, &vv, cov + (size_t)r * (size_t)n, &w, NULL);
                s[v] = acc;
            }
        }
        int32_t vs;
        if (mode == OR_CELF) {
            for (;;) {
                int64_t b; int32_t v, stamp;
                heap_pop(&H, &b, &v, &stamp);
                if (stamp == i) { s[v] = b; vs = v; break; }
                int64_t acc = 0;
                for (int32_t r = 0; r < R; r++)
                    acc += reach_count(S, r, rp, 1, &v, cov + (size_t)r * (size_t)n, &w, NULL);
                c_eval++;
                heap_push(&H, acc, v, i);
            }
        } else {
            vs = argmax_not_seed(n, s, is_seed);
        }
        seeds[i] = vs;
        gains[i] = (mode == OR_LITERAL) ? s[vs] - f_S : s[vs];
        f_S += gains[i];
        is_seed[vs] = 1;

        for (int32_t r = 0; r < R; r++) {
            uint8_t *cr = cov + (size_t)r * (size_t)n;
            const int64_t *orp = S->out_rp[r];
            const int32_t *ocol = S->out_col[r];
            /* N_r: forward BFS from v* that neither enters nor counts covered nodes */
            int64_t head = 0, tail = 0;
            if (cr[vs] == 0) { cr[vs] = 2; w.queue[tail++] = vs; }
            while (head < tail) {
                int32_t u = w.queue[head++];
                c_fwd += (uint64_t)(rp[u + 1] - rp[u]);
                for (int64_t j = orp[u]; j < orp[u + 1]; j++) {
                    int32_t x = ocol[j];
                    if (cr[x] != 0) continue;
                    cr[x] = 2;
                    w.queue[tail++] = x;
                }
            }
            if (mode == OR_DU) {
                /* queue[0 .. tail) holds N_r; reverse BFS from each member */
                int64_t nnew = tail;
                int32_t *newlist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnew > 0 ? nnew : 1));
                if (!newlist) { rc = OR_ENOMEM; goto done; }
                memcpy(newlist, w.queue, sizeof(int32_t) * (size_t)nnew);
                const int64_t *irp = S->in_rp[r];
                const int32_t *icol = S->in_col[r];
                for (int64_t t = 0; t < nnew; t++) {
                    ws_next(&w, n);
                    int64_t h2 = 0, t2 = 0;
                    w.mark[newlist[t]] = w.epoch;
                    w.queue[t2++] = newlist[t];
                    while (h2 < t2) {
                        int32_t u = w.queue[h2++];
                        if (cr[u] == 1) { rc = OR_EINVARIANT; free(newlist); goto done; }
                        s[u] -= 1;
                        c_rev += (uint64_t)indeg[u];
                        for (int64_t j = irp[u]; j < irp[u + 1]; j++) {
                            int32_t x = icol[j];
                            if (w.mark[x] == w.epoch) continue;
                            w.mark[x] = w.epoch;
                            w.queue[t2++] = x;
                        }
                    }
                }
                free(newlist);
            }
            for (int64_t x = 0; x < n; x++)
                if (cr[x] == 2) cr[x] = 1;
        }
        if (s_hist && mode == OR_DU) memcpy(s_hist + (size_t)i * (size_t)n, s, sizeof(int64_t) * (size_t)n);
    }
    if (counters) { counters[0] = c_init; counters[1] = c_fwd; counters[2] = c_rev; counters[3] = c_eval; }
done:
    heap_free(&H);
    ws_free(&w);
    free(s); free(is_seed); free(cov); free(indeg);
    snaps_free(S);
    return rc;
}

/* Initial gains only (Algorithm 2 first loop) over the snapshots with
 * absolute indices r0 .. r1-1, with their init snapshot-edge count.  Used
 * to time a bounded slice of the snapshots; r0 = 0, r1 = R gives the full
 * initial gains. */
int or_init_gains(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
                  int32_t r0, int32_t r1, uint64_t seed, int nthreads, int64_t *s,
                  uint64_t *init_edges, const int64_t *cid, const uint64_t *lo)
{
    if (n < 1 || r0 < 0 || r1 <= r0) return OR_EINVAL;
    or_snaps *S = snaps_build(n, rp, col, thr, r0, r1 - r0, seed, nthreads, cid, lo);
    if (!S) return OR_ENOMEM;
    int rc = init_gains(S, rp, nthreads, s, init_edges);
    snaps_free(S);
    return rc;
}

/* ------------------------------------------ on-demand coins (no storage) */

/* |R(G'_r, sources)| with every arc's coin flipped when the BFS first looks
 * at the arc instead of from a stored snapshot.  The coin of (e, r) is the
 * same function either way, so this equals reach_count on the stored
 * snapshot; it lets full-size graphs be checked without O(R m') storage.
 * mark/queue: n-entry scratch, mark zeroed by the caller. */
static int64_t reach_fly(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
                         uint64_t seed, uint32_t r, int32_t nsrc, const int32_t *src,
                         uint8_t *mark, int32_t *queue, uint64_t *edges, const int64_t *cid,
                         const uint64_t *lo)
{
    int64_t head = 0, tail = 0;
    for (int32_t i = 0; i < nsrc; i++)
        if (!mark[src[i]]) { mark[src[i]] = 1; queue[tail++] = src[i]; }
    while (head < tail) {
        int32_t u = queue[head++];
        if (edges) *edges += (uint64_t)(rp[u + 1] - rp[u]);
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
            int32_t x = col[e];
            if (mark[x]) continue;
            if (!arc_live(seed, r, e, thr, cid, lo)) continue;
            mark[x] = 1;
            queue[tail++] = x;
        }
    }
    for (int64_t i = 0; i < tail; i++) mark[queue[i]] = 0;
    (void)n;
    return tail;
}

/* f(S) = sum_r |R(G'_r, S)| (Section 3.1: the snapshot estimate of I(S),
 * times R), with on-demand coins; snapshots in parallel.  *edges (if not
 * NULL) gets the snapshot-edge count sum_r sum_{u in R(G'_r, S)} outdeg(u). */
int64_t or_spread(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
                  int32_t R, uint64_t seed, int32_t nS, const int32_t *Sset, int nthreads,
                  uint64_t *edges, const int64_t *cid, const uint64_t *lo)
{
    int64_t total = 0;
    uint64_t ed = 0;
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : total, ed)
#endif
    {
        uint8_t *mark = (uint8_t *)calloc((size_t)n, 1);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!mark || !queue) {
            failed = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int32_t r = 0; r < R; r++)
                total += reach_fly(n, rp, col, thr, seed, (uint32_t)r, nS, Sset, mark, queue, &ed, cid, lo);
        }
        free(mark); free(queue);
    }
    if (edges) *edges = ed;
    return failed ? (int64_t)OR_ENOMEM : total;
}

/* sum_r |R(G'_r, v)| for each listed v (initial gains of a sample of
 * sources), with on-demand coins; *edges gets the init snapshot-edge count
 * of those sources. */
int or_reach_sums(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *thr,
                  int32_t R, uint64_t seed, int32_t nv, const int32_t *v, int nthreads,
                  int64_t *out, uint64_t *edges, const int64_t *cid, const uint64_t *lo)
{
    uint64_t ed = 0;
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : ed)
#endif
    {
        uint8_t *mark = (uint8_t *)calloc((size_t)n, 1);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!mark || !queue) {
            failed = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int32_t i = 0; i < nv; i++) {
                int64_t acc = 0;
                for (int32_t r = 0; r < R; r++)
                    acc += reach_fly(n, rp, col, thr, seed, (uint32_t)r, 1, v + i, mark, queue, &ed, cid, lo);
                out[i] = acc;
            }
        }
        free(mark); free(queue);
    }
    if (edges) *edges = ed;
    return failed ? OR_ENOMEM : OR_OK;
}

/* Coins as 64-snapshot words: bit b of masks[e*W + w] is the coin of arc e
 * in snapshot 64w+b, for snapshots < R (higher bits of the last word 0). */
int or_live_masks(int64_t m, const uint64_t *thr, int32_t R, uint64_t seed, uint64_t *masks,
                  const int64_t *cid, const uint64_t *lo)
{
    int32_t W = (R + 63) / 64;
    for (int64_t e = 0; e < m; e++)
        for (int32_t w = 0; w < W; w++) {
            uint64_t word = 0;
            for (int32_t b = 0; b < 64; b++) {
                int32_t r = 64 * w + b;
                if (r < R && arc_live(seed, (uint32_t)r, e, thr, cid, lo)) word |= 1ULL << b;
            }
            masks[e * W + w] = word;
        }
    return OR_OK;
}
