// sg_celf.cu -- StaticGreedyCELF: greedy selection on the static snapshots
// with lazy forward evaluation (CELF of Leskovec et al., Section 2; the
// StaticGreedyCELF variant timed in Section 6) instead of the dynamic
// update.  The initial gains come from the same kernels as sg_select; the
// candidates then wait in a host priority queue ordered by (bound
// descending, id ascending).  A round pops the head: a bound computed in
// this round makes it the seed (every other candidate's gain is at most its
// bound, and an equal bound comes with a larger id, so this is the lowest-id
// argmax), otherwise its marginal gain sum_r |R(G'_r, v) \ Cov_r| is
// computed on the GPU -- a walk from v over a copy of the coverage bits --
// and it goes back with that bound.  The seed's walk over the coverage
// itself then marks what it newly covers.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <queue>
#include <vector>

#include "sg_internal.cuh"

using namespace sgi;

namespace {

struct CelfEntry {
    long long bound;
    int32_t v;
    int32_t stamp;  // round in which the bound was computed
};

// priority_queue keeps the "largest" on top: lower bound, then larger id,
// ranks lower
struct CelfLess {
    bool operator()(const CelfEntry &a, const CelfEntry &b) const
    {
        return a.bound < b.bound || (a.bound == b.bound && a.v > b.v);
    }
};

// One walk from v over the W words into vis; returns the newly reached
// (node, snapshot) pairs and their out-degree sum.
sg_status walk_from(sg_graph *g, sg_workspace &ws, const Coins &co, int model, int heavy_on, int32_t v,
                    unsigned long long *vis, long long *d_cnt, int32_t *d_v, long long *h_cnt, cudaStream_t st)
{
    SG_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 16, st));
    SG_CUDA_TRY(cudaMemcpyAsync(d_v, &v, 4, cudaMemcpyHostToDevice, st));
    SG_TRY(run_walk(g, ws, co, model, heavy_on, d_v, 1, vis, ws.pendf.p, ws.fq_a.p, ws.fq_b.p, d_cnt,
                    reinterpret_cast<unsigned long long *>(d_cnt + 1), st));
    SG_CUDA_TRY(cudaMemcpyAsync(h_cnt, d_cnt, 16, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    return SG_OK;
}

sg_status celf_impl(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, cudaStream_t st,
                    int32_t *out_seeds, int64_t *out_gains, int64_t *out_evals, sg_stats *stats)
{
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    const int model = c.model == SG_WIC ? MODEL_WIC : MODEL_UIC;
    const int launches0 = g_launches;
    sg_workspace &ws = g->ws;
    const size_t n = (size_t)g->n, nw = n * (size_t)co.W;
    SG_TRY(ensure_workspace(g, ws, co.W, k, st));
    // the linear threshold model reads every coin from the live-mask cache
    const int heavy_on = (!co.lt && heavy_index_enabled(g, co.W)) ? 1 : 0;
    if (heavy_on) SG_TRY(ensure_heavy_index(g, ws, co.W, st));
    ws.slists_on = 0;
    // every per-query cache is rebuilt for this query's coins
    ws.fl_on = 0;
    if (heavy_on) SG_TRY(ensure_fwd_lists(g, ws, co, c.p, model, st));
    SG_TRY(ensure_mask_cache(g, ws, co.W, st, co.lt != 0));

    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard()
        {
            for (int i = 0; i < 3; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    if (stats)
        for (auto &e : ev) SG_CUDA_TRY(cudaEventCreate(&e));
    if (stats) SG_CUDA_TRY(cudaEventRecord(ev[0], st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.s.p, 0, n * sizeof(long long), st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.cov.p, 0, nw * 8, st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, sizeof(Ctl), st));
    if (heavy_on) {
        SG_TRY(run_heavy_index(g, ws, co, model, st));
        if (ws.fl_on) SG_TRY(run_fwd_lists(g, ws, co, st));
        SG_TRY(run_row_desc(g, ws, co, st));
        ws.rd_on = 1;
    }
    if (ws.lm_on) SG_TRY(run_mask_cache(g, ws, co, model, st));
    SG_TRY(run_init_gains(g, ws, co, model, heavy_on, st, nullptr));
    SG_TRY(plant_injected_flags(ws, st));
    if (stats) SG_CUDA_TRY(cudaEventRecord(ev[1], st));
    std::vector<long long> s0(n);
    Ctl h;
    SG_CUDA_TRY(cudaMemcpyAsync(s0.data(), ws.s.p, n * 8, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    SG_TRY(flags_status(h.flags));

    // scratch: the coverage copy of an evaluation, two counters, the source
    DBuf<unsigned long long> scratch;
    DBuf<long long> cnt;
    DBuf<int32_t> dv;
    struct BufGuard {
        DBuf<unsigned long long> &a;
        DBuf<long long> &b;
        DBuf<int32_t> &c;
        cudaStream_t st;
        ~BufGuard()
        {
            dbuf_free(a, st);
            dbuf_free(b, st);
            dbuf_free(c, st);
        }
    } bufs{scratch, cnt, dv, st};
    SG_TRY(dbuf_alloc(scratch, nw, st));
    SG_TRY(dbuf_alloc(cnt, 2, st));
    SG_TRY(dbuf_alloc(dv, 1, st));

    std::vector<CelfEntry> heap;
    heap.reserve(n);
    for (size_t v = 0; v < n; ++v) heap.push_back(CelfEntry{s0[v], (int32_t)v, 0});
    std::priority_queue<CelfEntry, std::vector<CelfEntry>, CelfLess> pq(CelfLess(), std::move(heap));
    std::vector<int32_t> seeds((size_t)k);
    std::vector<int64_t> gains((size_t)k);
    long long evals = 0;
    unsigned long long fwd_edges = 0;
    long long hc[2];
    for (int32_t i = 0; i < k; ++i) {
        CelfEntry top;
        while (true) {
            top = pq.top();
            pq.pop();
            if (top.stamp == i) break;
            SG_CUDA_TRY(cudaMemcpyAsync(scratch.p, ws.cov.p, nw * 8, cudaMemcpyDeviceToDevice, st));
            SG_TRY(walk_from(g, ws, co, model, heavy_on, top.v, scratch.p, cnt.p, dv.p, hc, st));
            ++evals;
            pq.push(CelfEntry{hc[0], top.v, i});
        }
        seeds[(size_t)i] = top.v;
        gains[(size_t)i] = top.bound;
        SG_TRY(walk_from(g, ws, co, model, heavy_on, top.v, ws.cov.p, cnt.p, dv.p, hc, st));
        if (hc[0] != top.bound) {
            set_error("sg_select_celf: seed %d newly covers %lld, its gain was %lld", top.v, hc[0], top.bound);
            return SG_EINTERNAL;
        }
        fwd_edges += (unsigned long long)hc[1];
    }
    if (stats) {
        SG_CUDA_TRY(cudaEventRecord(ev[2], st));
        SG_CUDA_TRY(cudaEventSynchronize(ev[2]));
    }
    SG_CUDA_TRY(cudaMemcpy(out_seeds, seeds.data(), (size_t)k * 4, cudaMemcpyDefault));
    SG_CUDA_TRY(cudaMemcpy(out_gains, gains.data(), (size_t)k * 8, cudaMemcpyDefault));
    if (out_evals) *out_evals = evals;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->init_edges = h.init_edges;
        stats->fwd_edges = fwd_edges;
        stats->init_tier2_tasks = h.init_t2;
        stats->init_tier3_tasks = h.init_t3;
        stats->kernel_launches = g_launches - launches0;
        stats->heavy_index = heavy_on;
        stats->mask_cache = ws.lm_on;
        memcpy(stats->work_keys, h.work_keys, sizeof(h.work_keys));
        memcpy(stats->work_elems, h.work_elems, sizeof(h.work_elems));
        cudaEventElapsedTime(&stats->ms_init, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_rounds, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_total, ev[0], ev[2]);
    }
    return SG_OK;
}

}  // namespace

extern "C" sg_status sg_select_celf(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                                    int32_t *out_seeds, int64_t *out_gains, int64_t *out_evals, sg_stats *stats)
{
    clear_error();
    SG_TRY(check_query(g, R, k));
    if (!out_seeds || !out_gains) {
        set_error("sg_select_celf: output pointers must be non-NULL");
        return SG_EINVAL;
    }
    if (c.model == SG_UIC_UNDIRECTED) {
        set_error("sg_select_celf: the undirected cascade is served by sg_select (component bookkeeping)");
        return SG_EINVAL;
    }
    DeviceGuard dg(g->device);
    return celf_impl(g, R, k, c, seed, (cudaStream_t)stream, out_seeds, out_gains, out_evals, stats);
}
