// sg_host.cu -- host side of the C ABI: errors, device memory hooks, graph
// loading (canonicalisation, CSC, WIC thresholds) and the selection driver.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <thread>
#include <vector>

#include "sg_graph_build.h"
#include "sg_internal.cuh"

namespace sgi {

// ------------------------------------------------------------------ errors
namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// ------------------------------------------------------------ device flags
namespace {
// flags the next query plants into its device flags (sg_debug_inject_flags)
std::atomic<int> g_inject_flags{0};

__global__ void set_flags_kernel(Ctl *ctl, int flags) { atomicOr(&ctl->flags, flags); }

__global__ void poison_kernel(const Ctl *ctl, int32_t *seeds, long long *vals, long long count)
{
    const int32_t f = *(volatile const int32_t *)&ctl->flags;
    if (!f) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        if (seeds) seeds[i] = -1;
        vals[i] = -(long long)f;
    }
}
}  // namespace

sg_status flags_status(int32_t flags)
{
    if (!flags) return SG_OK;
    if (flags & FLAG_WAIT) {
        set_error("a bounded device-side wait gave up (device flags 0x%x)", flags);
        return SG_ETIMEOUT;
    }
    set_error("device-side check failed (device flags 0x%x)", flags);
    return SG_EINTERNAL;
}

sg_status plant_injected_flags(sg_workspace &ws, cudaStream_t st)
{
    const int f = g_inject_flags.exchange(0);
    if (!f) return SG_OK;
    set_flags_kernel<<<1, 1, 0, st>>>(ws.ctl.p, f);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

sg_status run_poison(const sg_graph *g, sg_workspace &ws, int32_t *seeds, long long *vals, long long count,
                     cudaStream_t st)
{
    if (count <= 0) return SG_OK;
    const int blocks = (int)std::min<long long>((count + 255) / 256, (long long)g->num_sms * 4);
    poison_kernel<<<blocks, 256, 0, st>>>(ws.ctl.p, seeds, vals, count);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

// ------------------------------------------------------------------ memory
int g_snapshot_lists = 1;
int g_mask_cache = 0;
int g_fwd_lists = 1;
int g_walk_groups = 64;
int g_word_major = 1;
int g_t1_direct = 16;

Knobs knobs()
{
    if (t_knobs) return *t_knobs;
    Knobs k;
    k.walk_groups = g_walk_groups;
    k.bu_mode = g_bu_mode;
    k.bu_div = g_bu_div;
    k.t1_keys = g_tier_limit[0];
    k.t2_keys = g_tier_limit[1];
    k.landmarks = g_landmarks;
    k.scc = g_scc;
    k.fwd_lists = g_fwd_lists;
    k.word_major = g_word_major;
    k.t1_direct = g_t1_direct;
    return k;
}

namespace {
int g_heavy_min_deg = 2;
sg_alloc_fn g_alloc = nullptr;
sg_release_fn g_release = nullptr;
void *g_alloc_ctx = nullptr;
}  // namespace

thread_local int g_builtin_alloc = 0;

void *dalloc(size_t bytes, cudaStream_t st)
{
    if (g_alloc && !g_builtin_alloc) return g_alloc(bytes, st, g_alloc_ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dfree(void *p, size_t bytes, cudaStream_t st)
{
    if (!p) return;
    if (g_release && !g_builtin_alloc) {
        g_release(p, bytes, st, g_alloc_ctx);
        return;
    }
    cudaFreeAsync(p, st);
}

void free_workspace(sg_workspace &ws, cudaStream_t st);
sg_status ensure_wic(sg_graph *g, cudaStream_t st);

namespace {

// Workers for host-side passes over rows.
__global__ void build_fw_kernel(long long m, const int32_t *col, const uint32_t *tmi, uint2 *fw)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
         e += (long long)gridDim.x * blockDim.x) {
        const int32_t y = col[e];
        fw[e] = make_uint2((uint32_t)y, tmi[y]);
    }
}

template <class T>
sg_status upload(sgi::DBuf<T> &b, const T *host, size_t count, cudaStream_t st)
{
    SG_TRY(dbuf_alloc(b, count, st));
    if (count) SG_CUDA_TRY(cudaMemcpyAsync(b.p, host, count * sizeof(T), cudaMemcpyHostToDevice, st));
    return SG_OK;
}

void free_graph_buffers(sg_graph *g, cudaStream_t st)
{
    free_workspace(g->ws, st);
    dbuf_free(g->rp, st);
    dbuf_free(g->col, st);
    dbuf_free(g->crp, st);
    dbuf_free(g->cin, st);
    dbuf_free(g->tmi, st);
    dbuf_free(g->fw, st);
    dbuf_free(g->hid_out, st);
    dbuf_free(g->hrow_out, st);
    dbuf_free(g->hpref_out, st);
    dbuf_free(g->hid_in, st);
    dbuf_free(g->hrow_in, st);
    dbuf_free(g->hpref_in, st);
    dbuf_free(g->cc_esrc, st);
    dbuf_free(g->cc_pmin, st);
}

// Heavy rows of one direction (row offsets rp): degree >= min_deg.
struct HeavyHost {
    std::vector<int32_t> hid, hrow;
    std::vector<long long> hpref;
};

HeavyHost heavy_rows(int64_t n, const sgh::hvec<int32_t> &rp, int min_deg)
{
    HeavyHost h;
    h.hid.assign((size_t)n, -1);
    h.hpref.push_back(0);
    if (min_deg <= 0) return h;
    for (int64_t v = 0; v < n; ++v) {
        const int d = rp[(size_t)v + 1] - rp[(size_t)v];
        if (d >= min_deg) {
            h.hid[(size_t)v] = (int32_t)h.hrow.size();
            h.hrow.push_back((int32_t)v);
            h.hpref.push_back(h.hpref.back() + d);
        }
    }
    return h;
}

// Build a graph handle from a canonical CSR held on the host.
sg_status finish_load(int64_t n, sgh::hvec<int32_t> &rp, sgh::hvec<int32_t> &col, cudaStream_t st,
                      sg_graph **out)
{
    const int64_t m = rp[(size_t)n];
    // CSC by a stable counting sort on destination: in-arcs of each node in
    // increasing (source, arc id) order
    sgh::hvec<int32_t> crp;
    sgh::hvec<sgh::Arc2> cin;
    sgh::build_csc(n, rp, col, crp, cin);
    static_assert(sizeof(sgh::Arc2) == sizeof(int2), "CSC entries upload as int2");
    std::vector<uint32_t> tmi((size_t)n);
    sgh::parallel_rows(n, [&](int64_t a, int64_t b) {
        for (int64_t v = a; v < b; ++v) {
            const int64_t d = crp[(size_t)v + 1] - crp[(size_t)v];
            tmi[(size_t)v] = d > 0 ? (uint32_t)((1ull << 32) / (uint64_t)d - 1ull) : 0xffffffffu;
        }
    });
    sg_graph *g = new (std::nothrow) sg_graph();
    if (!g) {
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    g->n = n;
    g->m = m;
    sg_status rc = SG_OK;
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        cudaGetLastError();
        set_error("no usable CUDA device");
        delete g;
        return SG_ECUDA;
    }
    const HeavyHost ho = heavy_rows(n, rp, g_heavy_min_deg);
    const HeavyHost hi = heavy_rows(n, crp, g_heavy_min_deg);
    g->heavy_min_deg = g_heavy_min_deg;
    {
        // landmarks: the 8 largest out-degrees (at least 32), lowest id first on ties
        std::vector<std::pair<int32_t, int32_t>> top;  // (degree, node)
        for (int64_t v = 0; v < n; ++v) {
            const int32_t d = rp[(size_t)v + 1] - rp[(size_t)v];
            if (d < 32) continue;
            if (top.size() < 8 || d > top.back().first) {
                top.emplace_back(d, (int32_t)v);
                std::stable_sort(top.begin(), top.end(),
                                 [](const std::pair<int32_t, int32_t> &x, const std::pair<int32_t, int32_t> &y) {
                                     return x.first > y.first;
                                 });
                if (top.size() > 8) top.pop_back();
            }
        }
        g->lmk_count = (int32_t)top.size();
        for (size_t i = 0; i < top.size(); ++i) g->lmk_nodes[i] = top[i].second;
    }
    g->nh_out = (int32_t)ho.hrow.size();
    g->nh_in = (int32_t)hi.hrow.size();
    {
        // expected live out-arcs per snapshot over the indexed rows under
        // the weighted cascade (sizes the forward per-snapshot lists); 64
        // fixed parts summed in order, so the value does not depend on the
        // host's thread count
        constexpr int P = 64;
        std::vector<double> part(P, 0.0);
        const size_t nr = ho.hrow.size(), pc = (nr + P - 1) / P;
        const int PT = std::min(P, sgh::host_threads());
        sgh::parallel_parts(PT, [&](int t) {
            for (int q = t; q < P; q += PT) {
                double acc = 0.0;
                for (size_t i = q * pc; i < std::min(nr, (q + 1) * pc); ++i) {
                    const int32_t x = ho.hrow[i];
                    for (int32_t e = rp[(size_t)x]; e < rp[(size_t)x + 1]; ++e) {
                        const int32_t y = col[(size_t)e];
                        acc += 1.0 / (double)(crp[(size_t)y + 1] - crp[(size_t)y]);
                    }
                }
                part[(size_t)q] = acc;
            }
        });
        double acc = 0.0;
        for (double v : part) acc += v;
        g->hlive_out_wic = acc;
    }
    g->hsum_out = ho.hpref.back();
    g->hsum_in = hi.hpref.back();
    if ((rc = upload(g->rp, rp.data(), (size_t)n + 1, st)) != SG_OK ||
        (rc = upload(g->col, col.data(), (size_t)m, st)) != SG_OK ||
        (rc = upload(g->crp, crp.data(), (size_t)n + 1, st)) != SG_OK ||
        (rc = upload(g->cin, reinterpret_cast<const int2 *>(cin.data()), (size_t)m, st)) != SG_OK ||
        (rc = upload(g->tmi, tmi.data(), (size_t)n, st)) != SG_OK ||
        (rc = upload(g->hid_out, ho.hid.data(), ho.hid.size(), st)) != SG_OK ||
        (rc = upload(g->hrow_out, ho.hrow.data(), ho.hrow.size(), st)) != SG_OK ||
        (rc = upload(g->hpref_out, ho.hpref.data(), ho.hpref.size(), st)) != SG_OK ||
        (rc = upload(g->hid_in, hi.hid.data(), hi.hid.size(), st)) != SG_OK ||
        (rc = upload(g->hrow_in, hi.hrow.data(), hi.hrow.size(), st)) != SG_OK ||
        (rc = upload(g->hpref_in, hi.hpref.data(), hi.hpref.size(), st)) != SG_OK) {
        free_graph_buffers(g, st);
        delete g;
        return rc;
    }
    if ((rc = ensure_wic(g, st)) != SG_OK) {
        free_graph_buffers(g, st);
        delete g;
        return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        free_graph_buffers(g, st);
        delete g;
        return SG_ECUDA;
    }
    *out = g;
    return SG_OK;
}

bool is_pageable(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeUnregistered;
}

}  // namespace

void free_workspace(sg_workspace &ws, cudaStream_t st)
{
    dbuf_free(ws.s, st);
    dbuf_free(ws.cov, st);
    dbuf_free(ws.nbits, st);
    dbuf_free(ws.pendf, st);
    dbuf_free(ws.fq_a, st);
    dbuf_free(ws.fq_b, st);
    dbuf_free(ws.du_x, st);
    dbuf_free(ws.list1, st);
    dbuf_free(ws.list2, st);
    dbuf_free(ws.tl, st);
    dbuf_free(ws.toff, st);
    dbuf_free(ws.coff, st);
    dbuf_free(ws.tcnt, st);
    dbuf_free(ws.du_cnt, st);
    dbuf_free(ws.anc, st);
    dbuf_free(ws.frw, st);
    dbuf_free(ws.anc_list, st);
    dbuf_free(ws.anc_cnt, st);
    dbuf_free(ws.lmk_rx, st);
    dbuf_free(ws.lmk_ux, st);
    dbuf_free(ws.lmk_any, st);
    dbuf_free(ws.lmk_U, st);
    dbuf_free(ws.lmk_H, st);
    dbuf_free(ws.lmk_E, st);
    dbuf_free(ws.lmk_HE, st);
    dbuf_free(ws.hcnt_out, st);
    dbuf_free(ws.hnbr_out, st);
    dbuf_free(ws.hmask_out, st);
    dbuf_free(ws.hcnt_in, st);
    dbuf_free(ws.hnbr_in, st);
    dbuf_free(ws.hmask_in, st);
    dbuf_free(ws.soff, st);
    dbuf_free(ws.snbr, st);
    dbuf_free(ws.svalid, st);
    dbuf_free(ws.scan_tmp, st);
    ws.soff_cap = 0;
    ws.snbr_cap = 0;
    ws.slists_on = 0;
    ws.hw_cap = 0;
    dbuf_free(ws.lm_out, st);
    dbuf_free(ws.lm_in, st);
    ws.lm_cap = 0;
    dbuf_free(ws.rdesc, st);
    ws.rd_cap = 0;
    ws.rd_on = 0;
    dbuf_free(ws.cc_lab, st);
    dbuf_free(ws.cc_size, st);
    dbuf_free(ws.cc_deg, st);
    dbuf_free(ws.cc_cov, st);
    dbuf_free(ws.cc_root, st);
    ws.cc_cap = 0;
    ws.cc_rcap = 0;
    dbuf_free(ws.fsoff, st);
    dbuf_free(ws.fscan, st);
    dbuf_free(ws.fsnbr, st);
    dbuf_free(ws.fsvalid, st);
    ws.fsoff_cap = 0;
    ws.fsnbr_cap = 0;
    ws.fl_on = 0;
    ws.lm_on = 0;
    dbuf_free(ws.slot_vis, st);
    dbuf_free(ws.slot_qa, st);
    dbuf_free(ws.slot_touched, st);
    dbuf_free(ws.ctl, st);
    dbuf_free(ws.am_gain, st);
    dbuf_free(ws.am_id, st);
    dbuf_free(ws.out_seeds, st);
    dbuf_free(ws.out_gains, st);
    ws.wcap = 0;
    ws.kcap = 0;
    ws.nslots = 0;
}

GraphView view_of(const sg_graph *g, const sg_workspace &ws, int heavy_on)
{
    GraphView v;
    v.n = (int32_t)g->n;
    v.m = g->m;
    v.rp = g->rp.p;
    v.col = g->col.p;
    v.fw = g->fw.p;
    v.crp = g->crp.p;
    v.cin = g->cin.p;
    v.tmi = g->tmi.p;
    v.hout = HeavyView{g->hid_out.p, g->hpref_out.p, ws.hcnt_out.p, ws.hnbr_out.p, ws.hmask_out.p,
                       nullptr, nullptr, nullptr};
    v.hin = HeavyView{g->hid_in.p, g->hpref_in.p, ws.hcnt_in.p, ws.hnbr_in.p, ws.hmask_in.p,
                      ws.slists_on ? ws.soff.p : nullptr, ws.snbr.p, ws.svalid.p};
    v.heavy_on = heavy_on;
    v.lm_out = ws.lm_on ? ws.lm_out.p : nullptr;
    v.lm_in = ws.lm_on ? ws.lm_in.p : nullptr;
    v.lm_w0 = 0;
    v.rdesc = (heavy_on && ws.rd_on) ? ws.rdesc.p : nullptr;
    const bool fl = heavy_on && ws.fl_on;
    v.fsoff = fl ? ws.fsoff.p : nullptr;
    v.fsnbr = fl ? ws.fsnbr.p : nullptr;
    v.fsvalid = fl ? ws.fsvalid.p : nullptr;
    return v;
}

// The live-mask cache takes 2 x W x m x 8 bytes (both arc orders); it is
// built while that stays within 16 GiB.
size_t mask_cache_bytes(const sg_graph *g, int32_t W)
{
    return (size_t)2 * (size_t)W * (size_t)g->m * 8;
}

static bool mask_cache_fits(const sg_graph *g, int32_t W)
{
    return g_mask_cache && g->m > 0 && mask_cache_bytes(g, W) <= ((size_t)16 << 30);
}

sg_status ensure_mask_cache(sg_graph *g, sg_workspace &ws, int32_t W, cudaStream_t st, bool required)
{
    ws.lm_on = 0;
    if (required && g->m > 0 && mask_cache_bytes(g, W) > ((size_t)16 << 30)) {
        set_error("the linear threshold model needs the live-mask cache (2 x W x m x 8 = %zu bytes > 16 GiB)",
                  mask_cache_bytes(g, W));
        return SG_ENOMEM;
    }
    if (!required && !mask_cache_fits(g, W)) return SG_OK;
    if (g->m == 0) return SG_OK;
    if (ws.lm_cap < W) {
        dbuf_free(ws.lm_out, st);
        dbuf_free(ws.lm_in, st);
        ws.lm_cap = 0;
        SG_TRY(dbuf_alloc(ws.lm_out, (size_t)W * (size_t)g->m, st));
        SG_TRY(dbuf_alloc(ws.lm_in, (size_t)W * (size_t)g->m, st));
        ws.lm_cap = W;
    }
    ws.lm_on = 1;
    return SG_OK;
}

// The heavy-row index reserves (sum of heavy degrees) x W entries of 12 B
// per direction; it is used while that stays within 8 GiB.
bool heavy_index_enabled(const sg_graph *g, int32_t W)
{
    if (g->heavy_min_deg <= 0 || (g->nh_out == 0 && g->nh_in == 0)) return false;
    const double bytes = (double)(g->hsum_out + g->hsum_in) * (double)W * 12.0;
    return bytes <= 8.0 * (double)(1ull << 30);
}

sg_status ensure_heavy_index(sg_graph *g, sg_workspace &ws, int32_t W, cudaStream_t st)
{
    ws.rd_on = 0;
    if (ws.rd_cap < W) {
        dbuf_free(ws.rdesc, st);
        ws.rd_cap = 0;
        SG_TRY(dbuf_alloc(ws.rdesc, (size_t)W * (size_t)g->n * 2, st));
        ws.rd_cap = W;
    }
    if (ws.hw_cap >= W) return SG_OK;
    dbuf_free(ws.hcnt_out, st);
    dbuf_free(ws.hnbr_out, st);
    dbuf_free(ws.hmask_out, st);
    dbuf_free(ws.hcnt_in, st);
    dbuf_free(ws.hnbr_in, st);
    dbuf_free(ws.hmask_in, st);
    dbuf_free(ws.soff, st);
    dbuf_free(ws.snbr, st);
    dbuf_free(ws.svalid, st);
    dbuf_free(ws.scan_tmp, st);
    ws.soff_cap = 0;
    ws.snbr_cap = 0;
    ws.slists_on = 0;
    ws.hw_cap = 0;
    SG_TRY(dbuf_alloc(ws.hcnt_out, (size_t)g->nh_out * W, st));
    SG_TRY(dbuf_alloc(ws.hnbr_out, (size_t)g->hsum_out * W, st));
    SG_TRY(dbuf_alloc(ws.hmask_out, (size_t)g->hsum_out * W, st));
    SG_TRY(dbuf_alloc(ws.hcnt_in, (size_t)g->nh_in * W, st));
    SG_TRY(dbuf_alloc(ws.hnbr_in, (size_t)g->hsum_in * W, st));
    SG_TRY(dbuf_alloc(ws.hmask_in, (size_t)g->hsum_in * W, st));
    ws.hw_cap = W;
    return SG_OK;
}

sg_status ensure_wic(sg_graph *g, cudaStream_t st)
{
    if (g->fw.p || g->m == 0) return SG_OK;
    SG_TRY(dbuf_alloc(g->fw, (size_t)g->m, st));
    const int blocks = (int)std::min<long long>((g->m + 255) / 256, (long long)g->num_sms * 8);
    build_fw_kernel<<<blocks, 256, 0, st>>>(g->m, g->col.p, g->tmi.p, g->fw.p);
    SG_CUDA_TRY(cudaGetLastError());
    ++g_launches;
    return SG_OK;
}

// Tier-3 slot memory: 4 KB per node per resident dense block per SM (48 KB
// at twelve), between 64 MB and 16 GiB per three blocks (64 GiB at twelve).
size_t tier3_budget(int64_t n)
{
    // about 24 bytes per node per slot, 4 KB per node for each block per
    // SM: every graph up to about 1.3 M nodes gets its full count of slots
    // (tier-3 tasks are latency-bound, so the number of resident blocks
    // sets their throughput)
    const size_t b = (size_t)n * 4096 * SG_DENSE_BLOCKS;
    const size_t cap = ((size_t)16 << 30) * (size_t)std::max(1, SG_DENSE_BLOCKS / 3);
    return std::min<size_t>(cap, std::max<size_t>((size_t)64 << 20, b));
}

// Device bytes a workspace for (W, k) takes, as ensure_workspace /
// ensure_heavy_index / ensure_snapshot_lists allocate them (upper bound).
size_t workspace_bytes(const sg_graph *g, int32_t W, int32_t k)
{
    const size_t n = (size_t)g->n, nw = n * (size_t)W, W64 = (size_t)64 * W;
    size_t b = 8 * n;                                  // s
    b += 8 * nw * 4;                                   // cov, nbits, pendf, bottom-up frontier
    b += 4 * nw * (size_t)std::max(8, knobs().walk_groups) * 2;  // forward queues
    b += 4 * nw;                                       // du_x
    b += 4 * (nw + W64 + 64) * 2;                      // task lists
    b += 4 * nw * 64;                                  // per-snapshot targets
    b += (8 + 8 + 4) * W64 + 4 * (size_t)W;            // offsets, counts
    b += 8 * nw + (4 * nw + 4 * (size_t)W) * (size_t)std::max(8, knobs().walk_groups);  // ancestors, lists
    b += 2 * 8 * nw * 8 + (W64 << 8) * (4 + 4 + 8 + 8);  // landmarks
    int qcap = 1;
    while ((size_t)qcap < n) qcap <<= 1;
    const size_t per_slot = n * 20 + (size_t)qcap * 4;
    const size_t slots = std::max<size_t>(1, std::min<size_t>((size_t)g->num_sms * SG_DENSE_BLOCKS, tier3_budget(g->n) / per_slot));
    b += slots * per_slot;
    b += (size_t)g->num_sms * 2 * 12 + (size_t)k * 12 + 4096;
    if (heavy_index_enabled(g, W)) {
        b += (size_t)(g->hsum_out + g->hsum_in) * W * 12 + (size_t)(g->nh_out + g->nh_in) * W * 4;
        b += (size_t)g->n * W * 32;  // forward row descriptors
        {
            // forward per-snapshot lists (upper bound: WIC expectation or all arcs)
            const size_t nq = (size_t)g->n * 64 * W + 1;
            const double want = 1.5 * 64.0 * W * std::max(g->hlive_out_wic, 0.1 * (double)g->hsum_out) + (1u << 20);
            const double fb = want * 4.0 + (double)(2 * nq + nq / 1024 + 16) * 8.0;
            if (knobs().fwd_lists && fb <= 8.0 * (double)(1ull << 30)) b += (size_t)fb;
        }
        const size_t nq = (size_t)g->nh_in * W64 + 1;
        b += nq * 16 + ((size_t)1 << 20) * 4 + (size_t)(1.5 * 64.0 * W * (double)g->nh_in) * 4;
    }
    if (mask_cache_fits(g, W)) b += mask_cache_bytes(g, W);
    return b;
}

sg_status ensure_workspace(sg_graph *g, sg_workspace &ws, int32_t W, int32_t k, cudaStream_t st)
{
    const int64_t n = g->n;
    if (ws.wcap < W) {
        free_workspace(ws, st);
        const size_t nw = (size_t)n * (size_t)W;
        SG_TRY(dbuf_alloc(ws.s, (size_t)n, st));
        SG_TRY(dbuf_alloc(ws.cov, nw, st));
        SG_TRY(dbuf_alloc(ws.nbits, nw, st));
        SG_TRY(dbuf_alloc(ws.pendf, nw, st));
        // one level queue per (word, walk group)
        ws.fq_groups = std::max(8, knobs().walk_groups);
        SG_TRY(dbuf_alloc(ws.fq_a, nw * (size_t)ws.fq_groups, st));
        SG_TRY(dbuf_alloc(ws.fq_b, nw * (size_t)ws.fq_groups, st));
        SG_TRY(dbuf_alloc(ws.du_x, nw, st));
        const size_t ltasks = nw + (size_t)64 * W + 64;
        SG_TRY(dbuf_alloc(ws.list1, ltasks, st));
        SG_TRY(dbuf_alloc(ws.list2, ltasks, st));
        SG_TRY(dbuf_alloc(ws.tl, nw * 64, st));
        SG_TRY(dbuf_alloc(ws.toff, (size_t)64 * W, st));
        SG_TRY(dbuf_alloc(ws.coff, (size_t)64 * W + 1, st));
        SG_TRY(dbuf_alloc(ws.tcnt, (size_t)64 * W, st));
        SG_TRY(dbuf_alloc(ws.du_cnt, (size_t)W, st));
        SG_TRY(dbuf_alloc(ws.anc, nw, st));
        SG_TRY(dbuf_alloc(ws.frw, nw, st));
        // one list of marked ancestors per (word, walk group)
        SG_TRY(dbuf_alloc(ws.anc_list, nw * (size_t)ws.fq_groups, st));
        SG_TRY(dbuf_alloc(ws.anc_cnt, (size_t)W * (size_t)ws.fq_groups, st));
        SG_TRY(dbuf_alloc(ws.lmk_rx, nw * 8, st));
        SG_TRY(dbuf_alloc(ws.lmk_ux, nw * 8, st));
        SG_TRY(dbuf_alloc(ws.lmk_any, nw, st));
        SG_TRY(dbuf_alloc(ws.lmk_U, ((size_t)64 * W) << 8, st));
        SG_TRY(dbuf_alloc(ws.lmk_H, ((size_t)64 * W) << 8, st));
        SG_TRY(dbuf_alloc(ws.lmk_E, ((size_t)64 * W) << 8, st));
        SG_TRY(dbuf_alloc(ws.lmk_HE, ((size_t)64 * W) << 8, st));
        SG_TRY(dbuf_alloc(ws.ctl, 1, st));

        SG_CUDA_TRY(cudaMemsetAsync(ws.nbits.p, 0, ws.nbits.bytes, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.pendf.p, 0, ws.pendf.bytes, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.frw.p, 0, ws.frw.bytes, st));
        // tier-3 slots: dense per-slot arrays (vis, pend, ring queue, touched), <= ~16 GiB in total
        int qcap = 1;
        while (qcap < n) qcap <<= 1;
        const size_t per_slot = (size_t)n * (2 * sizeof(unsigned long long) + sizeof(int32_t)) + (size_t)qcap * 4;
        const size_t budget = tier3_budget(n);
        int slots = (int)std::max<size_t>(1, std::min<size_t>((size_t)g->num_sms * SG_DENSE_BLOCKS, budget / per_slot));
        const size_t ns = (size_t)slots * (size_t)n;
        SG_TRY(dbuf_alloc(ws.slot_vis, 2 * ns, st));  // per node: visited and pending words side by side
        SG_TRY(dbuf_alloc(ws.slot_qa, (size_t)slots * (size_t)qcap, st));
        SG_TRY(dbuf_alloc(ws.slot_touched, ns, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.slot_vis.p, 0, ws.slot_vis.bytes, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.slot_qa.p, 0xff, ws.slot_qa.bytes, st));
        ws.slot_qmask = qcap - 1;
        ws.am_blocks = g->num_sms * 2;
        SG_TRY(dbuf_alloc(ws.am_gain, (size_t)ws.am_blocks, st));
        SG_TRY(dbuf_alloc(ws.am_id, (size_t)ws.am_blocks, st));
        ws.nslots = slots;
        ws.wcap = W;
        ws.n = n;
    }
    if (ws.kcap < k) {
        dbuf_free(ws.out_seeds, st);
        dbuf_free(ws.out_gains, st);
        SG_TRY(dbuf_alloc(ws.out_seeds, (size_t)k, st));
        SG_TRY(dbuf_alloc(ws.out_gains, (size_t)k, st));
        ws.kcap = k;
    }
    return SG_OK;
}

// Per-snapshot live in-lists of heavy rows.  Their total size is a random
// count with mean R * sum over heavy in-arcs of p(arc) (WIC: R per heavy
// row); the list buffer holds 1.5x that plus slack, and if a query exceeds
// it the device flag marks the lists invalid and the reverse tasks use the
// per-word index instead.  Skipped when the buffer would pass 2 GiB.
sg_status ensure_snapshot_lists(sg_graph *g, sg_workspace &ws, const Coins &co, double p_uic, int model,
                                cudaStream_t st)
{
    ws.slists_on = 0;
    if (g->nh_in == 0) return SG_OK;
    const double R = 64.0 * co.W;
    const double expect = model == MODEL_WIC ? R * (double)g->nh_in : R * p_uic * (double)g->hsum_in;
    const size_t want = (size_t)(expect * 1.5) + (1u << 20);
    const size_t nq = (size_t)g->nh_in * 64 * co.W + 1;
    if ((double)want * 4.0 + (double)nq * 16.0 > 2.0 * (double)(1ull << 30)) return SG_OK;
    if (ws.soff_cap < nq) {
        dbuf_free(ws.soff, st);
        dbuf_free(ws.scan_tmp, st);
        SG_TRY(dbuf_alloc(ws.soff, nq, st));
        SG_TRY(dbuf_alloc(ws.scan_tmp, nq + nq / 1024 + 16, st));
        ws.soff_cap = nq;
    }
    if (ws.snbr_cap < want) {
        dbuf_free(ws.snbr, st);
        SG_TRY(dbuf_alloc(ws.snbr, want, st));
        ws.snbr_cap = want;
    }
    if (!ws.svalid.p) SG_TRY(dbuf_alloc(ws.svalid, 1, st));
    ws.slists_on = 1;
    return SG_OK;
}

// Forward per-snapshot live lists of the indexed out-rows, node-indexed
// (offsets for n * 64W (node, snapshot) pairs).  The list buffer holds 1.5x
// the expected live (arc, snapshot) pairs plus slack; a query that exceeds
// it marks the lists invalid and expands through the index instead.
// Skipped when offsets, counts and lists would pass 8 GiB.
sg_status ensure_fwd_lists(sg_graph *g, sg_workspace &ws, const Coins &co, double p_uic, int model,
                           cudaStream_t st)
{
    ws.fl_on = 0;
    if (!knobs().fwd_lists || g->nh_out == 0) return SG_OK;
    const double R = 64.0 * co.W;
    const double expect = model == MODEL_WIC ? R * g->hlive_out_wic : R * p_uic * (double)g->hsum_out;
    const size_t want = (size_t)(expect * 1.5) + (1u << 20);
    const size_t nq = (size_t)g->n * 64 * co.W + 1;
    const size_t scan = nq + nq / 1024 + 16;
    if ((double)want * 4.0 + (double)(nq + scan) * 8.0 > 8.0 * (double)(1ull << 30)) return SG_OK;
    if (ws.fsoff_cap < nq) {
        dbuf_free(ws.fsoff, st);
        dbuf_free(ws.fscan, st);
        ws.fsoff_cap = 0;
        SG_TRY(dbuf_alloc(ws.fsoff, nq, st));
        SG_TRY(dbuf_alloc(ws.fscan, scan, st));
        ws.fsoff_cap = nq;
    }
    if (ws.fsnbr_cap < want) {
        dbuf_free(ws.fsnbr, st);
        ws.fsnbr_cap = 0;
        SG_TRY(dbuf_alloc(ws.fsnbr, want, st));
        ws.fsnbr_cap = want;
    }
    if (!ws.fsvalid.p) SG_TRY(dbuf_alloc(ws.fsvalid, 1, st));
    ws.fl_on = 1;
    return SG_OK;
}

sg_status make_coins(const sg_cascade &c, uint64_t seed, int32_t R, Coins *out)
{
    if (R < 1 || R >= (1 << 24)) {
        set_error("R must satisfy 1 <= R < 2^24 (got %d)", R);
        return SG_EINVAL;
    }
    Coins co;
    co.seed = seed;
    co.R = R;
    co.W = (R + 63) / 64;
    co.none_live = 0;
    co.uic_tm1 = 0xffffffffu;
    co.lt = 0;
    if (c.model == SG_UIC || c.model == SG_UIC_UNDIRECTED) {
        if (!(c.p >= 0.0 && c.p <= 1.0)) {
            set_error("UIC probability must lie in [0, 1]");
            return SG_EINVAL;
        }
        // thr = floor(p * 2^32) in [0, 2^32]; multiplying by 2^32 is exact
        const uint64_t thr = (uint64_t)std::floor(c.p * 4294967296.0);
        if (thr == 0) co.none_live = 1;
        else co.uic_tm1 = (uint32_t)(thr - 1);
    } else if (c.model == SG_LT) {
        co.lt = 1;  // per-node draws, materialised into the live-mask cache
    } else if (c.model != SG_WIC) {
        set_error("unknown cascade model %d", c.model);
        return SG_EINVAL;
    }
    *out = co;
    return SG_OK;
}

}  // namespace sgi

using namespace sgi;

namespace sgi {

sg_status check_query(const sg_graph *g, int32_t R, int32_t k)
{
    if (!g) {
        set_error("graph handle is NULL");
        return SG_EINVAL;
    }
    if (k < 1 || k > g->n) {
        set_error("k must satisfy 1 <= k <= n (k=%d, n=%lld)", k, (long long)g->n);
        return SG_EINVAL;
    }
    const int64_t W = ((int64_t)R + 63) / 64;
    if (R >= 1 && (g->n + 1) * W * 64 > (int64_t)INT32_MAX * 16) {
        set_error("n * ceil(R/64) too large for the per-snapshot target lists");
        return SG_EINVAL;
    }
    if (R >= 1 && g->n * W + 64 * W > (int64_t)INT32_MAX) {
        set_error("n * ceil(R/64) must stay below 2^31");
        return SG_EINVAL;
    }
    return SG_OK;
}

}  // namespace sgi

extern "C" {

const char *sg_last_error(void) { return g_err; }

const char *sg_version(void) { return "sg 0.1 (sm_103a)"; }

sg_status sg_set_heavy_threshold(int32_t min_degree)
{
    if (min_degree < 0) {
        set_error("heavy threshold must be >= 0");
        return SG_EINVAL;
    }
    g_heavy_min_deg = min_degree;
    return SG_OK;
}

sg_status sg_set_engine_limits(int32_t tier1_keys, int32_t tier2_keys)
{
    if (tier1_keys < 1 || tier2_keys < 1) {
        set_error("engine limits must be >= 1");
        return SG_EINVAL;
    }
    g_tier_limit[0] = tier1_keys;
    g_tier_limit[1] = tier2_keys;
    return SG_OK;
}

sg_status sg_set_snapshot_lists(int32_t enable)
{
    if (enable < 0 || enable > 1) {
        set_error("enable must be 0 or 1");
        return SG_EINVAL;
    }
    g_snapshot_lists = enable;
    return SG_OK;
}

sg_status sg_graph_trim(sg_graph *g)
{
    clear_error();
    if (!g) {
        set_error("sg_graph_trim: NULL graph");
        return SG_EINVAL;
    }
    DeviceGuard dg(g->device);
    SG_CUDA_TRY(cudaDeviceSynchronize());
    free_workspace(g->ws, (cudaStream_t)0);
    SG_CUDA_TRY(cudaDeviceSynchronize());
    return SG_OK;
}

sg_status sg_set_direction(int32_t mode, int32_t divisor)
{
    if (mode < 0 || mode > 2 || divisor < 1) {
        set_error("direction mode must be 0, 1 or 2 and the divisor >= 1 (got %d, %d)", mode, divisor);
        return SG_EINVAL;
    }
    g_bu_mode = mode;
    g_bu_div = divisor;
    return SG_OK;
}

sg_status sg_set_scc_condensation(int32_t enable)
{
    if (enable != 0 && enable != 1) {
        set_error("SCC condensation switch must be 0 or 1");
        return SG_EINVAL;
    }
    g_scc = enable;
    return SG_OK;
}

sg_status sg_set_walk_groups(int32_t groups)
{
    if (groups != 8 && groups != 16 && groups != 32 && groups != 64) {
        set_error("walk groups must be 8, 16, 32 or 64, got %d", groups);
        return SG_EINVAL;
    }
    g_walk_groups = groups;
    return SG_OK;
}

sg_status sg_set_forward_lists(int32_t enable)
{
    if (enable != 0 && enable != 1) {
        set_error("forward lists switch must be 0 or 1");
        return SG_EINVAL;
    }
    g_fwd_lists = enable;
    return SG_OK;
}

sg_status sg_set_mask_cache(int32_t enable)
{
    if (enable != 0 && enable != 1) {
        set_error("mask cache switch must be 0 or 1");
        return SG_EINVAL;
    }
    g_mask_cache = enable;
    return SG_OK;
}

sg_status sg_set_landmarks(int32_t count)
{
    if (count < 0 || count > 8) {
        set_error("landmark count must be in [0, 8]");
        return SG_EINVAL;
    }
    g_landmarks = count;
    return SG_OK;
}

sg_status sg_set_allocator(sg_alloc_fn alloc, sg_release_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) {
        set_error("alloc and release must both be set or both be NULL");
        return SG_EINVAL;
    }
    g_alloc = alloc;
    g_release = release;
    g_alloc_ctx = ctx;
    return SG_OK;
}

sg_status sg_load_graph(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, int is_device_ptr,
                        void *stream, sg_graph **out)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!out || n < 1 || n >= (int64_t)INT32_MAX || m < 0 || m >= (int64_t)INT32_MAX || !row_ptr ||
        (m > 0 && !col)) {
        set_error("sg_load_graph: need 1 <= n < 2^31, 0 <= m < 2^31 and non-NULL arrays");
        return SG_EINVAL;
    }
    // host arrays are read in place; device arrays are copied to the host
    std::vector<int64_t> rp_copy;
    std::vector<int32_t> c_copy;
    const int64_t *rp = row_ptr;
    const int32_t *c = col;
    if (is_device_ptr) {
        rp_copy.resize((size_t)n + 1);
        c_copy.resize((size_t)std::max<int64_t>(1, m));
        SG_CUDA_TRY(cudaMemcpyAsync(rp_copy.data(), row_ptr, rp_copy.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    st));
        if (m) SG_CUDA_TRY(cudaMemcpyAsync(c_copy.data(), col, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        rp = rp_copy.data();
        c = c_copy.data();
    }
    if (rp[0] != 0 || rp[(size_t)n] != m) {
        set_error("sg_load_graph: row_ptr[0] must be 0 and row_ptr[n] must be m");
        return SG_EINVAL;
    }
    const int64_t bu = sgh::parallel_first(n, [&](int64_t u) { return rp[(size_t)u + 1] < rp[(size_t)u]; });
    if (bu < n) {
        set_error("sg_load_graph: row_ptr decreases at row %lld", (long long)bu);
        return SG_EINVAL;
    }
    const int64_t be = sgh::parallel_first(m, [&](int64_t e) { return c[(size_t)e] < 0 || c[(size_t)e] >= n; });
    if (be < m) {
        set_error("sg_load_graph: col[%lld] = %d out of range", (long long)be, c[(size_t)be]);
        return SG_EINVAL;
    }
    sgh::hvec<int32_t> rpc, colc;
    sgh::canonicalise(n, rp, c, rpc, colc);
    return finish_load(n, rpc, colc, st, out);
}

sg_status sg_load_graph_coo(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int is_device_ptr,
                            void *stream, sg_graph **out)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!out || n < 1 || n >= (int64_t)INT32_MAX || m < 0 || m >= (int64_t)INT32_MAX ||
        (m > 0 && (!src || !dst))) {
        set_error("sg_load_graph_coo: need 1 <= n < 2^31, 0 <= m < 2^31 and non-NULL arrays");
        return SG_EINVAL;
    }
    std::vector<int32_t> s((size_t)std::max<int64_t>(1, m)), d((size_t)std::max<int64_t>(1, m));
    if (m) {
        if (is_device_ptr) {
            SG_CUDA_TRY(cudaMemcpyAsync(s.data(), src, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
            SG_CUDA_TRY(cudaMemcpyAsync(d.data(), dst, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
            SG_CUDA_TRY(cudaStreamSynchronize(st));
        } else {
            memcpy(s.data(), src, (size_t)m * 4);
            memcpy(d.data(), dst, (size_t)m * 4);
        }
    }
    std::vector<int64_t> rp((size_t)n + 1, 0);
    for (int64_t i = 0; i < m; ++i) {
        if (s[(size_t)i] < 0 || s[(size_t)i] >= n || d[(size_t)i] < 0 || d[(size_t)i] >= n) {
            set_error("sg_load_graph_coo: arc %lld has an endpoint out of range", (long long)i);
            return SG_EINVAL;
        }
        rp[(size_t)s[(size_t)i] + 1]++;
    }
    for (int64_t u = 0; u < n; ++u) rp[(size_t)u + 1] += rp[(size_t)u];
    std::vector<int32_t> c((size_t)std::max<int64_t>(1, m));
    {
        std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
        for (int64_t i = 0; i < m; ++i) c[(size_t)fill[(size_t)s[(size_t)i]]++] = d[(size_t)i];
    }
    sgh::hvec<int32_t> rpc, colc;
    sgh::canonicalise(n, rp.data(), c.data(), rpc, colc);
    return finish_load(n, rpc, colc, st, out);
}

sg_status sg_graph_info(const sg_graph *g, int64_t *n, int64_t *m_canonical)
{
    if (!g) {
        set_error("graph handle is NULL");
        return SG_EINVAL;
    }
    if (n) *n = g->n;
    if (m_canonical) *m_canonical = g->m;
    return SG_OK;
}

sg_status sg_graph_csr(const sg_graph *g, void *stream, int64_t *row_ptr, int32_t *col)
{
    clear_error();
    if (!g || !row_ptr || (g->m > 0 && !col)) {
        set_error("sg_graph_csr: NULL argument");
        return SG_EINVAL;
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> rp((size_t)g->n + 1);
    SG_CUDA_TRY(cudaMemcpyAsync(rp.data(), g->rp.p, rp.size() * 4, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> rp64(rp.begin(), rp.end());
    SG_CUDA_TRY(cudaMemcpyAsync(row_ptr, rp64.data(), rp64.size() * 8, cudaMemcpyDefault, st));
    if (g->m) SG_CUDA_TRY(cudaMemcpyAsync(col, g->col.p, (size_t)g->m * 4, cudaMemcpyDefault, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    return SG_OK;
}

void sg_free_graph(sg_graph *g)
{
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    free_graph_buffers(g, (cudaStream_t)0);
    cudaDeviceSynchronize();
    delete g;
}

}  // extern "C"

namespace sgi {

// The undirected variant (one coin per edge): Algorithm 2 by component
// bookkeeping (sg_cc.cu).  Same outputs, counters and statuses as the
// general path.  The first query on a graph checks its symmetry (one
// host synchronisation); prepare_only sizes the workspace.
sg_status cc_select_impl(sg_graph *g, sg_workspace &ws, const Coins &co, int32_t k, cudaStream_t st,
                         int32_t *out_seeds, int64_t *out_gains, sg_stats *stats, bool prepare_only)
{
    SG_TRY(cc_prepare_graph(g, st));
    const int launches0 = g_launches;
    SG_TRY(ensure_workspace(g, ws, co.W, k, st));
    SG_TRY(cc_ensure(g, ws, co.R, st));
    if (prepare_only) return SG_OK;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard()
        {
            for (int i = 0; i < 3; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    if (stats) {
        for (auto &e : ev) SG_CUDA_TRY(cudaEventCreate(&e));
        SG_CUDA_TRY(cudaEventRecord(ev[0], st));
    }
    SG_CUDA_TRY(cudaMemsetAsync(ws.s.p, 0, (size_t)g->n * sizeof(long long), st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, sizeof(Ctl), st));
    SG_TRY(cc_clear_cover(g, ws, co, st));
    SG_TRY(cc_init_gains(g, ws, co, st));
    if (stats) SG_CUDA_TRY(cudaEventRecord(ev[1], st));
    for (int32_t i = 0; i < k; ++i) {
        SG_TRY(run_argmax(g, ws, co, i, st));
        SG_TRY(cc_round(g, ws, co, st));
    }
    SG_TRY(plant_injected_flags(ws, st));
    SG_TRY(run_poison(g, ws, ws.out_seeds.p, ws.out_gains.p, k, st));
    SG_CUDA_TRY(cudaMemcpyAsync(out_seeds, ws.out_seeds.p, (size_t)k * 4, cudaMemcpyDefault, st));
    SG_CUDA_TRY(cudaMemcpyAsync(out_gains, ws.out_gains.p, (size_t)k * 8, cudaMemcpyDefault, st));
    if (stats) {
        SG_CUDA_TRY(cudaEventRecord(ev[2], st));
        Ctl h;
        SG_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        memset(stats, 0, sizeof(*stats));
        stats->init_edges = h.init_edges;
        stats->fwd_edges = h.fwd_edges;
        stats->rev_edges = h.rev_edges;
        stats->status_flags = h.flags;
        stats->kernel_launches = g_launches - launches0;
        cudaEventElapsedTime(&stats->ms_init, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_rounds, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_total, ev[0], ev[2]);
        return flags_status(h.flags);
    }
    if (is_pageable(out_seeds) || is_pageable(out_gains)) {
        int32_t fl = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&fl, &ws.ctl.p->flags, 4, cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        return flags_status(fl);
    }
    return SG_OK;
}

// Algorithm 2 end to end on graph g with workspace ws.  prepare_only: size
// the workspace for the query (allocations happen here) and launch nothing.
sg_status select_impl(sg_graph *g, sg_workspace &ws, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                      int32_t *out_seeds, int64_t *out_gains, sg_stats *stats, bool prepare_only)
{
    SG_TRY(check_query(g, R, k));
    if (!out_seeds || !out_gains) {
        set_error("sg_select: output pointers must be non-NULL");
        return SG_EINVAL;
    }
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c.model == SG_UIC_UNDIRECTED)
        return cc_select_impl(g, ws, co, k, st, out_seeds, out_gains, stats, prepare_only);
    const int model = c.model == SG_WIC ? MODEL_WIC : MODEL_UIC;
    const int launches0 = g_launches;
    SG_TRY(ensure_workspace(g, ws, co.W, k, st));
    // the linear threshold model reads every coin from the live-mask cache
    const int heavy_on = (!co.lt && heavy_index_enabled(g, co.W)) ? 1 : 0;
    if (heavy_on) SG_TRY(ensure_heavy_index(g, ws, co.W, st));
    ws.slists_on = 0;
    if (heavy_on && g_snapshot_lists) SG_TRY(ensure_snapshot_lists(g, ws, co, c.p, model, st));
    ws.fl_on = 0;
    if (heavy_on) SG_TRY(ensure_fwd_lists(g, ws, co, c.p, model, st));
    SG_TRY(ensure_mask_cache(g, ws, co.W, st, co.lt != 0));
    ws.walk_groups = std::min(knobs().walk_groups, ws.fq_groups);
    if (prepare_only) return SG_OK;
    // events: 0 start, 1 after index, 2 after init tier 1, 3 after init,
    // 4 end; per round: after forward update
    std::vector<cudaEvent_t> ev;
    auto mark = [&](void) -> cudaEvent_t {
        cudaEvent_t e = nullptr;
        if (!stats) return nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ev.push_back(e);
        return e;
    };
    struct EvGuard {
        std::vector<cudaEvent_t> &v;
        ~EvGuard()
        {
            for (auto e : v) cudaEventDestroy(e);
        }
    } guard{ev};
    cudaEvent_t e_start = mark(), e_index = mark(), e_init = mark(), e_end = mark();
    TierEvents tev;
    tev.start = mark();
    tev.t1 = mark();
    tev.t2 = mark();
    tev.t3 = mark();
    std::vector<cudaEvent_t> e_round(stats ? (size_t)k + 1 : 0), e_fwd(stats ? (size_t)k : 0);
    if (stats) {
        for (auto &e : e_round) e = mark();
        for (auto &e : e_fwd) e = mark();
        SG_CUDA_TRY(cudaEventRecord(e_start, st));
    }
    SG_CUDA_TRY(cudaMemsetAsync(ws.s.p, 0, (size_t)g->n * sizeof(long long), st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.cov.p, 0, (size_t)g->n * (size_t)co.W * 8, st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.anc.p, 0, (size_t)g->n * (size_t)co.W * 8, st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.anc_cnt.p, 0, (size_t)co.W * (size_t)ws.fq_groups * 4, st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, sizeof(Ctl), st));
    if (heavy_on) {
        SG_TRY(run_heavy_index(g, ws, co, model, st));
        if (ws.fl_on) SG_TRY(run_fwd_lists(g, ws, co, st));
        SG_TRY(run_row_desc(g, ws, co, st));
        ws.rd_on = 1;
    }
    if (ws.slists_on) SG_TRY(run_snapshot_lists(g, ws, co, st));
    if (ws.lm_on) SG_TRY(run_mask_cache(g, ws, co, model, st));
    if (stats) SG_CUDA_TRY(cudaEventRecord(e_index, st));
    SG_TRY(run_init_gains(g, ws, co, model, heavy_on, st, stats ? &tev : nullptr));
    if (stats) SG_CUDA_TRY(cudaEventRecord(e_init, st));
    for (int32_t i = 0; i < k; ++i) {
        if (stats) SG_CUDA_TRY(cudaEventRecord(e_round[(size_t)i], st));
        SG_TRY(run_round(g, ws, co, model, heavy_on, i, st, stats ? e_fwd[(size_t)i] : nullptr));
    }
    SG_TRY(plant_injected_flags(ws, st));
    SG_TRY(run_poison(g, ws, ws.out_seeds.p, ws.out_gains.p, k, st));
    if (stats) {
        SG_CUDA_TRY(cudaEventRecord(e_round[(size_t)k], st));
        SG_CUDA_TRY(cudaEventRecord(e_end, st));
    }
    SG_CUDA_TRY(cudaMemcpyAsync(out_seeds, ws.out_seeds.p, (size_t)k * 4, cudaMemcpyDefault, st));
    SG_CUDA_TRY(cudaMemcpyAsync(out_gains, ws.out_gains.p, (size_t)k * 8, cudaMemcpyDefault, st));
    if (stats) {
        Ctl h;
        SG_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        memset(stats, 0, sizeof(*stats));
        stats->init_edges = h.init_edges;
        stats->fwd_edges = h.fwd_edges;
        stats->rev_edges = h.rev_edges;
        stats->init_tier2_tasks = h.init_t2;
        stats->init_tier3_tasks = h.init_t3;
        stats->rev_tier2_tasks = h.rev_t2;
        stats->rev_tier3_tasks = h.rev_t3;
        stats->rev_tasks = h.rev_tasks;
        stats->du_entries = h.du_entries;
        stats->status_flags = h.flags;
        stats->kernel_launches = g_launches - launches0;
        stats->heavy_index = heavy_on;
        stats->mask_cache = ws.lm_on;
        memcpy(stats->work_keys, h.work_keys, sizeof(h.work_keys));
        memcpy(stats->work_elems, h.work_elems, sizeof(h.work_elems));
        memcpy(stats->list_elems, h.list_elems, sizeof(h.list_elems));
        cudaEventElapsedTime(&stats->ms_index, e_start, e_index);
        cudaEventElapsedTime(&stats->ms_init, e_start, e_init);
        cudaEventElapsedTime(&stats->ms_landmarks, e_index, tev.start);
        cudaEventElapsedTime(&stats->ms_init_tier1, tev.start, tev.t1);
        cudaEventElapsedTime(&stats->ms_init_tier2, tev.t1, tev.t2);
        cudaEventElapsedTime(&stats->ms_init_tier3, tev.t2, tev.t3);
        cudaEventElapsedTime(&stats->ms_rounds, e_init, e_end);
        cudaEventElapsedTime(&stats->ms_total, e_start, e_end);
        float fsum = 0.f;
        for (int32_t i = 0; i < k; ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e_round[(size_t)i], e_fwd[(size_t)i]);
            fsum += t;
        }
        stats->ms_fwd = fsum;
        return flags_status(h.flags);
    }
    if (is_pageable(out_seeds) || is_pageable(out_gains)) {
        int32_t fl = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&fl, &ws.ctl.p->flags, 4, cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        return flags_status(fl);
    }
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_debug_inject_flags(int32_t flags)
{
    clear_error();
    if (flags < 0) {
        set_error("sg_debug_inject_flags: flags must be >= 0, got %d", flags);
        return SG_EINVAL;
    }
    g_inject_flags.store(flags);
    return SG_OK;
}

sg_status sg_debug_set_wait_limit(int64_t polls)
{
    clear_error();
    if (polls < 0) {
        set_error("sg_debug_set_wait_limit: polls must be >= 0, got %lld", (long long)polls);
        return SG_EINVAL;
    }
    g_wait_polls = polls == 0 ? WAIT_POLLS_DEFAULT : (long long)polls;
    return SG_OK;
}

sg_status sg_select(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                    int32_t *out_seeds, int64_t *out_gains, sg_stats *stats)
{
    clear_error();
    if (!g) {
        set_error("graph handle is NULL");
        return SG_EINVAL;
    }
    return select_impl(g, g->ws, R, k, c, seed, stream, out_seeds, out_gains, stats, false);
}

sg_status sg_select_state(sg_graph *g, int32_t R, int32_t k, sg_cascade c, uint64_t seed, void *stream,
                          int32_t *out_seeds, int64_t *out_gains, int64_t *out_s, uint64_t *out_cov)
{
    clear_error();
    if (!g || !out_s || !out_cov) {
        set_error("sg_select_state: NULL argument");
        return SG_EINVAL;
    }
    if (c.model == SG_UIC_UNDIRECTED) {
        set_error("sg_select_state: the undirected variant keeps no coverage bitsets");
        return SG_EINVAL;
    }
    sg_stats stats;
    SG_TRY(select_impl(g, g->ws, R, k, c, seed, stream, out_seeds, out_gains, &stats, false));
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t W = (size_t)(R + 63) / 64;
    // the round loop leaves s and the coverage in the workspace (both are
    // cleared when the next query starts)
    SG_CUDA_TRY(cudaMemcpyAsync(out_s, g->ws.s.p, (size_t)g->n * sizeof(long long), cudaMemcpyDefault, st));
    SG_CUDA_TRY(cudaMemcpyAsync(out_cov, g->ws.cov.p, (size_t)g->n * W * 8, cudaMemcpyDefault, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    return SG_OK;
}

sg_status sg_workspace_create(const sg_graph *g, int32_t R_max, int32_t k_max, void *stream, sg_workspace **out)
{
    clear_error();
    if (!g || !out) {
        set_error("sg_workspace_create: NULL argument");
        return SG_EINVAL;
    }
    SG_TRY(check_query(g, R_max, k_max));
    if (R_max < 1 || R_max >= (1 << 24)) {
        set_error("R_max must satisfy 1 <= R_max < 2^24");
        return SG_EINVAL;
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    sg_workspace *ws = new (std::nothrow) sg_workspace();
    if (!ws) {
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    sg_graph *gm = const_cast<sg_graph *>(g);
    const int32_t W = (R_max + 63) / 64;
    sg_status rc = ensure_workspace(gm, *ws, W, k_max, st);
    if (rc == SG_OK && heavy_index_enabled(g, W)) rc = ensure_heavy_index(gm, *ws, W, st);
    if (rc == SG_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("sg_workspace_create: %s", cudaGetErrorString(cudaGetLastError()));
        rc = SG_ECUDA;
    }
    if (rc != SG_OK) {
        free_workspace(*ws, st);
        delete ws;
        return rc;
    }
    ws->owner_n = g->n;
    ws->device = g->device;
    *out = ws;
    return SG_OK;
}

sg_status sg_select_ws(sg_graph *g, sg_workspace *ws, int32_t R, int32_t k, sg_cascade c, uint64_t seed,
                       void *stream, int32_t *out_seeds, int64_t *out_gains, sg_stats *stats)
{
    clear_error();
    if (!g || !ws) {
        set_error("sg_select_ws: NULL handle");
        return SG_EINVAL;
    }
    if (ws->owner_n != g->n || ws->device != g->device) {
        set_error("sg_select_ws: workspace was created for another graph");
        return SG_EINVAL;
    }
    return select_impl(g, *ws, R, k, c, seed, stream, out_seeds, out_gains, stats, false);
}

sg_status sg_workspace_bytes(const sg_graph *g, int32_t R_max, int32_t k_max, size_t *bytes)
{
    clear_error();
    if (!g || !bytes) {
        set_error("sg_workspace_bytes: NULL argument");
        return SG_EINVAL;
    }
    SG_TRY(check_query(g, R_max, k_max));
    if (R_max < 1 || R_max >= (1 << 24)) {
        set_error("R_max must satisfy 1 <= R_max < 2^24");
        return SG_EINVAL;
    }
    *bytes = workspace_bytes(g, (R_max + 63) / 64, k_max);
    return SG_OK;
}

void sg_workspace_free(sg_workspace *ws)
{
    if (!ws) return;
    DeviceGuard dg(ws->device);
    cudaDeviceSynchronize();
    free_workspace(*ws, (cudaStream_t)0);
    cudaDeviceSynchronize();
    delete ws;
}

sg_status sg_spread(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, const int32_t *S, int32_t s_count,
                    void *stream, int64_t *out_total, uint64_t *out_edges)
{
    clear_error();
    if (!g || !out_total || s_count < 0 || (s_count > 0 && !S)) {
        set_error("sg_spread: NULL graph or output, or a negative or missing seed list");
        return SG_EINVAL;
    }
    SG_TRY(check_query(g, R, 1));
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int model = c.model == SG_WIC ? MODEL_WIC : MODEL_UIC;
    // the seed list, checked on the host (host or device input)
    std::vector<int32_t> hs((size_t)s_count);
    if (s_count > 0) SG_CUDA_TRY(cudaMemcpy(hs.data(), S, (size_t)s_count * 4, cudaMemcpyDefault));
    for (int32_t v : hs)
        if (v < 0 || v >= g->n) {
            set_error("sg_spread: seed %d is not a node (n = %lld)", v, (long long)g->n);
            return SG_EINVAL;
        }
    DBuf<int32_t> dS;
    DBuf<long long> dc;
    sg_status rc = SG_OK;
    if ((rc = dbuf_alloc(dS, (size_t)std::max(1, s_count), st)) != SG_OK) return rc;
    if ((rc = dbuf_alloc(dc, 2, st)) != SG_OK) {
        dbuf_free(dS, st);
        return rc;
    }
    if (s_count > 0 && cudaMemcpyAsync(dS.p, hs.data(), (size_t)s_count * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = SG_ECUDA;
    if (rc == SG_OK && cudaMemsetAsync(dc.p, 0, 16, st) != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK && s_count > 0) {
        if (c.model == SG_UIC_UNDIRECTED) {
            rc = cc_prepare_graph(g, st);
            if (rc == SG_OK) rc = ensure_workspace(g, g->ws, co.W, 1, st);
            if (rc == SG_OK) rc = cc_ensure(g, g->ws, co.R, st);
            if (rc == SG_OK)
                rc = cc_spread(g, g->ws, co, dS.p, s_count, dc.p, reinterpret_cast<unsigned long long *>(dc.p + 1),
                               st);
        } else {
            rc = run_spread(g, co, model, dS.p, s_count, dc.p, reinterpret_cast<unsigned long long *>(dc.p + 1),
                                st);
        }
    }
    long long hc[2] = {0, 0};
    if (rc == SG_OK && cudaMemcpyAsync(hc, dc.p, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SG_ECUDA;
    dbuf_free(dS, st);
    dbuf_free(dc, st);
    if (rc == SG_ECUDA && !g_err[0]) set_error("sg_spread: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc != SG_OK) return rc;
    SG_CUDA_TRY(cudaMemcpy(out_total, &hc[0], 8, cudaMemcpyDefault));
    if (out_edges) *out_edges = (uint64_t)hc[1];
    return SG_OK;
}

sg_status sg_init_gains(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, void *stream, int64_t *out_s,
                        uint64_t *init_edges)
{
    clear_error();
    SG_TRY(check_query(g, R, 1));
    if (!out_s) {
        set_error("sg_init_gains: out_s must be non-NULL");
        return SG_EINVAL;
    }
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int model = c.model == SG_WIC ? MODEL_WIC : MODEL_UIC;
    sg_workspace &ws = g->ws;
    SG_TRY(ensure_workspace(g, ws, co.W, 1, st));
    if (c.model == SG_UIC_UNDIRECTED) {
        SG_TRY(cc_prepare_graph(g, st));
        SG_TRY(cc_ensure(g, ws, co.R, st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.s.p, 0, (size_t)g->n * sizeof(long long), st));
        SG_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, sizeof(Ctl), st));
        SG_TRY(cc_init_gains(g, ws, co, st));
        SG_TRY(plant_injected_flags(ws, st));
        SG_TRY(run_poison(g, ws, nullptr, ws.s.p, g->n, st));
        SG_CUDA_TRY(cudaMemcpyAsync(out_s, ws.s.p, (size_t)g->n * 8, cudaMemcpyDefault, st));
        Ctl h;
        SG_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        if (init_edges) *init_edges = h.init_edges;
        return flags_status(h.flags);
    }
    const int heavy_on = (!co.lt && heavy_index_enabled(g, co.W)) ? 1 : 0;
    if (heavy_on) SG_TRY(ensure_heavy_index(g, ws, co.W, st));
    ws.slists_on = 0;
    ws.fl_on = 0;
    if (heavy_on) SG_TRY(ensure_fwd_lists(g, ws, co, c.p, model, st));
    SG_TRY(ensure_mask_cache(g, ws, co.W, st, co.lt != 0));
    SG_CUDA_TRY(cudaMemsetAsync(ws.s.p, 0, (size_t)g->n * sizeof(long long), st));
    SG_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, sizeof(Ctl), st));
    if (heavy_on) {
        SG_TRY(run_heavy_index(g, ws, co, model, st));
        if (ws.fl_on) SG_TRY(run_fwd_lists(g, ws, co, st));
        SG_TRY(run_row_desc(g, ws, co, st));
        ws.rd_on = 1;
    }
    if (ws.lm_on) SG_TRY(run_mask_cache(g, ws, co, model, st));
    SG_TRY(run_init_gains(g, ws, co, model, heavy_on, st));
    SG_TRY(plant_injected_flags(ws, st));
    SG_TRY(run_poison(g, ws, nullptr, ws.s.p, g->n, st));
    SG_CUDA_TRY(cudaMemcpyAsync(out_s, ws.s.p, (size_t)g->n * 8, cudaMemcpyDefault, st));
    if (init_edges) {
        Ctl h;
        SG_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        *init_edges = h.init_edges;
        return flags_status(h.flags);
    }
    if (is_pageable(out_s)) {
        int32_t fl = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&fl, &ws.ctl.p->flags, 4, cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        return flags_status(fl);
    }
    return SG_OK;
}

sg_status sg_live_masks(sg_graph *g, int32_t R, sg_cascade c, uint64_t seed, void *stream, uint64_t *out_masks)
{
    clear_error();
    if (!g || !out_masks) {
        set_error("sg_live_masks: NULL argument");
        return SG_EINVAL;
    }
    Coins co;
    SG_TRY(make_coins(c, seed, R, &co));
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int model = c.model == SG_WIC ? MODEL_WIC : MODEL_UIC;
    const size_t count = (size_t)g->m * (size_t)co.W;
    if (count == 0) return SG_OK;
    const int32_t *cid = nullptr;
    if (c.model == SG_UIC_UNDIRECTED) {
        SG_TRY(cc_prepare_graph(g, st));
        cid = g->cc_pmin.p;
    }
    if (!is_pageable(out_masks)) {
        cudaPointerAttributes at;
        SG_CUDA_TRY(cudaPointerGetAttributes(&at, out_masks));
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
            return run_live_masks(g, co, model, out_masks, st, cid);
    }
    DBuf<uint64_t> tmp;
    SG_TRY(dbuf_alloc(tmp, count, st));
    sg_status rc = run_live_masks(g, co, model, tmp.p, st, cid);
    if (rc == SG_OK && cudaMemcpyAsync(out_masks, tmp.p, count * 8, cudaMemcpyDefault, st) != cudaSuccess) {
        set_error("sg_live_masks: copy-out failed");
        rc = SG_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == SG_OK) rc = SG_ECUDA;
    dbuf_free(tmp, st);
    return rc;
}

}  // extern "C"
