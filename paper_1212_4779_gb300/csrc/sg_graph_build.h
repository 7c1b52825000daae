// Host-side graph construction for the graph loaders (plain C++, no CUDA):
// the canonical CSR and the CSC by a stable counting sort, parallel over the
// host's threads with results independent of the thread count.
#pragma once

#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <utility>
#include <thread>
#include <vector>

namespace sgh {

// std::vector whose resize leaves new elements of trivial types
// uninitialised (no zeroing pass before they are written).
template <class T>
struct default_init_alloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = default_init_alloc<U>;
    };
    default_init_alloc() = default;
    template <class U>
    default_init_alloc(const default_init_alloc<U> &) noexcept
    {
    }
    template <class U>
    void construct(U *p) noexcept
    {
        ::new ((void *)p) U;
    }
    template <class U, class... A>
    void construct(U *p, A &&...a)
    {
        ::new ((void *)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using hvec = std::vector<T, default_init_alloc<T>>;

// Host threads the builders use: the hardware's (at most 64), or the
// positive value set in thread_cap() (tests run several counts).
inline int &thread_cap()
{
    static int cap = 0;
    return cap;
}

inline int host_threads()
{
    if (thread_cap() > 0) return thread_cap();
    unsigned h = std::thread::hardware_concurrency();
    if (h == 0) h = 4;
    return (int)std::min(h, 64u);
}

// f(t) for t = 0 .. T-1 on T host threads (inline when T <= 1).
template <class F>
void parallel_parts(int T, F &&f)
{
    if (T <= 1) {
        f(0);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back([&f, t] { f(t); });
    for (auto &x : th) x.join();
}

// f(a, b) over contiguous ranges of [0, n) on the host threads.
template <class F>
void parallel_rows(int64_t n, F &&f)
{
    const int T = host_threads();
    if (n < 4096 || T <= 1) {
        f(0, n);
        return;
    }
    const int64_t chunk = (n + T - 1) / T;
    parallel_parts(T, [&](int t) {
        const int64_t a = std::min(n, t * chunk), b = std::min(n, a + chunk);
        if (a < b) f(a, b);
    });
}

// Smallest i in [0, count) with bad(i), or count.
template <class F>
int64_t parallel_first(int64_t count, F &&bad)
{
    const int T = count >= (1 << 20) ? host_threads() : 1;
    const int64_t chunk = (count + T - 1) / T;
    std::vector<int64_t> first((size_t)T, count);
    parallel_parts(T, [&](int t) {
        const int64_t a = std::min(count, t * chunk), b = std::min(count, a + chunk);
        for (int64_t i = a; i < b; ++i)
            if (bad(i)) {
                first[(size_t)t] = i;
                break;
            }
    });
    return *std::min_element(first.begin(), first.end());
}

// Canonical CSR (the paper treats parallel edges as one edge): per row,
// destinations sorted ascending, repeats merged, self-loops dropped.  Reads
// rows rp_in[u] .. rp_in[u + 1] of col_in, which it does not modify; rows
// that are canonical already are copied as they are.
inline void canonicalise(int64_t n, const int64_t *rp_in, const int32_t *col_in, hvec<int32_t> &rp_out,
                         hvec<int32_t> &col_out)
{
    std::vector<int32_t> len((size_t)n);
    std::vector<uint8_t> sorted_ok((size_t)n);
    auto unique_sorted = [](std::vector<int32_t> &tmp, int64_t u, int32_t *out) -> int32_t {
        std::sort(tmp.begin(), tmp.end());
        int32_t c = 0;
        for (size_t i = 0; i < tmp.size(); ++i)
            if (tmp[i] != u && (i == 0 || tmp[i] != tmp[i - 1])) {
                if (out) out[c] = tmp[i];
                ++c;
            }
        return c;
    };
    parallel_rows(n, [&](int64_t a, int64_t b) {
        std::vector<int32_t> tmp;
        for (int64_t u = a; u < b; ++u) {
            const int32_t *r = col_in + rp_in[u];
            const int64_t d = rp_in[u + 1] - rp_in[u];
            bool canon = true;
            for (int64_t i = 0; i < d && canon; ++i)
                if (r[i] == u || (i > 0 && r[i] <= r[i - 1])) canon = false;
            sorted_ok[(size_t)u] = canon ? 1 : 0;
            if (canon) {
                len[(size_t)u] = (int32_t)d;
                continue;
            }
            tmp.assign(r, r + d);
            len[(size_t)u] = unique_sorted(tmp, u, nullptr);
        }
    });
    rp_out.resize((size_t)n + 1);
    rp_out[0] = 0;
    for (int64_t u = 0; u < n; ++u) rp_out[(size_t)u + 1] = rp_out[(size_t)u] + len[(size_t)u];
    col_out.resize((size_t)std::max<int64_t>(1, rp_out[(size_t)n]));
    parallel_rows(n, [&](int64_t a, int64_t b) {
        std::vector<int32_t> tmp;
        for (int64_t u = a; u < b; ++u) {
            const int32_t *r = col_in + rp_in[u];
            const int64_t d = rp_in[u + 1] - rp_in[u];
            int32_t *o = col_out.data() + rp_out[(size_t)u];
            if (sorted_ok[(size_t)u]) {
                if (d) memcpy(o, r, (size_t)d * sizeof(int32_t));
                continue;
            }
            tmp.assign(r, r + d);
            unique_sorted(tmp, u, o);
        }
    });
}

// One in-arc of the CSC: its source and its arc id (CSR position).
struct Arc2 {
    int32_t x, y;
};

// CSC of a CSR by a stable counting sort on destination: the in-arcs of
// each node in increasing (source, arc id) order.  Thread t takes the rows
// holding about m / T consecutive arcs, counts its arcs per destination in
// a histogram of its own, and places them at offsets that put thread t's
// arcs of a destination after those of threads 0 .. t-1: the order is the
// sequential sort's for any thread count.
inline void build_csc(int64_t n, const hvec<int32_t> &rp, const hvec<int32_t> &col, hvec<int32_t> &crp,
                      hvec<Arc2> &cin)
{
    const int64_t m = rp[(size_t)n];
    int T = m >= (1 << 20) ? host_threads() : 1;
    // per-thread histograms: T * n counters, at most 2^28 (1 GiB)
    T = (int)std::max<int64_t>(1, std::min<int64_t>(T, ((int64_t)1 << 28) / std::max<int64_t>(1, n)));
    std::vector<int64_t> ub((size_t)T + 1);  // thread t: rows ub[t] .. ub[t + 1]
    for (int t = 0; t <= T; ++t) {
        const int64_t target = m * t / T;
        ub[(size_t)t] = std::lower_bound(rp.begin(), rp.begin() + n, (int32_t)target) - rp.begin();
    }
    ub[(size_t)T] = n;
    hvec<int32_t> cnt((size_t)T * (size_t)n);
    parallel_parts(T, [&](int t) {
        int32_t *h = cnt.data() + (size_t)t * (size_t)n;
        memset(h, 0, (size_t)n * sizeof(int32_t));  // first touch by the thread that uses it
        for (int64_t e = rp[(size_t)ub[(size_t)t]]; e < rp[(size_t)ub[(size_t)t + 1]]; ++e) h[col[(size_t)e]]++;
    });
    crp.resize((size_t)n + 1);
    crp[0] = 0;
    parallel_rows(n, [&](int64_t a, int64_t b) {
        for (int64_t y = a; y < b; ++y) {
            int32_t s = 0;
            for (int t = 0; t < T; ++t) {
                int32_t &c = cnt[(size_t)t * (size_t)n + (size_t)y];
                const int32_t v = c;
                c = s;
                s += v;
            }
            crp[(size_t)y + 1] = s;
        }
    });
    for (int64_t y = 0; y < n; ++y) crp[(size_t)y + 1] += crp[(size_t)y];
    cin.resize((size_t)std::max<int64_t>(1, m));
    parallel_parts(T, [&](int t) {
        int32_t *h = cnt.data() + (size_t)t * (size_t)n;
        for (int64_t u = ub[(size_t)t]; u < ub[(size_t)t + 1]; ++u)
            for (int32_t e = rp[(size_t)u]; e < rp[(size_t)u + 1]; ++e) {
                const int32_t y = col[(size_t)e];
                cin[(size_t)(crp[(size_t)y] + h[y]++)] = Arc2{(int32_t)u, e};
            }
    });
}

}  // namespace sgh
