// Hub sorting (Sec. VI-A): the top fraction of vertices by
// H(v) = D_o(v) * D_i(v) / (D_omax * D_imax) are moved to the front of the
// CSR in decreasing H; the other vertices keep their natural order.  Host
// code, run once at load time.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "hytg.h"

namespace {

void par_for(uint64_t n, const std::function<void(uint64_t, uint64_t)> &fn) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < (1u << 18)) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(fn, n * t / nt, n * (t + 1) / nt);
    fn(0, n / nt);
    for (auto &x : th) x.join();
}

}  // namespace

extern "C" hytg_status hytg_hub_order(uint64_t V, const uint64_t *offsets, const uint32_t *dst,
                                      double frac, uint32_t *perm, uint64_t *n_hubs) {
    if (!offsets || !perm || V == 0 || V > 0xFFFFFFFFull || !(frac >= 0.0 && frac <= 1.0))
        return HYTG_ERR_ARG;
    const uint64_t E = offsets[V];
    if (E > 0 && !dst) return HYTG_ERR_ARG;
    try {
        std::vector<std::atomic<uint32_t>> din(V);
        par_for(V, [&](uint64_t lo, uint64_t hi) {
            for (uint64_t v = lo; v < hi; ++v) din[v].store(0, std::memory_order_relaxed);
        });
        par_for(E, [&](uint64_t lo, uint64_t hi) {
            for (uint64_t e = lo; e < hi; ++e) din[dst[e]].fetch_add(1, std::memory_order_relaxed);
        });
        const uint64_t k = (uint64_t)std::floor(frac * (double)V);
        // H(v) up to the positive constant 1 / (D_omax * D_imax): D_o * D_i
        std::vector<uint32_t> order(V);
        for (uint64_t v = 0; v < V; ++v) order[v] = (uint32_t)v;
        auto key = [&](uint32_t v) {
            return (unsigned __int128)(offsets[v + 1] - offsets[v]) *
                   din[v].load(std::memory_order_relaxed);
        };
        auto before = [&](uint32_t a, uint32_t b) {   // larger H first, then smaller id
            const unsigned __int128 ka = key(a), kb = key(b);
            return ka != kb ? ka > kb : a < b;
        };
        if (k > 0 && k < V) std::nth_element(order.begin(), order.begin() + k, order.end(), before);
        std::sort(order.begin(), order.begin() + k, before);
        std::vector<unsigned char> is_hub(V, 0);
        for (uint64_t i = 0; i < k; ++i) is_hub[order[i]] = 1;
        uint64_t pos = 0;
        for (uint64_t i = 0; i < k; ++i) perm[pos++] = order[i];
        for (uint64_t v = 0; v < V; ++v)
            if (!is_hub[v]) perm[pos++] = (uint32_t)v;
        if (n_hubs) *n_hubs = k;
        return HYTG_OK;
    } catch (...) {
        return HYTG_ERR_HOSTMEM;
    }
}
