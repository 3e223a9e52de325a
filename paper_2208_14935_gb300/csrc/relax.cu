// Push relax kernels over the active edges of one route (Sec. II-A push
// model; Sec. VI-C processing kernels), and the compaction gather of the C
// route (Sec. II-B ExpTM-compaction, here done by the GPU over the host link).
//
// Load balancing: the active vertices of a route form a list ordered by
// vertex id; their out-edges form one "route edge space" [0, E_route).  A
// block takes a tile of kTile consecutive route edges, finds the list entries
// that own them (the entry holding the tile's first edge comes from the
// tile index written by k_bin), marks each entry's first edge in shared
// memory and fills the gaps with a max-scan, so every thread knows the owner
// of each of its edges in O(1).  Threads take edges k0 + tid + j * 256, so a
// warp reads consecutive edges of the same or adjacent lists: 128-byte lines
// when the lists are long, and neighbouring lists share lines when
// consecutive vertices are active.
//
// Edge sources (the route's transfer method):
//   host    zero-copy loads from pinned, device-mapped host memory (Eq. 3 route);
//   device  a device copy starting at CSR edge `shift` (cache and F routes:
//           the partition's edges are shifted by its first edge index);
//   compact the compacted buffer, where route edge k sits at k - shift.
#include "common.cuh"
#include "relax_tile.cuh"

namespace hytg {

namespace {

// hub_rep: this SM's replica row of the hub accumulators (PageRank only).
template <int ALGO>
__device__ __forceinline__ void relax_edge(const AlgoState &st, unsigned int v, unsigned int pay,
                                           unsigned int w, float *hub_rep) {
    if (ALGO == kPR || ALGO == kPPR) {
        // fire-and-forget reduction; the next frontier is rebuilt from delta
        // (delta > eps) by k_pr_frontier once every relax of the iteration is
        // done.  Pushes to the hottest vertices (hub-sorted ids below
        // n_hub_rep) go to this SM's replica, so thousands of SMs' updates do
        // not serialise on one L2 address.
        if (v < st.n_hub_rep) atomicAdd(&hub_rep[v], __uint_as_float(pay));
        else atomicAdd(&st.delta[v], __uint_as_float(pay));
    } else {
        unsigned int nv;
        if (ALGO == kBFS) {
            nv = pay + 1u;
        } else if (ALGO == kSSSP) {
            const unsigned long long s = (unsigned long long)pay + w;
            if (s >= 0xFFFFFFFEull) { *st.overflow = 1u; return; }
            nv = (unsigned int)s;
        } else {
            nv = pay;
        }
        // Fire-and-forget min and frontier bit when the pushed value beats the
        // value seen now.  If a concurrent push lowered v further in between,
        // v is still marked active: it then re-pushes its (current) value
        // next iteration, which is redundant but never wrong for min-updates.
        if (nv < __ldcg(&st.val[v])) {
            atomicMin(&st.val[v], nv);
            atomicOr(&st.bm_next[v >> 5], 1u << (v & 31));
        }
    }
}

// One tile of a relax launch: route edges [tile * kTile, ...) within [kb, ke).
template <int ALGO>
__device__ __forceinline__ void relax_tile(const AlgoState &st, const ListArrays &la, const Summary *sum,
                                           const RelaxTask &t, unsigned long long tile,
                                           unsigned long long kb, unsigned long long ke,
                                           TileSmem<false> &sm, float *hub_rep) {
    const bool weighted = (ALGO == kSSSP);
    unsigned long long k0;
    const int n = tile_setup<false>(sm, la, sum, t, tile, kb, ke, &k0);
    unsigned int dv[kRelaxIPT], wv[kRelaxIPT], pv[kRelaxIPT];
#pragma unroll
    for (int j = 0; j < kRelaxIPT; ++j) {
        const int slot = threadIdx.x + j * kRelaxBlock;
        dv[j] = kInf;
        wv[j] = 0;
        pv[j] = 0;
        if (slot < n) {
            const int i = sm.sid[slot];
            const long long e = (long long)(k0 + slot) + sm.delta[i];
            if (e >= 0 && (unsigned long long)e < t.src_len) {
                dv[j] = __ldg(t.dst + e);
                if (weighted) wv[j] = __ldg(t.w + e);
                pv[j] = sm.pay[i];
            } else {
                atomicOr(la.err, 8u);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kRelaxIPT; ++j)
        if (dv[j] != kInf) relax_edge<ALGO>(st, dv[j], pv[j], wv[j], hub_rep);
    __syncthreads();
}

template <int ALGO>
__global__ void __launch_bounds__(kRelaxBlock) k_relax(AlgoState st, ListArrays la,
                                                       const Summary *sum, RelaxTask t) {
    __shared__ TileSmem<false> sm;
    if (st.loop && !st.loop->work) return;
    const unsigned long long kb = t.device_sized ? 0ull : t.k_begin;
    const unsigned long long ke = t.device_sized ? sum->route_edges[t.route] : t.k_end;
    if (kb >= ke) return;
    const unsigned long long t_first = kb / kTile, t_last = (ke - 1) / kTile;
    float *hub_rep = st.hub_rep ? st.hub_rep + (size_t)(sm_id() % kHubReplicas) * st.n_hub_rep : nullptr;
    for (unsigned long long tile = t_first + blockIdx.x; tile <= t_last; tile += gridDim.x)
        relax_tile<ALGO>(st, la, sum, t, tile, kb, ke, sm, hub_rep);
}

// Two device-sized routes in one launch (cache and zero-copy in the device
// loop, where an iteration's frontier is often a few hundred vertices and a
// launch costs more than the work).
template <int ALGO>
__global__ void __launch_bounds__(kRelaxBlock) k_relax_pair(AlgoState st, ListArrays la,
                                                            const Summary *sum, RelaxTask ta,
                                                            RelaxTask tb) {
    __shared__ TileSmem<false> sm;
    if (st.loop && !st.loop->work) return;
    float *hub_rep = st.hub_rep ? st.hub_rep + (size_t)(sm_id() % kHubReplicas) * st.n_hub_rep : nullptr;
    const unsigned long long ea = sum->route_edges[ta.route], eb = sum->route_edges[tb.route];
    if (ea) {
        for (unsigned long long tile = blockIdx.x; tile <= (ea - 1) / kTile; tile += gridDim.x)
            relax_tile<ALGO>(st, la, sum, ta, tile, 0ull, ea, sm, hub_rep);
    }
    if (eb) {
        for (unsigned long long tile = blockIdx.x; tile <= (eb - 1) / kTile; tile += gridDim.x)
            relax_tile<ALGO>(st, la, sum, tb, tile, 0ull, eb, sm, hub_rep);
    }
}

__global__ void __launch_bounds__(kRelaxBlock) k_gather(ListArrays la, const Summary *sum,
                                                        RelaxTask t, unsigned int *out_dst,
                                                        unsigned int *out_w) {
    __shared__ TileSmem<false> sm;
    const unsigned long long kb = t.k_begin, ke = t.k_end;
    if (kb >= ke) return;
    const unsigned long long t_first = kb / kTile, t_last = (ke - 1) / kTile;
    for (unsigned long long tile = t_first + blockIdx.x; tile <= t_last; tile += gridDim.x) {
        unsigned long long k0;
        const int n = tile_setup<false>(sm, la, sum, t, tile, kb, ke, &k0);
        unsigned int dv[kRelaxIPT], wv[kRelaxIPT];
#pragma unroll
        for (int j = 0; j < kRelaxIPT; ++j) {
            const int slot = threadIdx.x + j * kRelaxBlock;
            dv[j] = 0;
            wv[j] = 0;
            if (slot < n) {
                const long long e = (long long)(k0 + slot) + sm.delta[sm.sid[slot]];
                if (e >= 0 && (unsigned long long)e < t.src_len) {
                    dv[j] = __ldg(t.dst + e);
                    if (out_w) wv[j] = __ldg(t.w + e);
                } else {
                    atomicOr(la.err, 8u);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kRelaxIPT; ++j) {
            const int slot = threadIdx.x + j * kRelaxBlock;
            if (slot < n) {
                const unsigned long long o = k0 + slot - kb;
                out_dst[o] = dv[j];
                if (out_w) out_w[o] = wv[j];
            }
        }
        __syncthreads();
    }
}

// Second pass over a resident vertex range (Sec. VI-A: a loaded subgraph is
// processed once more).  Vertices of [vlo, vhi) that became active again
// during this iteration (PageRank: delta > eps; others: frontier bit set and,
// for bucketed SSSP, dist below the bucket) are taken and pushed along their
// edges in `dst`/`w`, which hold CSR edges [shift, shift + src_len).
// A warp takes 32 consecutive vertices; vertices with more than
// kSecondPassMaxDeg edges are not taken and stay active for the next
// iteration's load-balanced relax.
constexpr unsigned long long kSecondPassMaxDeg = 4096;

template <int ALGO>
__device__ __forceinline__ bool second_pass_take(const AlgoState &st, unsigned long long v,
                                                 unsigned long long deg, unsigned int &pay) {
    if (ALGO == kPR || ALGO == kPPR) {
        // Take the delta seen now and subtract it with a reduction, so that
        // pushes landing on v meanwhile (relaxes of other streams) stay in
        // delta for later.  No second pass overlaps this vertex range and
        // k_bin never runs beside one, so this thread is the only writer of
        // rank[v] now: a plain update suffices.
        const float dl = __ldcg(&st.delta[v]);
        if (dl <= st.eps) return false;
        atomicAdd(&st.delta[v], -dl);
        st.rank[v] += dl;
        if (deg == 0) return false;
        pay = __float_as_uint(st.damping * dl / (float)deg);
        return true;
    } else {
        const unsigned int mask = 1u << (v & 31);
        if (!(__ldcg(&st.bm_cur[v >> 5]) & mask)) return false;
        if (st.bucket_limit != 0xFFFFFFFFu && __ldcg(&st.val[v]) >= st.bucket_limit) return false;
        const unsigned int old = atomicAnd(&st.bm_cur[v >> 5], ~mask);
        if (!(old & mask)) return false;
        pay = __ldcg(&st.val[v]);
        return true;
    }
}

template <int ALGO>
__global__ void __launch_bounds__(256) k_second_pass(AlgoState st, const unsigned long long *off,
                                                     const unsigned int *dst, const unsigned int *w,
                                                     long long shift, unsigned long long src_len,
                                                     unsigned long long vlo, unsigned long long vhi,
                                                     unsigned long long *edges_out, unsigned int *err) {
    if (st.loop) {
        if (!st.loop->work) return;
        st.bucket_limit = st.loop->bucket;
    }
    float *hub_rep = st.hub_rep ? st.hub_rep + (size_t)(sm_id() % kHubReplicas) * st.n_hub_rep : nullptr;
    const int lane = threadIdx.x & 31;
    unsigned long long done = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long first = vlo + ((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull);
    for (unsigned long long base = first; base < vhi; base += stride) {
        const unsigned long long v = base + lane;
        unsigned long long e0 = ~0ull, deg = 0;       // lanes past vhi own no edge
        unsigned int pay = 0;
        bool mine = false;
        if (v < vhi) {
            e0 = off[v];
            deg = off[v + 1] - e0;
            if (deg <= kSecondPassMaxDeg) mine = second_pass_take<ALGO>(st, v, deg, pay);
        }
        const unsigned int mask = __ballot_sync(0xffffffffu, mine);
        if (mask == 0) continue;                       // warp-uniform
        const unsigned long long act = warp_sum_u64(mine ? deg : 0ull);
        if (lane == 0) done += act;
        // The 32 vertices are consecutive, so their lists form one CSR range
        // [E0, E1).  If at least half of it belongs to taken vertices, the
        // warp streams the range with coalesced loads and each lane finds the
        // owner of its edge among the 32 list starts; otherwise it walks the
        // taken vertices one at a time.
        const int last = (int)((vhi - 1 - base) < 31 ? (vhi - 1 - base) : 31);
        const unsigned long long E0 = __shfl_sync(0xffffffffu, e0, 0);
        const unsigned long long E1 = __shfl_sync(0xffffffffu, e0 + deg, last);
        if (2 * act >= E1 - E0) {
            // kStream chunks of 32 edges per round: owners and loads of all
            // chunks first, then the pushes, so the loads overlap
            constexpr int kStream = 4;
            for (unsigned long long c0 = E0; c0 < E1; c0 += 32 * kStream) {
                unsigned int dv[kStream], wv[kStream], pv[kStream];
                bool ok[kStream];
#pragma unroll
                for (int q = 0; q < kStream; ++q) {
                    const unsigned long long k = c0 + 32 * q + lane;
                    int own = 0;                       // largest lane whose list starts at or before k
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const unsigned long long cand = __shfl_sync(0xffffffffu, e0, own + step);
                        if (cand <= k) own += step;
                    }
                    pv[q] = __shfl_sync(0xffffffffu, pay, own);
                    ok[q] = k < E1 && ((mask >> own) & 1u);
                    dv[q] = 0;
                    wv[q] = 0;
                    if (ok[q]) {
                        const long long i = (long long)k - shift;
                        if (i < 0 || (unsigned long long)i >= src_len) {
                            atomicOr(err, 16u);
                            ok[q] = false;
                        } else {
                            dv[q] = __ldg(dst + i);
                            if (ALGO == kSSSP) wv[q] = __ldg(w + i);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kStream; ++q)
                    if (ok[q]) relax_edge<ALGO>(st, dv[q], pv[q], wv[q], hub_rep);
            }
        } else {
            unsigned int m = mask;
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const unsigned long long ce0 = __shfl_sync(0xffffffffu, e0, src);
                const unsigned long long cdeg = __shfl_sync(0xffffffffu, deg, src);
                const unsigned int cpay = __shfl_sync(0xffffffffu, pay, src);
                for (unsigned long long k = lane; k < cdeg; k += 32) {
                    const long long i = (long long)(ce0 + k) - shift;
                    if (i < 0 || (unsigned long long)i >= src_len) { atomicOr(err, 16u); break; }
                    relax_edge<ALGO>(st, __ldg(dst + i), cpay, (ALGO == kSSSP) ? __ldg(w + i) : 0u, hub_rep);
                }
            }
        }
    }
    done = warp_sum_u64(done);
    if (lane == 0 && done) atomicAdd(edges_out, done);
}

}  // namespace

cudaError_t launch_second_pass(const AlgoState &st, const unsigned long long *off,
                               const unsigned int *dst, const unsigned int *w, long long shift,
                               unsigned long long src_len, unsigned long long vlo,
                               unsigned long long vhi, unsigned long long *edges_out,
                               unsigned int *err, cudaStream_t s) {
    if (vhi <= vlo) return cudaSuccess;
    unsigned long long blocks = (vhi - vlo + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    switch (st.algo) {
        case kBFS: k_second_pass<kBFS><<<(unsigned int)blocks, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, edges_out, err); break;
        case kSSSP: k_second_pass<kSSSP><<<(unsigned int)blocks, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, edges_out, err); break;
        case kCC: k_second_pass<kCC><<<(unsigned int)blocks, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, edges_out, err); break;
        default: k_second_pass<kPR><<<(unsigned int)blocks, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, edges_out, err); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relax(const AlgoState &st, const ListArrays &la, const Summary *sum,
                         const RelaxTask &t, int grid_cap, cudaStream_t s) {
    unsigned int grid = (unsigned int)grid_cap;
    if (!t.device_sized) {
        if (t.k_begin >= t.k_end) return cudaSuccess;
        const unsigned long long tiles = (t.k_end - 1) / kTile - t.k_begin / kTile + 1;
        if (tiles < grid) grid = (unsigned int)tiles;
    }
    switch (st.algo) {
        case kBFS: k_relax<kBFS><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, t); break;
        case kSSSP: k_relax<kSSSP><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, t); break;
        case kCC: k_relax<kCC><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, t); break;
        default: k_relax<kPR><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, t); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relax_pair(const AlgoState &st, const ListArrays &la, const Summary *sum,
                              const RelaxTask &ta, const RelaxTask &tb, int grid, cudaStream_t s) {
    switch (st.algo) {
        case kBFS: k_relax_pair<kBFS><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, ta, tb); break;
        case kSSSP: k_relax_pair<kSSSP><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, ta, tb); break;
        case kCC: k_relax_pair<kCC><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, ta, tb); break;
        default: k_relax_pair<kPR><<<grid, kRelaxBlock, 0, s>>>(st, la, sum, ta, tb); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const ListArrays &la, const Summary *sum, const RelaxTask &t,
                          unsigned int *out_dst, unsigned int *out_w, int grid_cap,
                          cudaStream_t s) {
    if (t.k_begin >= t.k_end) return cudaSuccess;
    const unsigned long long tiles = (t.k_end - 1) / kTile - t.k_begin / kTile + 1;
    unsigned int grid = tiles < (unsigned long long)grid_cap ? (unsigned int)tiles : (unsigned int)grid_cap;
    k_gather<<<grid, kRelaxBlock, 0, s>>>(la, sum, t, out_dst, out_w);
    return cudaGetLastError();
}

}  // namespace hytg
