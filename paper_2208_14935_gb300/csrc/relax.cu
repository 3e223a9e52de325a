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
    if (t.link_ctr) count_link_reads<false>(sm, k0, n, weighted ? 2u : 1u, t.link_ctr);
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
    unsigned long long kb, ke;
    task_range(t, sum, kb, ke);
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
                                                        unsigned int *out_w, const LoopCtl *loop) {
    __shared__ TileSmem<false> sm;
    if (loop && !loop->work) return;
    unsigned long long kb, ke;
    task_range(t, sum, kb, ke);
    if (kb >= ke) return;
    const unsigned long long t_first = kb / kTile, t_last = (ke - 1) / kTile;
    for (unsigned long long tile = t_first + blockIdx.x; tile <= t_last; tile += gridDim.x) {
        unsigned long long k0;
        const int n = tile_setup<false>(sm, la, sum, t, tile, kb, ke, &k0);
        if (t.link_ctr) count_link_reads<false>(sm, k0, n, out_w ? 2u : 1u, t.link_ctr);
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
//
// Two launches, so that the work is balanced over edges whatever the
// degrees: k_sp_take (a warp per 32 consecutive vertices) takes the vertices,
// records each one's push value and a taken bit, and writes for every chunk
// of kSpChunk edges whose first edge lies in a vertex's list that vertex as
// the chunk's owner; k_sp_push gives each warp whole chunks of the range's
// edges [E0, E1), finds each edge's owner among a window of 32 consecutive
// vertices (their list starts, by shuffles) and pushes the edges of taken
// owners with coalesced loads.
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
        return deg > 0;
    }
}

template <int ALGO>
__global__ void __launch_bounds__(256) k_sp_take(AlgoState st, const unsigned long long *off,
                                                 unsigned long long vlo, unsigned long long vhi,
                                                 SecondPassScratch sc, unsigned long long *edges_out) {
    if (st.loop) {
        if (!st.loop->work) return;
        st.bucket_limit = st.loop->bucket;
    }
    const int lane = threadIdx.x & 31;
    unsigned long long done = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // vlo is a multiple of 32 (partition bounds), so each warp's 32 vertices
    // fill one word of the taken mask
    for (unsigned long long base = vlo + ((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull);
         base < vhi; base += stride) {
        const unsigned long long v = base + lane;
        unsigned long long e0 = 0, deg = 0;
        unsigned int pay = 0;
        bool mine = false;
        if (v < vhi) {
            e0 = off[v];
            deg = off[v + 1] - e0;
            mine = second_pass_take<ALGO>(st, v, deg, pay);
            sc.pay[v] = pay;
        }
        const unsigned int taken = __ballot_sync(0xffffffffu, mine);
        if (lane == 0) sc.mask[base >> 5] = taken;
        done += mine ? deg : 0ull;
        // owners of the chunks [c_beg, c_end) whose first edge is in v's list,
        // written by the whole warp one vertex at a time
        const unsigned long long c_beg = deg ? (e0 + kSpChunk - 1) / kSpChunk : 0ull;
        const unsigned long long c_end = deg ? (e0 + deg - 1) / kSpChunk + 1 : 0ull;
        unsigned int has = __ballot_sync(0xffffffffu, c_end > c_beg);
        while (has) {
            const int l = __ffs(has) - 1;
            has &= has - 1;
            const unsigned long long cb = __shfl_sync(0xffffffffu, c_beg, l);
            const unsigned long long ce = __shfl_sync(0xffffffffu, c_end, l);
            for (unsigned long long c = cb + lane; c < ce; c += 32) sc.owner[c] = (unsigned int)(base + l);
        }
    }
    done = warp_sum_u64(done);
    if (lane == 0 && done) atomicAdd(edges_out, done);
}

template <int ALGO>
__global__ void __launch_bounds__(256) k_sp_push(AlgoState st, const unsigned long long *off,
                                                 const unsigned int *dst, const unsigned int *w,
                                                 long long shift, unsigned long long src_len,
                                                 unsigned long long vlo, unsigned long long vhi,
                                                 unsigned long long E0, unsigned long long E1,
                                                 SecondPassScratch sc, unsigned int *err) {
    if (st.loop && !st.loop->work) return;
    if (E1 <= E0) return;
    float *hub_rep = st.hub_rep ? st.hub_rep + (size_t)(sm_id() % kHubReplicas) * st.n_hub_rep : nullptr;
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long c_first = E0 / kSpChunk, c_last = (E1 - 1) / kSpChunk;
    for (unsigned long long c = c_first + ((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5);
         c <= c_last; c += nwarps) {
        const unsigned long long k0 = c * kSpChunk > E0 ? c * kSpChunk : E0;
        const unsigned long long k1 = (c + 1) * kSpChunk < E1 ? (c + 1) * kSpChunk : E1;
        // a vertex at or before the owner of k0: the recorded owner of the
        // chunk's first edge, or vlo for a chunk that starts before the range
        unsigned long long u0 = c * kSpChunk >= E0 ? (unsigned long long)sc.owner[c] : vlo;
        if (u0 < vlo || u0 >= vhi) {
            if (lane == 0) atomicOr(err, 32u);
            continue;
        }
        unsigned long long kb = k0;
        while (kb < k1) {
            // window of 32 candidate owners u0 .. u0 + 31 (past vhi: no edges)
            const unsigned long long u = u0 + lane;
            const unsigned long long su = u < vhi ? off[u] : E1;
            const unsigned long long ue = u0 + 32 < vhi ? u0 + 32 : vhi;
            const unsigned long long wend_all = off[ue];       // end of the window's edges
            const bool tk = u < vhi && ((sc.mask[u >> 5] >> (u & 31)) & 1u);
            const unsigned int pay = tk ? sc.pay[u] : 0u;
            const unsigned int tmask = __ballot_sync(0xffffffffu, tk);
            const unsigned long long wend = wend_all < k1 ? wend_all : k1;
            if (tmask) {
                constexpr int kStream = 4;
                for (unsigned long long r0 = kb; r0 < wend; r0 += 32 * kStream) {
                    unsigned int dv[kStream], wv[kStream], pv[kStream];
                    bool ok[kStream];
#pragma unroll
                    for (int q = 0; q < kStream; ++q) {
                        const unsigned long long k = r0 + 32 * q + lane;
                        int own = 0;                   // largest lane whose list starts at or before k
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const unsigned long long cand = __shfl_sync(0xffffffffu, su, own + step);
                            if (cand <= k) own += step;
                        }
                        pv[q] = __shfl_sync(0xffffffffu, pay, own);
                        ok[q] = k < wend && ((tmask >> own) & 1u);
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
            }
            if (wend <= kb && ue >= vhi) {          // no vertex left to own kb: inconsistent offsets
                if (lane == 0) atomicOr(err, 32u);
                break;
            }
            if (wend > kb) kb = wend;
            u0 += 32;
        }
    }
}

}  // namespace

cudaError_t launch_second_pass(const AlgoState &st, const unsigned long long *off,
                               const unsigned int *dst, const unsigned int *w, long long shift,
                               unsigned long long src_len, unsigned long long vlo,
                               unsigned long long vhi, unsigned long long E0, unsigned long long E1,
                               const SecondPassScratch &sc, unsigned long long *edges_out,
                               unsigned int *err, cudaStream_t s) {
    if (vhi <= vlo) return cudaSuccess;
    if (vlo & 31) return cudaErrorInvalidValue;          // ranges start on a mask word
    const unsigned long long cap = 8ull * device_sms();
    unsigned long long tb = (vhi - vlo + 255) / 256;
    if (tb > cap) tb = cap;
    const unsigned long long chunks = E1 > E0 ? (E1 - 1) / kSpChunk - E0 / kSpChunk + 1 : 0ull;
    unsigned long long pb = (chunks + 7) / 8;            // one chunk per warp per round
    if (pb > cap) pb = cap;
    if (pb == 0) pb = 1;
    switch (st.algo) {
        case kBFS:
            k_sp_take<kBFS><<<(unsigned int)tb, 256, 0, s>>>(st, off, vlo, vhi, sc, edges_out);
            k_sp_push<kBFS><<<(unsigned int)pb, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, E0, E1, sc, err);
            break;
        case kSSSP:
            k_sp_take<kSSSP><<<(unsigned int)tb, 256, 0, s>>>(st, off, vlo, vhi, sc, edges_out);
            k_sp_push<kSSSP><<<(unsigned int)pb, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, E0, E1, sc, err);
            break;
        case kCC:
            k_sp_take<kCC><<<(unsigned int)tb, 256, 0, s>>>(st, off, vlo, vhi, sc, edges_out);
            k_sp_push<kCC><<<(unsigned int)pb, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, E0, E1, sc, err);
            break;
        default:
            k_sp_take<kPR><<<(unsigned int)tb, 256, 0, s>>>(st, off, vlo, vhi, sc, edges_out);
            k_sp_push<kPR><<<(unsigned int)pb, 256, 0, s>>>(st, off, dst, w, shift, src_len, vlo, vhi, E0, E1, sc, err);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relax(const AlgoState &st, const ListArrays &la, const Summary *sum,
                         const RelaxTask &t, int grid_cap, cudaStream_t s) {
    unsigned int grid = (unsigned int)grid_cap;
    if (!t.device_sized && !t.dev_edge) {
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
                          cudaStream_t s, const LoopCtl *loop) {
    unsigned int grid = (unsigned int)grid_cap;
    if (!t.device_sized && !t.dev_edge) {
        if (t.k_begin >= t.k_end) return cudaSuccess;
        const unsigned long long tiles = (t.k_end - 1) / kTile - t.k_begin / kTile + 1;
        if (tiles < grid) grid = (unsigned int)tiles;
    }
    k_gather<<<grid, kRelaxBlock, 0, s>>>(la, sum, t, out_dst, out_w, loop);
    return cudaGetLastError();
}

}  // namespace hytg
