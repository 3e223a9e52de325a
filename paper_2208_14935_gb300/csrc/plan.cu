// Cost-aware task generation on the device (Sec. V-A, Alg. 1, cost part):
//   k_count   frontier bitmap -> per-partition |A_i|, active edges and
//             128-byte lines (footnote to Eq. 3);
//   k_select  one block: the engine of every partition from Eq. 1-3 and the
//             selection rule, then the prefix sums that give each partition
//             its place in its route's list (Alg. 1 gathers the C and the Z
//             partitions into one batch each on the GPU);
//   k_bin     writes the route lists (edge base, row offset, pushed value)
//             and the tile index of the load-balanced relax kernels, takes the
//             delta of delta-PageRank, and clears the bits it consumed.
// A partition's slice of its route list is filled through one 64-bit cursor
// per partition (entries in the low 24 bits, edges above), so a warp
// reserves the entry range and the edge range of a word in one atomic.
//
// Bucketed SSSP (delta-stepping): with a bucket limit B, only active
// vertices with dist < B are eligible; the others stay set in the bitmap and
// are counted as pending, with their smallest distance, for the next bucket.
#include "common.cuh"
#include "cost_model.cuh"

namespace hytg {

namespace {

constexpr int kBatch = 4;   // bitmap words whose loads are issued together
constexpr int kPrefetch = 8;   // 128-word blocks of the bitmap a warp loads before scanning them

// This warp's share of the bitmap, in blocks of 128 words (4 rounds of 32):
// block b = warp, warp + nwarps, ...  Each lane loads 4 consecutive words
// with one 16-byte load, kPrefetch blocks at a time, so their latencies
// overlap; a round (32 words) whose words are all zero -- most of them when
// the frontier is small -- is skipped.  body(rd, bits) sees each remaining
// round's index and this lane's word of it (reloaded: a cache hit).  The
// walk only reads the bitmap; body may rewrite its own round's words.
// The bitmap is padded to a multiple of 32 words, so a block's 4-word group
// is either wholly inside it or wholly outside.
template <class F>
__device__ __forceinline__ void for_rounds(const unsigned int *bm, unsigned long long n_rounds, F &&body) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long n_words = n_rounds * 32;
    const unsigned long long n_blocks = (n_rounds + 3) / 4;
    const uint4 *bm4 = reinterpret_cast<const uint4 *>(bm);
    for (unsigned long long b0 = w; b0 < n_blocks; b0 += nwarps * kPrefetch) {
        uint4 pre[kPrefetch];
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) {
            const unsigned long long blk = b0 + (unsigned long long)j * nwarps;
            const unsigned long long word = blk * 128 + 4 * lane;
            pre[j] = (blk < n_blocks && word < n_words) ? bm4[word / 4] : make_uint4(0u, 0u, 0u, 0u);
        }
        // live: bit 4 j + r for round r of block j; lanes 8 r .. 8 r + 7 hold round r
        unsigned int live = 0;
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) {
            const unsigned int nzl = __ballot_sync(0xffffffffu, (pre[j].x | pre[j].y | pre[j].z | pre[j].w) != 0u);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if ((nzl >> (8 * r)) & 0xFFu) live |= 1u << (4 * j + r);
        }
        while (live) {                              // warp-uniform
            const int q = __ffs(live) - 1;
            live &= live - 1;
            const unsigned long long rd = (b0 + (unsigned long long)(q >> 2) * nwarps) * 4 + (q & 3);
            body(rd, bm[rd * 32 + lane]);
        }
    }
}

// Partition holding bitmap word `widx` (bounds are word indices): the
// partition of the word's 32-word round from the round table, then forward
// over the partition bounds inside the round (partitions are whole words, so
// at most 31 steps, in practice none or one).
__device__ __forceinline__ unsigned int find_part(const GraphDev &g, unsigned long long widx) {
    unsigned int p = __ldg(&g.round_part[widx >> 5]);
    while (p + 1 < g.N && (unsigned long long)__ldg(&g.part_wb[p + 1]) <= widx) ++p;
    return p;
}

// Up to kBatch nonzero words of this warp's 32-word round, in order.
__device__ __forceinline__ void next_batch(unsigned int &nz, unsigned int bits,
                                           unsigned long long wbase, unsigned int (&wq)[kBatch],
                                           unsigned long long (&wi)[kBatch]) {
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
        wq[q] = 0;
        wi[q] = 0;
        if (nz) {                      // warp-uniform
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            wq[q] = __shfl_sync(0xffffffffu, bits, src);
            wi[q] = wbase + src;
        }
    }
}

__global__ void __launch_bounds__(256) k_count(GraphDev g, AlgoState st, PartArrays pa,
                                               unsigned long long m) {
    if (st.loop) st.bucket_limit = st.loop->bucket;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_rounds = g.n_words_alloc / 32;
    const bool bucketed = st.bucket_limit != 0xFFFFFFFFu;
    unsigned long long pend = 0;
    unsigned int pend_min = 0xFFFFFFFFu;
    for_rounds(st.bm_cur, n_rounds, [&](unsigned long long rd, unsigned int bits) {
        unsigned int cur_p = 0xFFFFFFFFu;
        unsigned long long p_lo = 1, p_hi = 0;   // word range of cur_p
        unsigned long long a_nact = 0, a_ent = 0, a_edges = 0, a_lines = 0, a_prio = 0;
        const unsigned long long wbase = rd * 32;
        unsigned int nz = __ballot_sync(0xffffffffu, bits != 0);
        while (nz) {
            unsigned int wq[kBatch];
            unsigned long long wi[kBatch], o0[kBatch], o1[kBatch];
            unsigned int dv[kBatch];
            float dl[kBatch];
            next_batch(nz, bits, wbase, wq, wi);
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                o0[q] = o1[q] = 0;
                dv[q] = 0;
                dl[q] = 0.f;
                if ((wq[q] >> lane) & 1u) {
                    const unsigned long long v = wi[q] * 32 + lane;
                    o0[q] = g.off[v];
                    o1[q] = g.off[v + 1];
                    if (bucketed) dv[q] = st.val[v];
                    if (st.prio) dl[q] = st.delta[v];
                }
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                if (wq[q] == 0) continue;          // warp-uniform
                const unsigned long long widx = wi[q];
                bool act = (wq[q] >> lane) & 1u;
                if (bucketed && act && dv[q] >= st.bucket_limit) {
                    ++pend;
                    pend_min = min(pend_min, dv[q]);
                    act = false;
                }
                const unsigned int elig = __ballot_sync(0xffffffffu, act);
                if (elig == 0) continue;
                if (widx < p_lo || widx >= p_hi) {
                    if (cur_p != 0xFFFFFFFFu && lane == 0 && a_nact) {
                        atomicAdd(&pa.n_act[cur_p], a_nact);
                        atomicAdd(&pa.entries[cur_p], a_ent);
                        atomicAdd(&pa.edges[cur_p], a_edges);
                        atomicAdd(&pa.lines[cur_p], a_lines);
                        if (st.prio) atomicAdd(&pa.prio[cur_p], a_prio);
                    }
                    a_nact = a_ent = a_edges = a_lines = a_prio = 0;
                    cur_p = find_part(g, widx);
                    p_lo = g.part_wb[cur_p];
                    p_hi = g.part_wb[cur_p + 1];
                }
                const unsigned long long deg = act ? o1[q] - o0[q] : 0ull;
                const unsigned long long ln =
                    (unsigned long long)st.n_arrays * lines_spanned(o0[q] * 4ull, deg * 4ull, m);
                a_nact += __popc(elig);
                a_ent += __popc(__ballot_sync(0xffffffffu, deg > 0));
                a_edges += warp_sum_lt43(deg);
                a_lines += warp_sum_lt43(ln);
                if (st.prio) {
                    // |delta| in units of 2^-24, capped at 2^40 per vertex; the
                    // sum only orders the F tasks, so rounding cannot matter
                    const float x = fminf(fabsf(dl[q]) * 16777216.f, 1099511627776.f);
                    a_prio += warp_sum_lt43(act ? (unsigned long long)x : 0ull);
                }
            }
        }
        if (lane == 0 && cur_p != 0xFFFFFFFFu && a_nact) {
            atomicAdd(&pa.n_act[cur_p], a_nact);
            atomicAdd(&pa.entries[cur_p], a_ent);
            atomicAdd(&pa.edges[cur_p], a_edges);
            atomicAdd(&pa.lines[cur_p], a_lines);
            if (st.prio) atomicAdd(&pa.prio[cur_p], a_prio);
        }
    });
    if (bucketed) {
        pend = warp_sum_u64(pend);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pend_min = min(pend_min, __shfl_xor_sync(0xffffffffu, pend_min, o));
        if (lane == 0 && pend) {
            atomicAdd(pa.pending, pend);
            atomicMax(pa.pending_inv, (unsigned long long)(~pend_min));   // max of ~d = ~min d
        }
    }
}

// ------------------------------------------------------------- k_select
// Exclusive block scan of K u64 values per thread (kSelectBlock threads).
template <int K>
__device__ void block_scan_excl(unsigned long long (&v)[K], unsigned long long (&total)[K],
                                unsigned long long *smem /* 33 * K */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long incl[K];
#pragma unroll
    for (int q = 0; q < K; ++q) incl[q] = warp_scan_u64(v[q]);
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < K; ++q) smem[wid * K + q] = incl[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            unsigned long long x = lane < nw ? smem[lane * K + q] : 0ull;
            unsigned long long xi = warp_scan_u64(x);
            if (lane < nw) smem[lane * K + q] = xi - x;      // exclusive warp offsets
            if (lane == 31) smem[32 * K + q] = xi;           // block total
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        total[q] = smem[32 * K + q];
        v[q] = smem[wid * K + q] + incl[q] - v[q];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSelectBlock) k_select(GraphDev g, PartArrays pa, CostParams cp,
                                                         Summary *sum) {
    __shared__ unsigned long long smem[33 * 11];
    const unsigned int N = g.N;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (unsigned int p = tid; p < N; p += nt)
        pa.route[p] = (unsigned char)decide_route_counts(p, g.part_eb[p + 1] - g.part_eb[p], pa.n_act[p],
                                                         pa.edges[p], pa.lines[p], cp);
    __syncthreads();

    // per-route prefixes over partitions (contiguous chunk per thread)
    const unsigned int ppt = (N + nt - 1) / nt;
    const unsigned int p0 = min(N, tid * ppt), p1 = min(N, p0 + ppt);
    unsigned long long v[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) v[q] = 0;
    unsigned long long red[11];
#pragma unroll
    for (int q = 0; q < 11; ++q) red[q] = 0;
    for (unsigned int p = p0; p < p1; ++p) {
        const int r = pa.route[p];
        const unsigned long long ent = pa.entries[p], edg = pa.edges[p], lin = pa.lines[p];
        // compile-time indices keep v[] and red[] in registers
#pragma unroll
        for (int q = 0; q < kRoutes; ++q) {
            if (r == q) {
                v[q] += ent;
                v[kRoutes + q] += edg;
                red[q] += lin;
                red[kRoutes + q] += 1;
            }
        }
        red[10] += pa.n_act[p];
    }
    unsigned long long tot[10];
    block_scan_excl<10>(v, tot, smem);
    unsigned long long redtot[11];
    block_scan_excl<11>(red, redtot, smem);

    unsigned long long ebase[kRoutes], tbase[kRoutes];
    {
        unsigned long long e = 0, t = 0;
        for (int r = 0; r < kRoutes; ++r) {
            ebase[r] = e;
            tbase[r] = t;
            e += tot[r];
            t += (tot[kRoutes + r] + kTile - 1) / kTile;
        }
    }
    for (unsigned int p = p0; p < p1; ++p) {
        const int r = pa.route[p];
        const unsigned long long ent = pa.entries[p], edg = pa.edges[p];
#pragma unroll
        for (int q = 0; q < kRoutes; ++q) {
            if (r == q) {
                pa.route_entry[p] = v[q];
                pa.route_edge[p] = v[kRoutes + q];
                v[q] += ent;
                v[kRoutes + q] += edg;
            }
        }
    }
    if (tid == 0) {
        sum->n_active = redtot[10];
        for (int r = 0; r < kRoutes; ++r) {
            sum->route_entries[r] = tot[r];
            sum->route_edges[r] = tot[kRoutes + r];
            sum->route_lines[r] = redtot[r];
            sum->route_parts[r] = (unsigned int)redtot[kRoutes + r];
            sum->route_entry_base[r] = ebase[r];
            sum->route_tile_base[r] = tbase[r];
        }
        sum->pending = *pa.pending;
        sum->pending_min = ~(unsigned int)(*pa.pending_inv);
        sum->alive = pa.alive ? *pa.alive : 0ull;
    }
}

// ---------------------------------------------------------------- k_bin
__global__ void __launch_bounds__(256) k_bin(GraphDev g, AlgoState st, PartArrays pa, ListArrays la,
                                             const Summary *sum) {
    if (st.loop) {
        if (!st.loop->work) return;
        st.bucket_limit = st.loop->bucket;
    }
    const int lane = threadIdx.x & 31;
    const unsigned int lt_mask = (1u << lane) - 1u;
    const unsigned long long n_rounds = g.n_words_alloc / 32;
    const bool batched = st.batch_mode != kBatchNone;
    const bool is_pr = !batched && (st.algo == kPR || st.algo == kPPR);
    const bool bucketed = st.bucket_limit != 0xFFFFFFFFu;
    unsigned long long work = 0;
    for_rounds(st.bm_cur, n_rounds, [&](unsigned long long rd, unsigned int bits) {
        unsigned int cur_p = 0xFFFFFFFFu;
        unsigned long long p_lo = 1, p_hi = 0, rbase = 0, tbase = 0, pe0 = 0, pg0 = 0;
        const unsigned long long wbase = rd * 32;
        unsigned int keep = bits;                       // bits left for a later bucket
        unsigned int nz = __ballot_sync(0xffffffffu, bits != 0);
        while (nz) {
            unsigned int wq[kBatch];
            unsigned long long wi[kBatch], o0[kBatch], o1[kBatch];
            unsigned int vv[kBatch];
            float rk[kBatch];
            unsigned long long bf[kBatch];
            next_batch(nz, bits, wbase, wq, wi);
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                o0[q] = o1[q] = 0;
                vv[q] = 0;
                rk[q] = 0.0f;
                bf[q] = 0;
                if ((wq[q] >> lane) & 1u) {
                    const unsigned long long v = wi[q] * 32 + lane;
                    o0[q] = g.off[v];
                    o1[q] = g.off[v + 1];
                    if (batched) bf[q] = st.batch_mode == kBatchPPR ? st.b_fr32[v] : st.b_fr[v];
                    else if (is_pr) { vv[q] = __float_as_uint(st.delta[v]); rk[q] = st.rank[v]; }
                    else vv[q] = st.val[v];
                }
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                if (wq[q] == 0) continue;          // warp-uniform
                const unsigned long long widx = wi[q];
                bool act = (wq[q] >> lane) & 1u;
                if (bucketed && act && vv[q] >= st.bucket_limit) act = false;
                const unsigned int elig = __ballot_sync(0xffffffffu, act);
                if (elig == 0) continue;
                if (lane == (int)(widx - wbase)) keep = wq[q] & ~elig;
                if (widx < p_lo || widx >= p_hi) {
                    cur_p = find_part(g, widx);
                    p_lo = g.part_wb[cur_p];
                    p_hi = g.part_wb[cur_p + 1];
                    const int rp = pa.route[cur_p];
                    rbase = sum->route_entry_base[rp];
                    tbase = sum->route_tile_base[rp];
                    pe0 = pa.route_entry[cur_p];
                    pg0 = pa.route_edge[cur_p];
                }
                const unsigned long long v = widx * 32 + lane;
                const unsigned long long deg = act ? o1[q] - o0[q] : 0ull;
                unsigned int pay = 0;
                if (act) {
                    if (is_pr) {
                        // take the accumulated delta (Sec. VI-A delta-based PageRank)
                        const float dl = __uint_as_float(vv[q]);
                        st.delta[v] = 0.0f;
                        st.rank[v] = rk[q] + dl;
                        pay = __float_as_uint(deg ? st.damping * dl / (float)deg : 0.0f);
                    } else {
                        pay = vv[q];
                    }
                }
                const unsigned int bal = __ballot_sync(0xffffffffu, deg > 0);
                const unsigned long long incl = warp_scan_small(deg);
                const unsigned long long w_edges = __shfl_sync(0xffffffffu, incl, 31);
                unsigned long long old = 0;
                if (lane == 0 && bal)
                    old = atomicAdd(&pa.cursor[cur_p], (w_edges << 24) | (unsigned long long)__popc(bal));
                old = __shfl_sync(0xffffffffu, old, 0);
                if (deg > 0) {
                    const unsigned long long idx = rbase + pe0 + (old & 0xFFFFFFull) + __popc(bal & lt_mask);
                    const unsigned long long eb = pg0 + (old >> 24) + (incl - deg);
                    const unsigned long long t0 = (eb + kTile - 1) / kTile;
                    const unsigned long long t1 = (eb + deg - 1) / kTile;
                    if (idx >= la.cap_entries || (t0 <= t1 && tbase + t1 >= la.cap_tiles)) {
                        atomicOr(la.err, 2u);
                    } else {
                        la.ebase[idx] = eb;
                        la.soff[idx] = o0[q];
                        la.pay[idx] = pay;
                        if (batched) {
                            la.pay64[idx] = bf[q];
                            la.vid[idx] = (unsigned int)v;
                            work += (unsigned long long)__popcll(bf[q]) * deg;
                        }
                        const unsigned int rel = (unsigned int)(idx - rbase);
                        for (unsigned long long t = t0; t <= t1; ++t) la.tile_first[tbase + t] = rel;
                    }
                }
            }
        }
        if (keep != bits) st.bm_cur[wbase + lane] = keep;
    });
    if (batched) {
        work = warp_sum_u64(work);
        if (lane == 0 && work) atomicAdd(st.src_work, work);
    }
}

}  // namespace

// Blocks of 256 threads that fit on the device at once for `kernel`.
template <class K>
unsigned long long resident_blocks(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 2ull * device_sms();
    return (unsigned long long)sms * (unsigned long long)per_sm;
}

// Grid of a bitmap walk: one resident wave, at most one round per warp.
unsigned long long walk_blocks(unsigned long long rounds, unsigned long long resident) {
    unsigned long long blocks = (rounds + 7) / 8;
    return blocks < resident ? blocks : resident;
}

cudaError_t launch_count(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                         unsigned long long m, cudaStream_t s) {
    const unsigned long long rounds = g.n_words_alloc / 32;
    if (rounds == 0) return cudaSuccess;
    static const unsigned long long resident = resident_blocks(k_count);
    const unsigned long long blocks = walk_blocks(rounds, resident);
    k_count<<<(unsigned int)blocks, 256, 0, s>>>(g, st, pa, m);
    return cudaGetLastError();
}

cudaError_t launch_select(const GraphDev &g, const PartArrays &pa, const CostParams &cp,
                          Summary *sum, cudaStream_t s) {
    k_select<<<1, kSelectBlock, 0, s>>>(g, pa, cp, sum);
    return cudaGetLastError();
}

cudaError_t launch_bin(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                       const ListArrays &la, const Summary *sum, cudaStream_t s) {
    const unsigned long long rounds = g.n_words_alloc / 32;
    if (rounds == 0) return cudaSuccess;
    static const unsigned long long resident = resident_blocks(k_bin);
    const unsigned long long blocks = walk_blocks(rounds, resident);
    k_bin<<<(unsigned int)blocks, 256, 0, s>>>(g, st, pa, la, sum);
    return cudaGetLastError();
}

}  // namespace hytg
