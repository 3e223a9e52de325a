// Cost-aware task generation on the device (Sec. V-A, Alg. 1, cost part):
//   k_count   frontier bitmap -> per-partition |A_i|, active edges, 128-byte
//             lines (footnote to Eq. 3), and per-segment totals for the
//             ordered compaction;
//   k_select  one block: the engine of every partition from Eq. 1-3 and the
//             selection rule, then the prefix sums that place each partition's
//             active vertices in its route's list ("pre-combine on GPU",
//             Alg. 1 lines for Vc and Vz);
//   k_bin     writes the route lists (edge base, row offset, pushed value)
//             and the tile index of the load-balanced relax kernels, takes the
//             delta of delta-PageRank, and clears the consumed bitmap.
#include "common.cuh"
#include "cost_model.cuh"

namespace hytg {

namespace {

constexpr int kBatch = 4;   // bitmap words whose loads are issued together

// Partition holding bitmap word `widx` (bounds are word indices).
__device__ __forceinline__ unsigned int find_part(const unsigned int *wb, unsigned int N,
                                                  unsigned long long widx) {
    unsigned int lo = 0, hi = N;  // invariant: wb[lo] <= widx < wb[hi]
    while (hi - lo > 1) {
        unsigned int mid = (lo + hi) >> 1;
        if ((unsigned long long)__ldg(&wb[mid]) <= widx) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_count(GraphDev g, AlgoState st, PartArrays pa,
                                               SegArrays sa, unsigned long long m) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned int elem = 4;
    for (unsigned long long seg = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         seg < g.n_segs; seg += nwarps) {
        unsigned long long seg_ent = 0, seg_edges = 0;
        unsigned int cur_p = 0xFFFFFFFFu;
        unsigned long long p_lo = 1, p_hi = 0;   // word range of cur_p
        unsigned long long a_nact = 0, a_ent = 0, a_edges = 0, a_lines = 0;
        for (int r = 0; r < kSegWords / 32; ++r) {
            const unsigned long long wbase = seg * kSegWords + r * 32;
            const unsigned int bits = st.bm_cur[wbase + lane];
            unsigned int nz = __ballot_sync(0xffffffffu, bits != 0);
            while (nz) {
                unsigned int wq[kBatch];
                unsigned long long wi[kBatch], o0[kBatch], o1[kBatch];
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
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    o0[q] = o1[q] = 0;
                    if ((wq[q] >> lane) & 1u) {
                        const unsigned long long v = wi[q] * 32 + lane;
                        o0[q] = g.off[v];
                        o1[q] = g.off[v + 1];
                    }
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                if (wq[q] == 0) continue;          // warp-uniform
                const unsigned int w = wq[q];
                const unsigned long long widx = wi[q];
                if (widx < p_lo || widx >= p_hi) {
                    if (cur_p != 0xFFFFFFFFu && lane == 0 && a_nact) {
                        atomicAdd(&pa.n_act[cur_p], a_nact);
                        atomicAdd(&pa.entries[cur_p], a_ent);
                        atomicAdd(&pa.edges[cur_p], a_edges);
                        atomicAdd(&pa.lines[cur_p], a_lines);
                    }
                    a_nact = a_ent = a_edges = a_lines = 0;
                    cur_p = find_part(g.part_wb, g.N, widx);
                    p_lo = g.part_wb[cur_p];
                    p_hi = g.part_wb[cur_p + 1];
                }
                const unsigned long long deg = o1[q] - o0[q];
                const unsigned long long ln =
                    (unsigned long long)st.n_arrays * lines_spanned(o0[q] * elem, deg * elem, m);
                const unsigned int ent = __popc(__ballot_sync(0xffffffffu, deg > 0));
                const unsigned long long e_sum = warp_sum_u64(deg);
                const unsigned long long l_sum = warp_sum_u64(ln);
                a_nact += __popc(w);
                a_ent += ent;
                a_edges += e_sum;
                a_lines += l_sum;
                seg_ent += ent;
                seg_edges += e_sum;
                }
            }
        }
        if (lane == 0) {
            if (cur_p != 0xFFFFFFFFu && a_nact) {
                atomicAdd(&pa.n_act[cur_p], a_nact);
                atomicAdd(&pa.entries[cur_p], a_ent);
                atomicAdd(&pa.edges[cur_p], a_edges);
                atomicAdd(&pa.lines[cur_p], a_lines);
            }
            sa.entries[seg] = seg_ent;
            sa.edges[seg] = seg_edges;
        }
    }
}

// ------------------------------------------------------------- k_select
// Exclusive block scan of K u64 values per thread (kSelectBlock threads).
template <int K>
__device__ void block_scan_excl(unsigned long long (&v)[K], unsigned long long (&total)[K],
                                unsigned long long *smem /* 32 * K */) {
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

__global__ void __launch_bounds__(kSelectBlock) k_select(GraphDev g, PartArrays pa, SegArrays sa,
                                                         CostParams cp, Summary *sum) {
    __shared__ unsigned long long smem[33 * 12];
    const unsigned int N = g.N;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (unsigned int p = tid; p < N; p += nt)
        pa.route[p] = (unsigned char)decide_route_counts(p, g.part_eb[p + 1] - g.part_eb[p], pa.n_act[p],
                                                         pa.edges[p], pa.lines[p], cp);
    __syncthreads();

    // per-route and global prefixes over partitions (contiguous chunk per thread)
    const unsigned int ppt = (N + nt - 1) / nt;
    const unsigned int p0 = min(N, tid * ppt), p1 = min(N, p0 + ppt);
    unsigned long long v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = 0;
    unsigned long long lines_r[kRoutes] = {0, 0, 0, 0, 0}, parts_r[kRoutes] = {0, 0, 0, 0, 0},
                       nact = 0;
    for (unsigned int p = p0; p < p1; ++p) {
        const int r = pa.route[p];
        v[r] += pa.entries[p];
        v[kRoutes + r] += pa.edges[p];
        v[10] += pa.entries[p];
        v[11] += pa.edges[p];
        lines_r[r] += pa.lines[p];
        parts_r[r] += 1;
        nact += pa.n_act[p];
    }
    unsigned long long tot[12];
    block_scan_excl<12>(v, tot, smem);
    unsigned long long red[11];
#pragma unroll
    for (int r = 0; r < kRoutes; ++r) { red[r] = lines_r[r]; red[kRoutes + r] = parts_r[r]; }
    red[10] = nact;
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
        pa.route_entry[p] = v[r];
        pa.route_edge[p] = v[kRoutes + r];
        pa.entry_delta[p] = ebase[r] + v[r] - v[10];      // modulo 2^64
        pa.edge_delta[p] = v[kRoutes + r] - v[11];
        v[r] += pa.entries[p];
        v[kRoutes + r] += pa.edges[p];
        v[10] += pa.entries[p];
        v[11] += pa.edges[p];
    }

    // exclusive prefix over bitmap segments
    const unsigned long long S = g.n_segs;
    const unsigned long long spt = (S + nt - 1) / nt;
    const unsigned long long s0 = min(S, (unsigned long long)tid * spt), s1 = min(S, s0 + spt);
    unsigned long long sv[2] = {0, 0}, stot[2];
    for (unsigned long long s = s0; s < s1; ++s) { sv[0] += sa.entries[s]; sv[1] += sa.edges[s]; }
    block_scan_excl<2>(sv, stot, smem);
    for (unsigned long long s = s0; s < s1; ++s) {
        sa.entry_prefix[s] = sv[0];
        sa.edge_prefix[s] = sv[1];
        sv[0] += sa.entries[s];
        sv[1] += sa.edges[s];
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
    }
}

// ---------------------------------------------------------------- k_bin
__global__ void __launch_bounds__(256) k_bin(GraphDev g, AlgoState st, PartArrays pa, SegArrays sa,
                                             ListArrays la, const Summary *sum) {
    const int lane = threadIdx.x & 31;
    const unsigned int lt_mask = (1u << lane) - 1u;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const bool is_pr = st.algo == kPR || st.algo == kPPR;
    for (unsigned long long seg = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         seg < g.n_segs; seg += nwarps) {
        unsigned long long run_ent = sa.entry_prefix[seg], run_edg = sa.edge_prefix[seg];
        unsigned int cur_p = 0xFFFFFFFFu;
        unsigned long long p_lo = 1, p_hi = 0, ed = 0, gd = 0, rbase = 0, tbase = 0;
        int rp = 0;
        for (int r = 0; r < kSegWords / 32; ++r) {
            const unsigned long long wbase = seg * kSegWords + r * 32;
            const unsigned int bits = st.bm_cur[wbase + lane];
            if (bits) st.bm_cur[wbase + lane] = 0u;
            unsigned int nz = __ballot_sync(0xffffffffu, bits != 0);
            while (nz) {
                // up to kBatch nonzero words at once: their loads are issued
                // together before the per-word scans (latency hiding)
                unsigned int wq[kBatch];
                unsigned long long wi[kBatch], o0[kBatch], o1[kBatch];
                unsigned int vv[kBatch];
                float rk[kBatch];
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
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    o0[q] = o1[q] = 0;
                    vv[q] = 0;
                    rk[q] = 0.0f;
                    if ((wq[q] >> lane) & 1u) {
                        const unsigned long long v = wi[q] * 32 + lane;
                        o0[q] = g.off[v];
                        o1[q] = g.off[v + 1];
                        if (is_pr) { vv[q] = __float_as_uint(st.delta[v]); rk[q] = st.rank[v]; }
                        else vv[q] = st.val[v];
                    }
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                if (wq[q] == 0) continue;          // warp-uniform
                const unsigned int w = wq[q];
                const unsigned long long widx = wi[q];
                if (widx < p_lo || widx >= p_hi) {
                    cur_p = find_part(g.part_wb, g.N, widx);
                    p_lo = g.part_wb[cur_p];
                    p_hi = g.part_wb[cur_p + 1];
                    rp = pa.route[cur_p];
                    ed = pa.entry_delta[cur_p];
                    gd = pa.edge_delta[cur_p];
                    rbase = sum->route_entry_base[rp];
                    tbase = sum->route_tile_base[rp];
                }
                const bool active = (w >> lane) & 1u;
                const unsigned long long v = widx * 32 + lane;
                const unsigned long long deg = o1[q] - o0[q];
                unsigned int pay = 0;
                if (active) {
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
                const bool is_ent = deg > 0;
                const unsigned int bal = __ballot_sync(0xffffffffu, is_ent);
                const unsigned long long incl = warp_scan_u64(deg);
                if (is_ent) {
                    const unsigned long long idx = run_ent + __popc(bal & lt_mask) + ed;
                    const unsigned long long eb = run_edg + (incl - deg) + gd;
                    const unsigned long long t0 = (eb + kTile - 1) / kTile;
                    const unsigned long long t1 = (eb + deg - 1) / kTile;
                    if (idx >= la.cap_entries || (t0 <= t1 && tbase + t1 >= la.cap_tiles)) {
                        atomicOr(la.err, 2u);
                    } else {
                        la.ebase[idx] = eb;
                        la.soff[idx] = o0[q];
                        la.pay[idx] = pay;
                        const unsigned int rel = (unsigned int)(idx - rbase);
                        for (unsigned long long t = t0; t <= t1; ++t) la.tile_first[tbase + t] = rel;
                    }
                }
                run_ent += __popc(bal);
                run_edg += __shfl_sync(0xffffffffu, incl, 31);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_count(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                         const SegArrays &sa, unsigned long long m, cudaStream_t s) {
    if (g.n_segs == 0) return cudaSuccess;
    const unsigned long long warps = g.n_segs;
    unsigned long long blocks = (warps + 7) / 8;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    k_count<<<(unsigned int)blocks, 256, 0, s>>>(g, st, pa, sa, m);
    return cudaGetLastError();
}

cudaError_t launch_select(const GraphDev &g, const PartArrays &pa, const SegArrays &sa,
                          const CostParams &cp, Summary *sum, cudaStream_t s) {
    k_select<<<1, kSelectBlock, 0, s>>>(g, pa, sa, cp, sum);
    return cudaGetLastError();
}

cudaError_t launch_bin(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                       const SegArrays &sa, const ListArrays &la, const Summary *sum,
                       cudaStream_t s) {
    if (g.n_segs == 0) return cudaSuccess;
    unsigned long long blocks = (g.n_segs + 7) / 8;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    k_bin<<<(unsigned int)blocks, 256, 0, s>>>(g, st, pa, sa, la, sum);
    return cudaGetLastError();
}

}  // namespace hytg
