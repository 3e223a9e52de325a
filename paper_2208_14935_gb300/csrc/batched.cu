// Batched runs: up to 64 BFS or SSSP sources, or up to 32 personalised
// PageRank seeds, share one run and therefore every partition transfer.  The
// planner works on the union frontier (bit v set when v is active for any
// source), so each partition's edges cross the host link once per iteration
// for all sources together.
//
// Per-vertex state (values in frames of 8 sources, see BatchState):
//   BFS/SSSP  fr[v], vis[v], nxt[v]  64-bit source masks (frontier, reached,
//             reached or improved this iteration); *bval(v, s) level or
//             distance of source s.
//   PPR       *bdelta(v, s), *brank(v, s), *bmsg(v, s) (the push of seed s
//             taken this iteration), fr32[v] mask of seeds taken.
#include "common.cuh"
#include "relax_tile.cuh"

namespace hytg {

namespace {

inline unsigned int grid_for(unsigned long long n, unsigned int block) {
    unsigned long long g = (n + block - 1) / block;
    const unsigned long long cap = 32ull * device_sms();
    if (g > cap) g = cap;
    return g == 0 ? 1u : (unsigned int)g;
}

__global__ void k_frame_init(BatchState b, unsigned long long V, unsigned int g) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long n = V * kFrameSources;
    if (b.mode == kBatchPPR) {
        // messages too: the vector push adds a whole frame's messages
        for (unsigned long long i = t0; i < n; i += stride) {
            b.delta[g][i] = 0.0f;
            b.rank[g][i] = 0.0f;
            b.msg[g][i] = 0.0f;
        }
    } else {
        for (unsigned long long i = t0; i < n; i += stride) b.val[g][i] = 0xFFFFFFFFu;
    }
}

// Masks and bitmap of a new run (the frames are filled by k_frame_init).
__global__ void k_b_init(BatchState b, unsigned long long V, unsigned long long n_words_alloc,
                         unsigned int *bm) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (b.mode == kBatchPPR) {
        for (unsigned long long v = t0; v < V; v += stride) b.fr32[v] = 0;
    } else {
        for (unsigned long long v = t0; v < V; v += stride) {
            b.fr[v] = 0;
            b.vis[v] = 0;
            b.nxt[v] = 0;
        }
    }
    for (unsigned long long w = t0; w < n_words_alloc; w += stride) bm[w] = 0;
}

// Sources (internal ids) enter the frontier.  One thread per source.
__global__ void k_b_sources(BatchState b, const unsigned int *src, unsigned int K, float base,
                            unsigned int *bm) {
    const unsigned int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= K) return;
    const unsigned int v = src[s];
    if (b.mode == kBatchPPR) {
        *bdelta(b, v, s) = base;
    } else {
        atomicOr(&b.fr[v], 1ull << s);
        atomicOr(&b.vis[v], 1ull << s);
        *bval(b, v, s) = 0u;
    }
    atomicOr(&bm[v >> 5], 1u << (v & 31));
}

// BFS/SSSP after an iteration: the improved sources of v become its frontier.
// BFS also records the level of each newly reached source.  One warp per 32
// vertices so the bitmap word is written whole (the binning pass cleared it).
__global__ void k_b_commit(BatchState b, unsigned long long V, unsigned long long n_words_alloc,
                           unsigned int level, unsigned int *bm) {
    if (b.loop) level = b.loop->it;
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         w < n_words_alloc; w += nw) {
        const unsigned long long v = w * 32 + lane;
        unsigned long long n = 0;
        if (v < V) {
            n = b.nxt[v];
            if (b.mode == kBatchBFS && n) {
                n &= ~b.vis[v];
                b.vis[v] |= n;
                unsigned long long m = n;
                while (m) {
                    const int s = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    *bval(b, v, (unsigned int)s) = level;
                }
            }
            b.fr[v] = n;
            if (b.nxt[v]) b.nxt[v] = 0;
        }
        const unsigned int word = __ballot_sync(0xffffffffu, n != 0);
        if (lane == 0) bm[w] = word;
        if (b.alive && word) {
            unsigned long long orv = n;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) orv |= __shfl_xor_sync(0xffffffffu, orv, o);
            if (lane == 0) atomicOr(b.alive, orv);
        }
    }
}

// PPR: for every vertex marked in the bitmap, take the residual of each seed
// above eps (rank += delta, delta = 0, msg = d * delta / D_o) and keep the
// vertex in the frontier iff some seed was taken.  One warp per bitmap word,
// lanes are seeds.
__global__ void k_b_take(BatchState b, const unsigned long long *off, unsigned long long n_words_alloc,
                         unsigned int K, float damping, float eps, unsigned int *bm) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         w < n_words_alloc; w += nw) {
        unsigned int bits = bm[w];
        if (bits == 0) continue;
        unsigned int keep = 0;
        unsigned int seen = 0;
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            const unsigned long long v = w * 32 + bit;
            const unsigned long long deg = off[v + 1] - off[v];
            // lanes are seeds; a seed past K, or in a frame not allocated, has no state
            const bool has = lane < (int)K && b.delta[lane >> 3] != nullptr;
            const float dl = has ? *bdelta(b, v, lane) : 0.0f;
            const bool act = has && dl > eps;
            float msg = 0.0f;
            if (act) {
                *bdelta(b, v, lane) = 0.0f;
                *brank(b, v, lane) += dl;
                msg = deg ? damping * dl / (float)deg : 0.0f;
            }
            if (has) *bmsg(b, v, lane) = msg;
            const unsigned int mask = __ballot_sync(0xffffffffu, act);
            if (lane == 0) b.fr32[v] = mask;
            if (mask) keep |= 1u << bit;
            seen |= mask;
        }
        if (lane == 0) {
            bm[w] = keep;
            if (b.alive && seen) atomicOr(b.alive, (unsigned long long)seen);
        }
    }
}

// Serving: clear one slot's column, then seed its source (at an iteration
// boundary: no relax of the slot is in flight, and the slot's source enters
// through nxt / delta so that the next commit or take activates it).
__global__ void k_serve_clear(BatchState b, unsigned long long V, unsigned int slot) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long bit = 1ull << slot;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride) {
        if (b.mode == kBatchPPR) {
            *bdelta(b, v, slot) = 0.0f;
            *brank(b, v, slot) = 0.0f;
        } else {
            *bval(b, v, slot) = 0xFFFFFFFFu;
            if (b.fr[v] & bit) b.fr[v] &= ~bit;
            if (b.vis[v] & bit) b.vis[v] &= ~bit;
            if (b.nxt[v] & bit) b.nxt[v] &= ~bit;
        }
    }
}
__global__ void k_serve_seed(BatchState b, unsigned int slot, unsigned int src, float base,
                             unsigned int *bm) {
    if (b.mode == kBatchPPR) {
        *bdelta(b, src, slot) = base;
        atomicOr(&bm[src >> 5], 1u << (src & 31));
    } else {
        if (b.mode == kBatchSSSP) *bval(b, src, slot) = 0u;
        atomicOr(&b.nxt[src], 1ull << slot);
    }
}

// One finished slot's result in original vertex order: BFS levels relative to
// the slot's admission iteration, SSSP distances, PPR ranks normalised.
__global__ void k_serve_extract(BatchState b, unsigned long long V, unsigned int slot,
                                const unsigned int *perm, unsigned int offset, void *out,
                                const double *sums) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride) {
        const unsigned long long ov = perm ? perm[v] : v;
        if (b.mode == kBatchPPR) {
            const double S = sums[slot];
            ((float *)out)[ov] = S > 0.0 ? (float)((double)*brank(b, v, slot) / S) : 0.0f;
        } else {
            const unsigned int x = *bval(b, v, slot);
            ((unsigned int *)out)[ov] = (x == 0xFFFFFFFFu || b.mode != kBatchBFS) ? x : x - offset;
        }
    }
}

// Multi-source BFS relax: one thread per edge; the sources of u not yet
// reached at v are ORed into nxt[v].
__global__ void __launch_bounds__(kRelaxBlock) k_relax_msbfs(BatchState b, ListArrays la,
                                                             const Summary *sum, RelaxTask t) {
    __shared__ TileSmem<true> sm;
    if (b.loop && !b.loop->work) return;
    unsigned long long kb, ke;
    task_range(t, sum, kb, ke);
    if (kb >= ke) return;
    const unsigned long long t_first = kb / kTile, t_last = (ke - 1) / kTile;
    for (unsigned long long tile = t_first + blockIdx.x; tile <= t_last; tile += gridDim.x) {
        unsigned long long k0;
        const int n = tile_setup<true>(sm, la, sum, t, tile, kb, ke, &k0);
        if (t.link_ctr) count_link_reads<true>(sm, k0, n, 1u, t.link_ctr);
        unsigned int dv[kRelaxIPT];
        unsigned long long fv[kRelaxIPT];
#pragma unroll
        for (int j = 0; j < kRelaxIPT; ++j) {
            const int slot = threadIdx.x + j * kRelaxBlock;
            dv[j] = kInf;
            fv[j] = 0;
            if (slot < n) {
                const int i = sm.sid[slot];
                const long long e = (long long)(k0 + slot) + sm.delta[i];
                if (e >= 0 && (unsigned long long)e < t.src_len) {
                    dv[j] = __ldg(t.dst + e);
                    fv[j] = sm.pay[i];
                } else {
                    atomicOr(la.err, 8u);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kRelaxIPT; ++j) {
            if (dv[j] == kInf) continue;
            const unsigned long long nb = fv[j] & ~__ldcg(&b.vis[dv[j]]);
            if (nb) atomicOr(&b.nxt[dv[j]], nb);
        }
        __syncthreads();
    }
}

// Multi-source SSSP and batched PPR relax.  A warp loads 32 edges at once
// (coalesced), one per lane, each with its source vertex u and the mask of
// sources active at u.  PPR: every lane pushes its own edge, a frame of 8
// seeds per pair of vector reductions (ppr_push_vec).  SSSP: when the masks
// are dense (on average "batch_sparse_below" or more sources per edge) the
// warp walks its edges one at a time with a lane per source (s = lane and
// lane + 32), reading each source's value row in one sector per frame;
// otherwise every lane keeps its own edge and loops over the sources active
// at its u, so that 32 edges' loads are in flight together instead of one
// edge's.
template <int MODE>
__global__ void __launch_bounds__(kRelaxBlock) k_relax_mswarp(BatchState b, ListArrays la,
                                                              const Summary *sum, RelaxTask t,
                                                              unsigned int *bm,
                                                              unsigned int *overflow) {
    __shared__ TileSmem<true> sm;
    if (b.loop && !b.loop->work) return;
    unsigned long long kb, ke;
    task_range(t, sum, kb, ke);
    if (kb >= ke) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long t_first = kb / kTile, t_last = (ke - 1) / kTile;
    for (unsigned long long tile = t_first + blockIdx.x; tile <= t_last; tile += gridDim.x) {
        unsigned long long k0;
        const int n = tile_setup<true>(sm, la, sum, t, tile, kb, ke, &k0);
        if (t.link_ctr) count_link_reads<true>(sm, k0, n, MODE == kBatchSSSP ? 2u : 1u, t.link_ctr);
        const int per_warp = kTile / (kRelaxBlock / 32);           // 256 slots
        for (int c = wid * per_warp; c < (wid + 1) * per_warp && c < n; c += 32) {
            const int slot = c + lane;
            unsigned int dj = kInf, wj = 0, uj = 0;
            unsigned long long fj = 0;
            if (slot < n) {
                const int i = sm.sid[slot];
                const long long e = (long long)(k0 + slot) + sm.delta[i];
                if (e >= 0 && (unsigned long long)e < t.src_len) {
                    dj = __ldg(t.dst + e);
                    if (MODE == kBatchSSSP) wj = __ldg(t.w + e);
                    uj = sm.vid[i];
                    fj = sm.pay[i];
                } else {
                    atomicOr(la.err, 8u);
                }
            }
            if (dj == kInf) fj = 0;
            if (MODE == kBatchPPR) {
                // a lane per edge, a frame's 8 seeds per pair of vector reductions
                const unsigned int m = (unsigned int)fj;
                if (m) {
                    atomicOr(&bm[dj >> 5], 1u << (dj & 31));
                    ppr_push_vec(b, uj, dj, m);
                }
                continue;
            }
            unsigned int pop = __popcll(fj);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pop += __shfl_xor_sync(0xffffffffu, pop, o);
            if (pop < b.sparse_below * 32u) {
                // sparse masks: a lane per edge, looping over its active sources
                if (MODE == kBatchSSSP) {
                    unsigned long long m = fj, imp = 0;
                    while (m) {
                        const unsigned int s = (unsigned int)(__ffsll((long long)m) - 1);
                        m &= m - 1;
                        const unsigned long long nd = (unsigned long long)__ldcg(bval(b, uj, s)) + wj;
                        if (nd >= 0xFFFFFFFEull) {
                            *overflow = 1u;
                        } else if ((unsigned int)nd < __ldcg(bval(b, dj, s))) {
                            atomicMin(bval(b, dj, s), (unsigned int)nd);
                            imp |= 1ull << s;
                        }
                    }
                    if (imp) atomicOr(&b.nxt[dj], imp);
                }
                continue;
            }
            const int cnt = min(32, n - c);
            for (int jj = 0; jj < cnt; ++jj) {
                const unsigned int v = __shfl_sync(0xffffffffu, dj, jj);
                if (v == kInf) continue;                               // warp-uniform
                const unsigned int u = __shfl_sync(0xffffffffu, uj, jj);
                const unsigned long long f = __shfl_sync(0xffffffffu, fj, jj);
                if (MODE == kBatchSSSP) {
                    const unsigned int w = __shfl_sync(0xffffffffu, wj, jj);
                    unsigned long long imp = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const unsigned int s = lane + 32 * h;
                        bool better = false;
                        if ((f >> s) & 1ull) {
                            const unsigned long long nd = (unsigned long long)__ldcg(bval(b, u, s)) + w;
                            if (nd >= 0xFFFFFFFEull) {
                                *overflow = 1u;
                            } else if ((unsigned int)nd < __ldcg(bval(b, v, s))) {
                                atomicMin(bval(b, v, s), (unsigned int)nd);
                                better = true;
                            }
                        }
                        imp |= (unsigned long long)__ballot_sync(0xffffffffu, better) << (32 * h);
                    }
                    if (lane == 0 && imp) atomicOr(&b.nxt[v], imp);
                }
            }
        }
        __syncthreads();
    }
}

// Batched PPR second pass over a resident range [vlo, vhi) whose edges sit in
// `dst` (CSR edge shift at index 0), Sec. VI-A: the seeds whose residual at a
// vertex of the range rose above eps during this iteration are taken again
// and pushed along the still-resident edges.  k_bsp_take: a warp per 32
// consecutive vertices, lanes are seeds; each vertex's taken seeds go to
// sc.pay[v] (a 32-bit mask), the vertex's taken bit to sc.mask, and the
// owners of the 256-edge chunks starting in its list to sc.owner.  The
// residual is read and then subtracted with a reduction, so pushes that land
// meanwhile (other streams' relaxes) stay for later.
__global__ void k_bsp_take(BatchState b, const unsigned long long *off, unsigned long long vlo,
                           unsigned long long vhi, unsigned int K, float damping, float eps,
                           SecondPassScratch sc, unsigned long long *edges_out) {
    if (b.loop && !b.loop->work) return;
    const int lane = threadIdx.x & 31;
    const bool has = lane < (int)K && b.delta[lane >> 3] != nullptr;
    unsigned long long done = 0;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long base = vlo + (((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5) << 5);
         base < vhi; base += nw * 32) {
        unsigned int bits = 0;
        for (int q = 0; q < 32 && base + q < vhi; ++q) {
            const unsigned long long v = base + q;
            const unsigned long long e0 = off[v], deg = off[v + 1] - e0;
            const float dl = has ? __ldcg(bdelta(b, v, lane)) : 0.0f;
            const bool act = has && dl > eps;
            if (act) {
                atomicAdd(bdelta(b, v, lane), -dl);
                *brank(b, v, lane) += dl;
            }
            const unsigned int seeds = __ballot_sync(0xffffffffu, act) & (deg ? 0xffffffffu : 0u);
            // the vector push adds whole frames: the seeds not taken carry 0
            // (this task's relax of v, the only reader of v's old messages,
            // has finished on this stream)
            if (seeds && has) *bmsg(b, v, lane) = act ? damping * dl / (float)deg : 0.0f;
            if (lane == 0) sc.pay[v] = seeds;
            if (seeds) {
                bits |= 1u << q;
                done += (unsigned long long)__popc(seeds) * deg;
            }
            // every chunk that starts in v's list has v as its owner, taken or
            // not: the push starts its owner search there
            if (deg) {
                const unsigned long long c_beg = (e0 + kSpChunk - 1) / kSpChunk, c_end = (e0 + deg - 1) / kSpChunk + 1;
                for (unsigned long long c = c_beg + lane; c < c_end; c += 32) sc.owner[c] = (unsigned int)v;
            }
        }
        if (lane == 0) sc.mask[base >> 5] = bits;
    }
    if (lane == 0 && done) atomicAdd(edges_out, done);
}

// Batched PPR second-pass push: whole 256-edge chunks per warp, the owner of
// each edge found among a window of 32 consecutive vertices; a lane keeps its
// edge and loops over the seeds taken at the edge's source.
__global__ void k_bsp_push(BatchState b, const unsigned long long *off, const unsigned int *dst,
                           long long shift, unsigned long long src_len, unsigned long long vlo,
                           unsigned long long vhi, unsigned long long E0, unsigned long long E1,
                           SecondPassScratch sc, unsigned int *bm, unsigned int *err) {
    if (b.loop && !b.loop->work) return;
    if (E1 <= E0) return;
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long c_first = E0 / kSpChunk, c_last = (E1 - 1) / kSpChunk;
    for (unsigned long long c = c_first + ((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5);
         c <= c_last; c += nwarps) {
        const unsigned long long k0 = c * kSpChunk > E0 ? c * kSpChunk : E0;
        const unsigned long long k1 = (c + 1) * kSpChunk < E1 ? (c + 1) * kSpChunk : E1;
        unsigned long long u0 = c * kSpChunk >= E0 ? (unsigned long long)sc.owner[c] : vlo;
        if (u0 < vlo || u0 >= vhi) {
            if (lane == 0) atomicOr(err, 32u);
            continue;
        }
        unsigned long long kb = k0;
        while (kb < k1) {
            const unsigned long long u = u0 + lane;
            const unsigned long long su = u < vhi ? off[u] : E1;
            const unsigned long long ue = u0 + 32 < vhi ? u0 + 32 : vhi;
            const unsigned long long wend_all = off[ue];
            const bool tk = u < vhi && ((sc.mask[u >> 5] >> (u & 31)) & 1u);
            const unsigned int seeds = tk ? sc.pay[u] : 0u;
            const unsigned int tmask = __ballot_sync(0xffffffffu, tk);
            const unsigned long long wend = wend_all < k1 ? wend_all : k1;
            if (tmask) {
                for (unsigned long long r0 = kb; r0 < wend; r0 += 32) {
                    const unsigned long long k = r0 + lane;
                    int own = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const unsigned long long cand = __shfl_sync(0xffffffffu, su, own + step);
                        if (cand <= k) own += step;
                    }
                    unsigned int m = __shfl_sync(0xffffffffu, seeds, own);
                    if (k >= wend) m = 0;
                    if (m) {
                        const long long i = (long long)k - shift;
                        if (i < 0 || (unsigned long long)i >= src_len) {
                            atomicOr(err, 16u);
                        } else {
                            const unsigned int w = __ldg(dst + i);
                            atomicOr(&bm[w >> 5], 1u << (w & 31));
                            ppr_push_vec(b, u0 + own, w, m);
                        }
                    }
                }
            }
            if (wend <= kb && ue >= vhi) {
                if (lane == 0) atomicOr(err, 32u);
                break;
            }
            if (wend > kb) kb = wend;
            u0 += 32;
        }
    }
}

__global__ void k_b_out(BatchState b, unsigned long long V, unsigned int K, const unsigned int *perm,
                        unsigned int *out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < V * K;
         i += stride) {
        const unsigned long long s = i / V, v = i % V;
        const unsigned long long ov = perm ? perm[v] : v;
        out[s * V + ov] = *bval(b, v, (unsigned int)s);
    }
}

__global__ void k_b_pr_sums(BatchState b, unsigned long long V, unsigned int K, double *sums) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    double acc = 0.0, res = 0.0;
    const bool has = lane < (int)K && b.rank[lane >> 3] != nullptr;
    for (unsigned long long v = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         has && v < V; v += nw) {
        acc += *brank(b, v, lane);
        res += fabs((double)*bdelta(b, v, lane));
    }
    if (has) {
        atomicAdd(&sums[lane], acc);
        atomicAdd(&sums[32 + lane], res);
    }
}

__global__ void k_b_pr_out(BatchState b, unsigned long long V, unsigned int K, const unsigned int *perm,
                           const double *sums, float *out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < V * K;
         i += stride) {
        const unsigned long long s = i / V, v = i % V;
        const unsigned long long ov = perm ? perm[v] : v;
        const double S = sums[s];
        out[s * V + ov] = S > 0.0 ? (float)((double)*brank(b, v, (unsigned int)s) / S) : 0.0f;
    }
}

}  // namespace

cudaError_t launch_b_init(const BatchState &b, unsigned long long V, unsigned long long n_words_alloc,
                          const unsigned int *src_dev, unsigned int K, float base, unsigned int *bm,
                          cudaStream_t s) {
    k_b_init<<<grid_for(V, 256), 256, 0, s>>>(b, V, n_words_alloc, bm);
    if (K) k_b_sources<<<1, 64, 0, s>>>(b, src_dev, K, base, bm);
    return cudaGetLastError();
}

cudaError_t launch_frame_init(const BatchState &b, unsigned long long V, unsigned int g, cudaStream_t s) {
    const bool ok = b.mode == kBatchPPR ? (g < kMaxPprFrames && b.delta[g] && b.rank[g])
                                        : (g < kMaxFrames && b.val[g]);
    if (!ok) return cudaErrorInvalidValue;
    k_frame_init<<<grid_for(V * kFrameSources, 256), 256, 0, s>>>(b, V, g);
    return cudaGetLastError();
}

cudaError_t launch_b_commit(const BatchState &b, unsigned long long V, unsigned long long n_words_alloc,
                            unsigned int level, unsigned int *bm, cudaStream_t s) {
    k_b_commit<<<grid_for(n_words_alloc * 32, 256), 256, 0, s>>>(b, V, n_words_alloc, level, bm);
    return cudaGetLastError();
}

cudaError_t launch_b_take(const BatchState &b, const unsigned long long *off,
                          unsigned long long n_words_alloc, unsigned int K, float damping, float eps,
                          unsigned int *bm, cudaStream_t s) {
    k_b_take<<<grid_for(n_words_alloc * 32, 256), 256, 0, s>>>(b, off, n_words_alloc, K, damping, eps, bm);
    return cudaGetLastError();
}

cudaError_t launch_relax_batched(const BatchState &b, const ListArrays &la, const Summary *sum,
                                 const RelaxTask &t, int grid_cap, unsigned int *bm,
                                 unsigned int *overflow, cudaStream_t s) {
    unsigned int grid = (unsigned int)grid_cap;
    if (!t.device_sized && !t.dev_edge) {
        if (t.k_begin >= t.k_end) return cudaSuccess;
        const unsigned long long tiles = (t.k_end - 1) / kTile - t.k_begin / kTile + 1;
        if (tiles < grid) grid = (unsigned int)tiles;
    }
    if (b.mode == kBatchBFS) k_relax_msbfs<<<grid, kRelaxBlock, 0, s>>>(b, la, sum, t);
    else if (b.mode == kBatchSSSP)
        k_relax_mswarp<kBatchSSSP><<<grid, kRelaxBlock, 0, s>>>(b, la, sum, t, bm, overflow);
    else k_relax_mswarp<kBatchPPR><<<grid, kRelaxBlock, 0, s>>>(b, la, sum, t, bm, overflow);
    return cudaGetLastError();
}

cudaError_t launch_second_pass_batched(const BatchState &b, const unsigned long long *off,
                                       const unsigned int *dst, long long shift,
                                       unsigned long long src_len, unsigned long long vlo,
                                       unsigned long long vhi, unsigned long long E0,
                                       unsigned long long E1, unsigned int K, float damping, float eps,
                                       const SecondPassScratch &sc, unsigned long long *edges_out,
                                       unsigned int *bm, unsigned int *err, cudaStream_t s) {
    if (vhi <= vlo) return cudaSuccess;
    if ((vlo & 31) || b.mode != kBatchPPR) return cudaErrorInvalidValue;
    const unsigned long long cap = 8ull * device_sms();
    unsigned long long tb = (vhi - vlo + 255) / 256;          // 8 warps of 32 vertices per block
    if (tb > cap) tb = cap;
    const unsigned long long chunks = E1 > E0 ? (E1 - 1) / kSpChunk - E0 / kSpChunk + 1 : 0ull;
    unsigned long long pb = (chunks + 7) / 8;
    if (pb > cap) pb = cap;
    if (pb == 0) pb = 1;
    k_bsp_take<<<(unsigned int)tb, 256, 0, s>>>(b, off, vlo, vhi, K, damping, eps, sc, edges_out);
    k_bsp_push<<<(unsigned int)pb, 256, 0, s>>>(b, off, dst, shift, src_len, vlo, vhi, E0, E1, sc, bm, err);
    return cudaGetLastError();
}

cudaError_t launch_serve_admit(const BatchState &b, unsigned long long V, unsigned int slot,
                               unsigned int src, float base, unsigned int *bm, cudaStream_t s) {
    k_serve_clear<<<grid_for(V, 256), 256, 0, s>>>(b, V, slot);
    k_serve_seed<<<1, 1, 0, s>>>(b, slot, src, base, bm);
    return cudaGetLastError();
}

cudaError_t launch_serve_extract(const BatchState &b, unsigned long long V, unsigned int slot,
                                 const unsigned int *perm, unsigned int offset, void *out,
                                 double *sums, cudaStream_t s) {
    if (b.mode == kBatchPPR) {
        cudaError_t e = cudaMemsetAsync(sums, 0, 64 * sizeof(double), s);
        if (e != cudaSuccess) return e;
        k_b_pr_sums<<<grid_for(V * 32, 256), 256, 0, s>>>(b, V, 32, sums);
    }
    k_serve_extract<<<grid_for(V, 256), 256, 0, s>>>(b, V, slot, perm, offset, out, sums);
    return cudaGetLastError();
}

cudaError_t launch_b_finalize(const BatchState &b, unsigned long long V, unsigned int K,
                              const unsigned int *perm, void *out, double *sums, cudaStream_t s) {
    if (b.mode == kBatchPPR) {
        cudaError_t e = cudaMemsetAsync(sums, 0, 64 * sizeof(double), s);
        if (e != cudaSuccess) return e;
        k_b_pr_sums<<<grid_for(V * 32, 256), 256, 0, s>>>(b, V, K, sums);
        k_b_pr_out<<<grid_for(V * K, 256), 256, 0, s>>>(b, V, K, perm, sums, (float *)out);
    } else {
        k_b_out<<<grid_for(V * K, 256), 256, 0, s>>>(b, V, K, perm, (unsigned int *)out);
    }
    return cudaGetLastError();
}

}  // namespace hytg
