// Internal declarations shared by the kernels and the host runtime of the
// hybrid-transfer graph engine.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hytg {

constexpr int kRoutes = 5;            // NONE, CACHE, F, C, Z (hytg_route)
constexpr int kRouteNone = 0, kRouteCache = 1, kRouteF = 2, kRouteC = 3, kRouteZ = 4;

// Frontier bitmap: one bit per vertex, 32-bit words, padded to a multiple of
// 32 words; the planning kernels walk it one 32-word round per warp.  One
// bitmap serves a whole run: k_bin clears the bits it takes, the relax
// kernels set the bits of changed vertices for the next iteration.
constexpr int kBitmapPadWords = 32;

// Edge tiles of the load-balanced relax kernels.
constexpr int kRelaxBlock = 256;
constexpr int kRelaxIPT = 8;
constexpr int kTile = kRelaxBlock * kRelaxIPT;   // 2048 edges per tile

constexpr int kSelectBlock = 512;    // 128 registers per thread: the per-route sums stay in registers

enum Algo : int { kBFS = 0, kSSSP = 1, kCC = 2, kPR = 3, kPPR = 4 };

// Cost-model parameters of one iteration (Sec. V-A).  alpha, beta, gamma are
// rationals num / 1e6 so that the device decision is exact.
struct CostParams {
    unsigned long long alpha_num, beta_num, gamma_num;   // over kParamDen
    unsigned long long m, MR;
    unsigned long long d1;          // bytes read per edge (4 or 8)
    unsigned long long d2;          // bytes per index entry (8)
    unsigned int n_cached;          // partitions [0, n_cached) are resident
    int force_route;                // -1 cost model; 1..4 forced route; 5 random
    unsigned long long seed;        // for force_route 5
    unsigned int iteration;
};
constexpr unsigned long long kParamDen = 1000000ull;

// Device-side summary of one iteration, copied to the host in one piece
// together with the per-partition arrays that follow it in memory.
struct alignas(16) Summary {
    unsigned long long n_active;                 // active vertices (any degree)
    unsigned long long route_entries[kRoutes];   // list entries (active, degree > 0)
    unsigned long long route_edges[kRoutes];     // active edges
    unsigned long long route_lines[kRoutes];     // 128-byte lines (cost-model count)
    unsigned long long route_entry_base[kRoutes];// first index of each route in the list
    unsigned long long route_tile_base[kRoutes]; // first tile of each route
    unsigned int route_parts[kRoutes];
    unsigned int pending_min;                    // bucketed SSSP: smallest pending dist
    unsigned long long pending;                  // bucketed SSSP: active but not yet eligible
    unsigned long long alive;                    // batched: sources with a frontier this iteration
};

// Per-partition arrays, laid out right after the Summary in one buffer.
struct PartArrays {
    unsigned long long *n_act;      // |A_i|
    unsigned long long *entries;    // active vertices with degree > 0
    unsigned long long *edges;      // sum of D_o over A_i
    unsigned long long *lines;      // 128-byte lines spanned (all arrays read)
    unsigned long long *route_entry;// first list index of the partition inside its route
    unsigned long long *route_edge; // first edge index of the partition inside its route
    unsigned long long *cursor;     // fill cursor: entries (low 24 bits) | edges << 24
    unsigned long long *pending;    // bucketed SSSP: pending vertex count
    unsigned long long *pending_inv;// bucketed SSSP: max of ~dist over pending vertices
    unsigned long long *prio;       // delta-first order: sum over A_i of |delta| * 2^24 (PageRank)
    unsigned char *route;           // hytg_route
    const unsigned long long *alive;// batched: source mask of the frontier (or nullptr)
};

// The list of active vertices of one iteration, grouped by route and, inside
// a route, ordered by partition and vertex id.
struct ListArrays {
    unsigned long long *ebase;      // first edge of the entry in its route's edge space
    unsigned long long *soff;       // row offset of the vertex (its first edge in the CSR)
    unsigned int *pay;              // value pushed along its edges (uint32 or float bits)
    unsigned int *tile_first;       // per route tile: list entry (route-relative) holding its first edge
    unsigned long long cap_entries; // capacity of ebase / soff / pay
    unsigned long long cap_tiles;   // capacity of tile_first
    unsigned int *err;              // device word: nonzero if an index check failed
    unsigned long long *pay64;      // batched runs: per-source frontier word of the entry
    unsigned int *vid;              // batched runs: the entry's vertex
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long lines_spanned(unsigned long long start,
                                                            unsigned long long len,
                                                            unsigned long long m) {
    return len == 0 ? 0ull : (start + len - 1) / m - start / m + 1;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// inclusive warp scan
__device__ __forceinline__ unsigned long long warp_scan_u64(unsigned long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Warp sum of values below 2^43 with two 32-bit warp reductions: the low
// 16 bits of 32 lanes sum below 2^21 and the bits above below 2^32, so both
// halves are exact.  (Degrees and line counts are below E, and the
// PageRank priority is capped at 2^40.)  Needs all 32 lanes.
__device__ __forceinline__ unsigned long long warp_sum_lt43(unsigned long long x) {
    const unsigned int lo = __reduce_add_sync(0xffffffffu, (unsigned int)(x & 0xFFFFull));
    const unsigned int hi = __reduce_add_sync(0xffffffffu, (unsigned int)(x >> 16));
    return ((unsigned long long)hi << 16) + lo;
}

// Inclusive warp scan in 32-bit arithmetic when every lane's value is below
// 2^27 (the warp's total then stays below 2^32), else in 64-bit.
__device__ __forceinline__ unsigned long long warp_scan_small(unsigned long long x) {
    if (__all_sync(0xffffffffu, x < (1ull << 27))) {
        const int lane = threadIdx.x & 31;
        unsigned int y = (unsigned int)x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        return y;
    }
    return warp_scan_u64(x);
}

// Counter-based mix used only for the "random route" test mode.
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// ------------------------------------------------------------- launchers
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount),
// read once per device and cached; grid caps are multiples of it.
unsigned int device_sms();

struct GraphDev {
    const unsigned long long *off;      // V+1 row offsets (device)
    unsigned long long V, n_words_alloc;
    const unsigned int *part_wb;        // partition bounds in bitmap words, N+1
    const unsigned long long *part_eb;  // partition bounds in edges, N+1
    const unsigned int *round_part;     // partition holding word 32 * r, per 32-word round
    unsigned int N;
};

// Control block of the device-driven iteration loop (a CUDA graph whose
// WHILE node repeats plan + cache/Z relax until an iteration needs the F or C
// route, the frontier is empty, or the iteration cap is reached).
enum LoopStatus : unsigned int { kLoopRun = 0, kLoopDone = 1, kLoopHost = 2, kLoopMaxIt = 3, kLoopCancel = 4 };
struct LoopCtl {
    unsigned int status;            // LoopStatus when the loop exits
    unsigned int it;                // number of the iteration being planned
    unsigned int bucket;            // SSSP delta-stepping bucket limit (~0u: off)
    unsigned int work;              // 1: this iteration's bin and relax run on the device
    unsigned int n_rec, rec_cap;    // iteration records written / capacity
    unsigned long long delta;       // bucket width (0: no buckets)
    unsigned long long max_it;
    unsigned long long m;           // request bytes (link bytes of zero-copy lines)
    void *rec;                      // hytg_iter_record[rec_cap]
    // F and C iterations inside the loop ("device_loop" 2): the IF-node
    // handle of every partition's F task (nullptr: F iterations go to the
    // host) and of the C route (0: C iterations go to the host)
    const unsigned long long *f_handles;
    unsigned long long c_handle;
    unsigned long long c_cap;       // compaction buffer, in edges (larger C routes go to the host)
    const unsigned char *route;     // per-partition routes of the iteration
    const unsigned long long *part_eb;
    unsigned int n_parts, n_arrays;
    // a word of mapped host memory that the host sets to end the loop at the
    // next iteration boundary (a run past its deadline); nullptr: none
    const volatile unsigned int *cancel;
    // totals over the device iterations of this launch
    unsigned long long route_parts[kRoutes], route_entries[kRoutes], route_edges[kRoutes];
    unsigned long long z_lines, vertices, edges, iterations;
    unsigned long long f_parts, f_bytes, c_iters, c_lines;
};

struct AlgoState {
    int algo;
    unsigned int *val;       // BFS level / SSSP dist / CC label
    float *rank, *delta;     // PageRank state
    float damping, eps;
    unsigned int *bm_cur, *bm_next;
    unsigned int *overflow;  // device flag
    unsigned int n_arrays;   // edge arrays read per edge (1 or 2)
    const unsigned int *perm;// internal id -> original id (hub sorting), or nullptr
    // PageRank pushes to hub ids [0, n_hub_rep) go to per-SM replicas
    // hub_rep[(smid % kHubReplicas) * n_hub_rep + v], summed into delta once per iteration
    float *hub_rep;
    unsigned int n_hub_rep;
    unsigned int bucket_limit;  // SSSP delta-stepping: only dist < limit is eligible (~0u: off)
    LoopCtl *loop;              // device loop: bucket from loop->bucket; bin/relax run if loop->work
    int prio;                   // PageRank/PPR: k_count sums |delta| per partition (delta-first order)
    // batched runs (BatchMode): k_bin takes the per-source frontier word as payload
    int batch_mode;
    const unsigned long long *b_fr;   // BFS/SSSP: 64-bit source mask per vertex
    const unsigned int *b_fr32;       // PPR: 32-bit seed mask per vertex
    unsigned long long *src_work;     // sum over entries of popcount(mask) * degree
};

enum BatchMode : int { kBatchNone = 0, kBatchBFS = 1, kBatchSSSP = 2, kBatchPPR = 3 };

// Per-source state of batched runs and serving lives in frames of
// kFrameSources consecutive sources, so that serving can allocate and release
// it eight queries at a time.  Frame g holds sources [8 g, 8 g + 8): BFS/SSSP
// val[g][v * 8 + (s & 7)] (V * 32 bytes); PPR delta[g], rank[g], msg[g], each
// V * 8 floats (V * 96 bytes in all).  A warp that reads every source of one
// vertex reads one 32-byte sector per frame, as a contiguous vertex-major
// layout would.  Only frames of sources that can be active are read.
constexpr unsigned int kFrameSources = 8;
constexpr unsigned int kMaxFrames = 8;           // 64 BFS/SSSP sources; PPR uses 4 (32 seeds)
constexpr unsigned int kMaxPprFrames = 4;
struct BatchState {
    int mode;
    unsigned long long *fr, *vis, *nxt;   // BFS/SSSP source masks
    unsigned int *val[kMaxFrames];        // BFS level / SSSP distance frames (nullptr: none)
    float *delta[kMaxPprFrames], *rank[kMaxPprFrames], *msg[kMaxPprFrames];   // PPR frames
    unsigned int *fr32;                   // PPR seeds taken at v this iteration
    unsigned long long *alive;            // OR of every vertex's frontier mask (serving)
    const LoopCtl *loop;                  // device loop: level from loop->it; relax gated by loop->work
    unsigned int sparse_below;            // SSSP/PPR relax: a warp whose 32 edges carry fewer than
                                          // this many active sources per edge on average loops
                                          // over sources per lane (0: never)
};
__device__ __forceinline__ unsigned int *bval(const BatchState &b, unsigned long long v, unsigned int s) {
    return b.val[s >> 3] + v * kFrameSources + (s & 7);
}
__device__ __forceinline__ float *bdelta(const BatchState &b, unsigned long long v, unsigned int s) {
    return b.delta[s >> 3] + v * kFrameSources + (s & 7);
}
__device__ __forceinline__ float *brank(const BatchState &b, unsigned long long v, unsigned int s) {
    return b.rank[s >> 3] + v * kFrameSources + (s & 7);
}
__device__ __forceinline__ float *bmsg(const BatchState &b, unsigned long long v, unsigned int s) {
    return b.msg[s >> 3] + v * kFrameSources + (s & 7);
}
// PPR push of u's messages along one edge u -> w for the seeds in `m` (a
// 32-bit mask): per frame holding an active seed, the frame's 8 messages of
// u are read as two float4 and added to w's 8 residuals with two vector
// reductions (red.global.add.v4.f32, one L2 operation for four seeds); a
// half with no active seed is skipped.  The other seeds of a half carry a
// zero message (the take kernels write 0 for every seed they do not take),
// so adding them leaves their residuals unchanged.
__device__ __forceinline__ void ppr_push_vec(const BatchState &b, unsigned long long u, unsigned long long w,
                                             unsigned int m) {
    while (m) {
        const unsigned int g = (unsigned int)(__ffs(m) - 1) >> 3;
        const unsigned int fm = (m >> (8 * g)) & 0xFFu;
        m &= ~(0xFFu << (8 * g));
        const float4 *src = (const float4 *)(b.msg[g] + u * kFrameSources);
        float4 *dst = (float4 *)(b.delta[g] + w * kFrameSources);
        if (fm & 0x0Fu) atomicAdd(dst, __ldcg(src));
        if (fm & 0xF0u) atomicAdd(dst + 1, __ldcg(src + 1));
    }
}
constexpr unsigned int kHubReplicas = 256;

cudaError_t launch_count(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                         unsigned long long m, cudaStream_t s);
cudaError_t launch_select(const GraphDev &g, const PartArrays &pa, const CostParams &cp,
                          Summary *sum, cudaStream_t s);
cudaError_t launch_bin(const GraphDev &g, const AlgoState &st, const PartArrays &pa,
                       const ListArrays &la, const Summary *sum, cudaStream_t s);

// Edge source of a relax / gather launch.
enum EdgeMode : int { kModeHost = 0, kModeDevice = 1, kModeCompact = 2 };

struct RelaxTask {
    int route;                          // which route's list / tiles
    int mode;                           // EdgeMode
    const unsigned int *dst;            // edge destinations (device or mapped host)
    const unsigned int *w;              // weights or nullptr
    long long shift;                    // edge index of dst[0] (device copies)
    unsigned long long k_begin, k_end;  // edge range in the route's edge space
    unsigned long long first_entry;     // route-relative entry holding k_begin
    bool device_sized;                  // take k_end from the summary (k_begin = 0)
    unsigned long long src_len;         // valid indices of dst / w: [0, src_len)
    unsigned long long *link_ctr;       // host-memory reads (Z relax, C gather): {32-byte
                                        // sectors, 128-byte lines} read, or nullptr
    // One partition's F task inside the device loop: its first edge in the F
    // route's edge space, its active edges and its first list entry, read on
    // the device where k_select and k_bin left them (nullptr: host bounds)
    const unsigned long long *dev_edge, *dev_len, *dev_entry;
};

cudaError_t launch_relax(const AlgoState &st, const ListArrays &la, const Summary *sum,
                         const RelaxTask &t, int grid_cap, cudaStream_t s);
// Both tasks device-sized (routes of the current list); plain runs only.
cudaError_t launch_relax_pair(const AlgoState &st, const ListArrays &la, const Summary *sum,
                              const RelaxTask &ta, const RelaxTask &tb, int grid, cudaStream_t s);
// Second pass (Sec. VI-A) over vertices [vlo, vhi) (vlo a multiple of 32)
// whose edges [E0, E1) are resident in dst / w (CSR edge shift at index 0):
// a take launch and an edge-balanced push launch.  Scratch shared by every
// second pass of a run (their vertex and edge ranges never overlap):
constexpr unsigned long long kSpChunk = 256;      // edges per push chunk
struct SecondPassScratch {
    unsigned int *owner;    // per CSR chunk of kSpChunk edges: vertex owning its first edge
    unsigned int *pay;      // per vertex: value it pushes (taken vertices)
    unsigned int *mask;     // per 32 vertices: bit set when taken
};
cudaError_t launch_second_pass(const AlgoState &st, const unsigned long long *off,
                               const unsigned int *dst, const unsigned int *w, long long shift,
                               unsigned long long src_len, unsigned long long vlo,
                               unsigned long long vhi, unsigned long long E0, unsigned long long E1,
                               const SecondPassScratch &sc, unsigned long long *edges_out,
                               unsigned int *err, cudaStream_t s);
// Batched PPR: the second pass (Sec. VI-A) over a resident range, taking
// each seed whose residual rose above eps again (K seeds).
cudaError_t launch_second_pass_batched(const BatchState &b, const unsigned long long *off,
                                       const unsigned int *dst, long long shift,
                                       unsigned long long src_len, unsigned long long vlo,
                                       unsigned long long vhi, unsigned long long E0,
                                       unsigned long long E1, unsigned int K, float damping, float eps,
                                       const SecondPassScratch &sc, unsigned long long *edges_out,
                                       unsigned int *bm, unsigned int *err, cudaStream_t s);
cudaError_t launch_gather(const ListArrays &la, const Summary *sum, const RelaxTask &t,
                          unsigned int *out_dst, unsigned int *out_w, int grid_cap,
                          cudaStream_t s, const LoopCtl *loop = nullptr);

cudaError_t launch_b_init(const BatchState &b, unsigned long long V, unsigned long long n_words_alloc,
                          const unsigned int *src_dev, unsigned int K, float base, unsigned int *bm,
                          cudaStream_t s);
// Fill frame g of the batched state with "no value" (BFS/SSSP: unreached;
// PPR: zero delta and rank), as every frame must hold before it is used.
cudaError_t launch_frame_init(const BatchState &b, unsigned long long V, unsigned int g, cudaStream_t s);
cudaError_t launch_b_commit(const BatchState &b, unsigned long long V, unsigned long long n_words_alloc,
                            unsigned int level, unsigned int *bm, cudaStream_t s);
cudaError_t launch_b_take(const BatchState &b, const unsigned long long *off,
                          unsigned long long n_words_alloc, unsigned int K, float damping, float eps,
                          unsigned int *bm, cudaStream_t s);
cudaError_t launch_relax_batched(const BatchState &b, const ListArrays &la, const Summary *sum,
                                 const RelaxTask &t, int grid_cap, unsigned int *bm,
                                 unsigned int *overflow, cudaStream_t s);
cudaError_t launch_serve_admit(const BatchState &b, unsigned long long V, unsigned int slot,
                               unsigned int src, float base, unsigned int *bm, cudaStream_t s);
cudaError_t launch_serve_extract(const BatchState &b, unsigned long long V, unsigned int slot,
                                 const unsigned int *perm, unsigned int offset, void *out,
                                 double *sums, cudaStream_t s);
cudaError_t launch_b_finalize(const BatchState &b, unsigned long long V, unsigned int K,
                              const unsigned int *perm, void *out, double *sums, cudaStream_t s);

cudaError_t launch_zero_u64(unsigned long long *p, unsigned long long n, cudaStream_t s);
// Copy n 4-byte words from mapped host memory to device memory with 16-byte
// loads (the device loop's F copy where a memcpy node cannot be used);
// gated by loop->work.  Both addresses 16-byte aligned, n a multiple of 4
// except for the tail, which is copied word by word.
cudaError_t launch_copy_words(const unsigned int *src, unsigned int *dst, unsigned long long n,
                              const LoopCtl *loop, cudaStream_t s);
cudaError_t launch_loop_decide(const Summary *sum, LoopCtl *ctl, unsigned long long cond_handle,
                               cudaStream_t s);

cudaError_t launch_init(const AlgoState &st, unsigned long long V, unsigned long long n_words_alloc,
                        unsigned int source, cudaStream_t s);
cudaError_t launch_pr_finalize(const AlgoState &st, unsigned long long V, float *out,
                               double *sums, cudaStream_t s);
cudaError_t launch_pr_frontier(const AlgoState &st, unsigned long long V,
                               unsigned long long n_words_alloc, cudaStream_t s);
cudaError_t launch_hub_reduce(const AlgoState &st, cudaStream_t s);
cudaError_t launch_cc_jump(const AlgoState &st, unsigned long long n_words_alloc, cudaStream_t s);
cudaError_t launch_cc_final(const AlgoState &st, unsigned long long V, unsigned int *tmp,
                            unsigned int *out, cudaStream_t s);
cudaError_t launch_to_original(const unsigned int *perm, const unsigned int *in, float *out,
                               unsigned long long V, cudaStream_t s);
cudaError_t launch_upload_bitmap(const unsigned char *active_dev, unsigned int *bm,
                                 unsigned long long V, unsigned long long n_words_alloc,
                                 cudaStream_t s);
cudaError_t launch_red_probe(unsigned int *idx, float *d, unsigned long long n, int skew, bool gen,
                             cudaStream_t s, float *rep = nullptr, unsigned int n_rep = 0);
cudaError_t launch_frame_probe(const unsigned int *idx, float *d, unsigned long long n, int width,
                               cudaStream_t s);
cudaError_t launch_stage_copy(const unsigned int *src, unsigned int *dst, unsigned long long n,
                              unsigned int blocks_per_sm, cudaStream_t s);
cudaError_t launch_zc_probe(const uint4 *src, unsigned long long n16, unsigned long long *sink,
                            int grid, cudaStream_t s);

}  // namespace hytg
