// Host runtime and C ABI of the hybrid-transfer graph engine.
//
// One hytg_run alternates, until no vertex is active (Sec. IV, overview):
//   1. cost-aware task generation on the device (Sec. V-A): k_count,
//      k_select, then one small device-to-host copy of the per-partition
//      routes and counts (Alg. 1, "copy ... to host");
//   2. k_bin builds the per-route active lists; the cache and zero-copy
//      routes are launched at once with device-side sizes;
//   3. on the host, task combination (Sec. V-B, Alg. 1 combination part):
//      up to k consecutive F partitions become one copy plus one relax; the
//      C partitions are compacted and relaxed in chunks of the compaction
//      buffer;
//   4. multi-stream issue (Sec. VI-B): every F task on its own stream and
//      staging slot (copy engine overlapped with the relax of the previous
//      task), the C route on another stream, cache and Z on the main stream.
// The next iteration's planning kernels wait, on the device, for every
// stream of the previous one, so the host only blocks on the summary copy.
#include <sys/mman.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "hytg.h"

using namespace hytg;

namespace {

constexpr int kMaxStreams = 8;        // F compute streams
constexpr int kMaxSlots = 16;         // staging slots, each with its own copy stream
constexpr uint64_t kPoolSlack = 16384;  // budget pool bytes beyond the budget: alignment padding
constexpr int kKindSecondPass = HYTG_K_SECOND_PASS;   // timed kind beyond the first 12: second_pass_ms
// Second-pass edge counters of one run: slot 0 for the passes inside the
// device-loop graph, slots 1.. for host-issued launches in issue order; the
// last slot is shared by every launch beyond it.
constexpr uint32_t kSpSlots = 16384;

struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
    int stream;                 // 0 main, 1 compaction, 2 + i F stream i
    uint64_t bytes, edges, vertices;
    int sp_slot;                // second pass: its counter slot, else -1
    uint32_t part_first, part_last;
};

// One F task after combination: partitions [i, j], their edges, and the
// pending delta they hold (delta-first order).
struct FTask {
    uint32_t i, j;
    uint64_t edges, prio;
};

// Persistent host worker threads for the host-compaction variant of the C
// route: run(fn) calls fn(t) once for every t in [0, size()), t = 0 on the
// calling thread, and returns when all calls have returned.
class HostPool {
public:
    explicit HostPool(unsigned n) {
        for (unsigned i = 1; i < n; ++i) th_.emplace_back([this, i] { loop(i); });
    }
    ~HostPool() {
        { std::lock_guard<std::mutex> l(mu_); stop_ = true; }
        go_.notify_all();
        for (auto &t : th_) t.join();
    }
    unsigned size() const { return (unsigned)th_.size() + 1; }
    void run(const std::function<void(unsigned)> &fn) {
        {
            std::lock_guard<std::mutex> l(mu_);
            job_ = &fn;
            left_ = (unsigned)th_.size();
            ++gen_;
        }
        go_.notify_all();
        fn(0);
        std::unique_lock<std::mutex> l(mu_);
        done_.wait(l, [&] { return left_ == 0; });
    }

private:
    void loop(unsigned id) {
        uint64_t seen = 0;
        for (;;) {
            const std::function<void(unsigned)> *f;
            {
                std::unique_lock<std::mutex> l(mu_);
                go_.wait(l, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                f = job_;
            }
            (*f)(id);
            std::lock_guard<std::mutex> l(mu_);
            if (--left_ == 0) done_.notify_one();
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable go_, done_;
    const std::function<void(unsigned)> *job_ = nullptr;
    uint64_t gen_ = 0;
    unsigned left_ = 0;
    bool stop_ = false;
};

struct Carve {
    int n_arrays = 0;           // 0: not planned
    uint64_t budget = 0, part_edges = 0;
    uint64_t slot_edges = 0;
    uint32_t n_slots = 0;
    uint64_t compact_edges = 0;
    uint32_t n_cached = 0;
    uint64_t cache_edges = 0;
    uint32_t *cache_dst = nullptr, *cache_w = nullptr;
    uint32_t *slot_dst[kMaxSlots] = {}, *slot_w[kMaxSlots] = {};
    uint32_t *cmp_dst = nullptr, *cmp_w = nullptr;
    uint64_t used = 0;
    uint64_t end = 0;           // bytes of the pool the carve spans (with alignment padding)
};

}  // namespace

struct hytg_ctx {
    int device = 0;
    std::string err;

    cudaStream_t s_main = nullptr, s_c = nullptr;
    cudaStream_t s_f[kMaxStreams] = {};
    cudaStream_t s_cp[kMaxSlots] = {};                   // copy stream of each staging slot
    cudaEvent_t ev_sum[2] = {}, ev_bin = nullptr, ev_f[kMaxStreams] = {}, ev_c = nullptr;
    cudaEvent_t ev_copied[kMaxSlots] = {}, ev_free[kMaxSlots] = {};   // slot filled / slot's last use done
    cudaEvent_t ev_run[2] = {};                          // device time of a run

    // graph
    bool loaded = false;
    int symmetric = -1;                                  // CSR symmetry: -1 not checked yet, 0 no, 1 yes
    uint64_t V = 0, E = 0;
    bool weighted = false;
    uint32_t *h_dst = nullptr, *h_w = nullptr;          // pinned, mapped
    size_t h_map_bytes[2] = {};                          // "host_huge": mmap'd length of h_dst / h_w (0: cudaHostAlloc)
    void *h_map_base[2] = {};
    const uint32_t *m_dst = nullptr, *m_w = nullptr;    // device view of the same memory
    std::vector<uint64_t> h_off;                         // row offsets in internal ids
    // hub sorting (Sec. VI-A): internal id n holds original vertex perm[n]
    bool permuted = false;
    uint64_t n_hubs = 0;
    std::vector<uint32_t> h_perm, h_inv;                 // internal->original, original->internal
    unsigned int *d_perm = nullptr;
    float *d_hub_rep = nullptr;                          // kHubReplicas x n_hub_rep floats
    unsigned int n_hub_rep = 0;

    // batched runs (several sources in one run, sharing every transfer)
    BatchState bs{};
    bool bs_alloc_mask = false, bs_alloc_ppr = false;
    unsigned int *own_val[kMaxFrames] = {};              // hytg_run's BFS/SSSP frames (V * 32 B each)
    float *own_ppr[kMaxPprFrames] = {};                  // hytg_run's PPR frames (V * 96 B each)
    int batch_mode = kBatchNone;
    unsigned int batch_K = 0;
    unsigned int *d_src = nullptr;                       // 64 source ids
    unsigned long long *d_pay64 = nullptr;
    unsigned int *d_vid = nullptr;
    void *d_bout = nullptr;                              // K x V results
    uint32_t bout_rows = 0;                              // rows of V results d_bout holds
    unsigned long long *d_src_work = nullptr;
    double *d_bsums = nullptr;
    unsigned long long *d_alive = nullptr;
    unsigned long long *d_sp = nullptr;                  // second-pass edge counters (kSpSlots)
    unsigned int *d_sp_owner = nullptr;                  // second pass: owner of each kSpChunk-edge chunk
    unsigned int *d_sp_mask = nullptr;                   // second pass: taken bits (one word per 32 vertices)
    uint32_t sp_launches = 0;                            // host-issued second passes this run
    unsigned long long *d_link_ctr = nullptr;            // per route {sectors, lines} read from host memory
    // serving (continuous batching over the batched state)
    bool serving = false;
    int serve_algo = -1;
    uint32_t serve_it = 0;
    uint64_t serve_busy = 0, serve_alive = 0;
    uint32_t serve_admit_it[64] = {};
    // serving's query frames, carved from the budget pool behind the edge-side carve
    char *serve_frame_base = nullptr;
    uint64_t serve_frame_bytes = 0;
    uint32_t serve_frames = 0;                           // frames the budget holds
    uint32_t serve_frames_used = 0;                      // bit f: frame f attached to a group
    int serve_group_frame[kMaxFrames] = {};              // frame of each group of 8 slots, or -1
    uint64_t serve_edge_budget = 0;

    // partitions
    uint64_t part_edges = 0, max_part_edges = 0;
    std::vector<uint64_t> part_vb, part_eb;
    std::vector<uint32_t> part_wb;
    unsigned int *d_part_wb = nullptr;
    unsigned int *d_round_part = nullptr;                // partition of each 32-word bitmap round
    unsigned long long *d_part_eb = nullptr;

    // vertex-side device state
    unsigned long long *d_off = nullptr;
    unsigned int *d_val = nullptr;
    float *d_delta = nullptr;
    unsigned int *d_bm[2] = {};
    unsigned int *d_overflow = nullptr;
    unsigned int *d_err = nullptr;                       // device index-check flags
    uint64_t n_tiles_alloc = 0;
    double *d_prsums = nullptr;
    float *d_out = nullptr;                              // normalised PageRank
    unsigned long long n_words_alloc = 0;
    // lists
    unsigned long long *d_ebase = nullptr, *d_soff = nullptr;
    unsigned int *d_pay = nullptr, *d_tiles = nullptr;
    // summary + per-partition arrays
    void *d_sumbuf = nullptr;
    void *h_sumbuf[2] = {};
    size_t sum_host_bytes = 0, sum_dev_bytes = 0;
    uint64_t vertex_bytes = 0;

    // budget pool
    uint64_t budget = 0;
    void *d_pool = nullptr;
    Carve carve;
    int cache_filled_arrays = 0;
    uint32_t cache_filled_n = 0;

    // parameters
    double alpha = 0.8, beta = 0.4, gamma = 0.625, m = 128, MR = 256, k = 4;
    double part_bytes = 4.0 * 1024 * 1024;
    double streams = 4, staging_frac = 0.5, compact_frac = 0.05;
    double prefetch_slots = 4;                           // staging slots beyond one per F stream
    double force_route = -1, seed = 1, pr_damping = 0.85, pr_eps = 1e-9, max_iters = 1e8;
    double timing = 0;
    double hub_frac = 0.08;                              // Sec. VI-A: top 8 % of vertices
    double hub_replicas = 4096;                          // hub ids with per-SM accumulators
    double sssp_delta = -1;                              // bucket width; -1 auto, 0 off
    double two_pass = 1;                                 // Sec. VI-A second pass: 0, 1 (PageRank), 2 (all)
    double two_pass_min_degree = 4;                      // second pass only for ranges of at least this mean degree
    double run_timeout_ms = 0;                           // hytg_run deadline (0: none)
    double slot_reuse = 0;                               // 1: run F tasks from slots that still hold them
    double f_ahead = 0;                                  // F tasks copied ahead for the next iteration
    double f_copy = 0;                                   // F copies: 0 copy engine, n: copy kernel, n blocks/SM
    double compact_host = 0;                             // C route compacted by this many host threads (0: GPU gather)
    double priority = 1;                                 // Sec. VI-A: F tasks in delta-first order (PageRank/PPR)
    double device_loop = 1;                              // cache/Z-only iterations inside a CUDA graph
    double loop_after_fc = 0;                            // 1: enter the device loop right after an F/C iteration
    double z_blocks = 12;                                // zero-copy relax (host-issued): blocks per SM
    bool last_fc = false;                                // the last host-issued iteration had F or C work
    double host_huge = 0;                                // 1: edge arrays in transparent huge pages, registered
    double serve_frames_param = 0;                       // serving: cap on query frames (0: what the slots need)
    double batch_sparse_below = -1;                      // batched SSSP/PPR relax path switch (sources per
                                                         // edge); -1: 16 for SSSP, always for PPR
    uint64_t auto_delta = 0;                             // auto bucket width from the weights

    // last run
    bool have_result = false;
    int last_algo = -1;
    hytg_stats stats{};
    std::vector<hytg_iter_record> iters;
    std::vector<TimedLaunch> timed;
    std::vector<hytg_timed_launch> timeline;             // the last run's timed launches
    std::vector<FTask> f_tasks_buf;
    std::vector<int> f_hit_buf;                          // per task: staging slot that holds it, or -1
    std::vector<uint32_t> f_order_buf;                   // issue order of the tasks
    // what each staging slot holds for "slot_reuse": partitions [i0, j] with
    // n_arrays arrays (n_arrays 0: nothing known)
    struct SlotHeld { uint32_t i0 = 0, j = 0; int n_arrays = 0; } slot_held[kMaxSlots];
    // copies ahead ("f_ahead"): the slots that the end of one iteration filled
    // with partitions [i0, j] for the next host-issued iteration (work_seq ==
    // ahead_seq), and the position of the slot ring, which then continues
    // across iterations so that copies ahead take the least recently used slots
    struct AheadCopy { uint32_t slot, i0, j; int n_arrays; };
    std::vector<AheadCopy> ahead;
    uint64_t work_seq = 0, ahead_seq = 0;
    uint32_t ring_pos = 0;
    std::vector<std::pair<size_t, cudaEvent_t>> iter_ev; // (iteration index, start mark), timing on
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;

    // host compaction of the C route (ExpTM-C as a CPU gather)
    HostPool *pool = nullptr;
    uint32_t *h_cstage[2] = {};                          // pinned: dst chunk, then w chunk
    uint64_t h_cstage_edges = 0;
    unsigned long long *h_clist = nullptr;               // pinned: soff[cap], then ebase[cap]
    uint64_t h_clist_cap = 0;
    cudaEvent_t ev_cstage[2] = {}, ev_clist = nullptr;

    // device-driven iteration loop: a graph whose WHILE node repeats one
    // iteration (plan, k_loop_decide, bin, cache and Z relax) on the device
    cudaStream_t s_cap = nullptr;                        // capture stream
    cudaStream_t s_cap2 = nullptr;                       // capture stream of the IF-node bodies
    // F and C iterations inside the loop: IF-node handles (host copy, device
    // array), the C route's node, kernels per F / C body, how F copies run
    std::vector<unsigned long long> loop_fh;
    unsigned long long *d_loop_fh = nullptr;
    unsigned long long loop_ch = 0;
    uint32_t loop_f_kernels = 0, loop_c_kernels = 0;
    bool loop_fc = false;                                // the captured body holds F and C nodes
    int last_run_arrays = 1;                             // edge arrays the current run reads
    int loop_fc_copy = 0;                                // 0 memcpy nodes, 1 copy kernel, 2 not available

    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    std::string loop_key;                                // what the captured body depends on
    LoopCtl *d_loop = nullptr, *h_loop = nullptr;        // device control block, pinned mirror
    unsigned int *h_cancel = nullptr, *d_cancel = nullptr;  // mapped word: end the device loop
    bool has_deadline = false;
    std::chrono::steady_clock::time_point run_deadline;
    hytg_iter_record *d_loop_rec = nullptr;
    uint32_t loop_rec_cap = 4096;
    uint32_t loop_kernels = 0;                           // kernels in one body iteration
    bool capturing = false;
    bool loop_unavailable = false;                       // the graph could not be built here
    std::string loop_error;
};

namespace {

const char *kStatusStr[] = {"ok", "invalid argument", "CUDA error", "device budget too small",
                            "pinned host allocation failed", "SSSP distance overflow",
                            "device wait timed out", "call out of order"};

hytg_status fail(hytg_ctx *c, hytg_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess)                                                                \
            return fail(c, HYTG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_loop_graph(hytg_ctx *c) {
    if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
    if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
    c->loop_exec = nullptr;
    c->loop_graph = nullptr;
    c->loop_key.clear();
}

void parallel_chunks(uint64_t n, const std::function<void(uint64_t, uint64_t)> &fn);

hytg_status alloc_edge_array_huge(hytg_ctx *c, int a, uint32_t **out, size_t bytes);

// Pinned, device-mapped host memory for edge array a (0 dst, 1 weights).
// cudaHostAlloc by default.  With "host_huge" = 1 an anonymous mapping
// advised for transparent huge pages, aligned to 512 MiB (the huge-page size
// of a 64 KiB base-page kernel; a 2 MiB one divides it) and registered with
// the driver, falling back to cudaHostAlloc if that fails.  It is not the
// default: in alternating runs it gave the slowest zero-copy and copy
// episodes (a few runs 10-15x slower than the rest), base pages the mildest.
hytg_status alloc_edge_array(hytg_ctx *c, int a, uint32_t **out, size_t bytes) {
    *out = nullptr;
    if (c->host_huge != 0 && alloc_edge_array_huge(c, a, out, bytes) == HYTG_OK) return HYTG_OK;
    if (cudaHostAlloc((void **)out, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return HYTG_ERR_HOSTMEM;
    }
    return HYTG_OK;
}

hytg_status alloc_edge_array_huge(hytg_ctx *c, int a, uint32_t **out, size_t bytes) {
    const size_t align = size_t(512) << 20;
    const size_t len = (bytes + align - 1) / align * align + align;
    void *base = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return HYTG_ERR_HOSTMEM;
    char *p = (char *)(((uintptr_t)base + align - 1) & ~(uintptr_t)(align - 1));
    madvise(p, bytes, MADV_HUGEPAGE);
    // touch every page so that it is faulted in (as a huge page where the
    // kernel can) before the driver pins it
    parallel_chunks(bytes / 4096, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t i = lo; i < hi; ++i) p[i * 4096] = 0;
    });
    if (cudaHostRegister(p, bytes, cudaHostRegisterMapped | cudaHostRegisterPortable) != cudaSuccess) {
        cudaGetLastError();
        munmap(base, len);
        return HYTG_ERR_HOSTMEM;
    }
    c->h_map_base[a] = base;
    c->h_map_bytes[a] = len;
    *out = (uint32_t *)p;
    return HYTG_OK;
}

void free_edge_array(hytg_ctx *c, int a, uint32_t *p) {
    if (!p) return;
    if (c->h_map_bytes[a]) {
        cudaHostUnregister(p);
        munmap(c->h_map_base[a], c->h_map_bytes[a]);
        c->h_map_bytes[a] = 0;
        c->h_map_base[a] = nullptr;
    } else {
        cudaFreeHost(p);
    }
}

void free_graph(hytg_ctx *c) {
    free_loop_graph(c);             // its body holds pointers into the graph's arrays
    free_edge_array(c, 0, c->h_dst);
    free_edge_array(c, 1, c->h_w);
    c->h_dst = c->h_w = nullptr;
    c->m_dst = c->m_w = nullptr;
    dfree(c->d_off); dfree(c->d_val); dfree(c->d_delta); dfree(c->d_bm[0]); dfree(c->d_bm[1]);
    dfree(c->d_out); dfree(c->d_ebase); dfree(c->d_soff); dfree(c->d_pay); dfree(c->d_tiles);
    dfree(c->d_part_wb); dfree(c->d_part_eb); dfree(c->d_sumbuf); dfree(c->d_perm); dfree(c->d_round_part);
    dfree(c->d_hub_rep);
    dfree(c->d_sp_owner);
    dfree(c->d_sp_mask);
    c->n_hub_rep = 0;
    dfree(c->bs.fr); dfree(c->bs.vis); dfree(c->bs.nxt); dfree(c->bs.fr32);
    dfree(c->d_pay64); dfree(c->d_vid); dfree(c->d_bout);
    c->bout_rows = 0;
    for (auto &f : c->own_val) dfree(f);
    for (auto &f : c->own_ppr) dfree(f);
    c->bs = BatchState{};
    c->bs_alloc_mask = c->bs_alloc_ppr = false;
    c->batch_mode = kBatchNone;
    c->permuted = false;
    c->n_hubs = 0;
    c->h_perm.clear();
    c->h_inv.clear();
    for (int i = 0; i < 2; ++i) {
        if (c->h_sumbuf[i]) cudaFreeHost(c->h_sumbuf[i]);
        c->h_sumbuf[i] = nullptr;
    }
    c->loaded = false;
    c->symmetric = -1;
    c->have_result = false;
    c->h_off.clear();
    c->cache_filled_arrays = 0;
    c->cache_filled_n = 0;
    c->carve = Carve();
}

void parallel_chunks(uint64_t n, const std::function<void(uint64_t, uint64_t)> &fn) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < (1u << 20)) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(fn, n * t / nt, n * (t + 1) / nt);
    fn(0, n / nt);
    for (auto &x : th) x.join();
}

// fn(v_lo, v_hi) over vertex ranges holding about equal numbers of edges
// (hub sorting puts most edges in the first few vertices).
void parallel_edge_balanced(const std::vector<uint64_t> &off, uint64_t V,
                            const std::function<void(uint64_t, uint64_t)> &fn) {
    const uint64_t E = off[V];
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (E < (1u << 20)) nt = 1;
    std::vector<uint64_t> vb(nt + 1, V);
    vb[0] = 0;
    for (unsigned t = 1; t < nt; ++t)
        vb[t] = (uint64_t)(std::lower_bound(off.begin(), off.begin() + V + 1, E * t / nt) - off.begin());
    for (unsigned t = 1; t <= nt; ++t) vb[t] = std::max(vb[t], vb[t - 1]);
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(fn, vb[t], vb[t + 1]);
    fn(vb[0], vb[1]);
    for (auto &x : th) x.join();
}

// Whether the loaded CSR is symmetric, as connected components need (the
// weakly connected components of a directed graph are those of its
// symmetrised form, Sec. VII-A runs CC on directed graphs): every edge u->v
// has a reverse v->u with the same multiplicity, a self-loop being its own
// reverse.  In-degrees must equal out-degrees; the reverse rows then have the
// CSR's own offsets, and each row, sorted, must equal the sorted list of the
// vertex's in-neighbours.  O(E) plus the row sorts, on host threads.
bool csr_symmetric(const std::vector<uint64_t> &off, const uint32_t *dst, uint64_t V) {
    const uint64_t E = off[V];
    std::vector<uint64_t> indeg(V, 0);
    parallel_chunks(E, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t e = lo; e < hi; ++e) __atomic_fetch_add(&indeg[dst[e]], 1ull, __ATOMIC_RELAXED);
    });
    std::atomic<bool> ok{true};
    parallel_chunks(V, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t v = lo; v < hi; ++v)
            if (indeg[v] != off[v + 1] - off[v]) { ok = false; return; }
    });
    if (!ok) return false;
    std::vector<uint64_t> cur(off.begin(), off.begin() + V);
    std::vector<uint32_t> rev(std::max<uint64_t>(E, 1));
    parallel_edge_balanced(off, V, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t u = lo; u < hi; ++u)
            for (uint64_t e = off[u]; e < off[u + 1]; ++e)
                rev[__atomic_fetch_add(&cur[dst[e]], 1ull, __ATOMIC_RELAXED)] = (uint32_t)u;
    });
    parallel_edge_balanced(off, V, [&](uint64_t lo, uint64_t hi) {
        std::vector<uint32_t> row;
        for (uint64_t v = lo; v < hi && ok; ++v) {
            const uint64_t b = off[v], n = off[v + 1] - b;
            if (n == 0) continue;
            row.assign(dst + b, dst + b + n);
            std::sort(row.begin(), row.end());
            std::sort(rev.begin() + b, rev.begin() + b + n);
            if (!std::equal(row.begin(), row.end(), rev.begin() + b)) ok = false;
        }
    });
    return ok;
}

// Layout of the summary buffer: the Summary, then the per-partition arrays.
// [n_act, zero_end) is zeroed before every count; [0, host_end) is copied to
// the host once per iteration.
struct SumLayout {
    size_t n_act, entries, edges, lines, cursor, prio, pending, pend_inv, zero_end, route_entry,
        route_edge, route, host_end, total;
};
SumLayout sum_layout(uint32_t N) {
    SumLayout L;
    size_t o = (sizeof(Summary) + 15) & ~size_t(15);
    const size_t a = (size_t)N * 8;
    L.n_act = o; o += a;
    L.entries = o; o += a;
    L.edges = o; o += a;
    L.lines = o; o += a;
    L.cursor = o; o += a;
    L.prio = o; o += a;
    L.pending = o; o += 8;
    L.pend_inv = o; o += 8;
    L.zero_end = o;
    L.route_entry = o; o += a;
    L.route_edge = o; o += a;
    L.route = o; o += ((size_t)N + 15) & ~size_t(15);
    L.host_end = o;
    L.total = o;
    return L;
}

PartArrays part_arrays(hytg_ctx *c) {
    SumLayout L = sum_layout((uint32_t)(c->part_vb.size() - 1));
    char *b = (char *)c->d_sumbuf;
    PartArrays pa;
    pa.n_act = (unsigned long long *)(b + L.n_act);
    pa.entries = (unsigned long long *)(b + L.entries);
    pa.edges = (unsigned long long *)(b + L.edges);
    pa.lines = (unsigned long long *)(b + L.lines);
    pa.route_entry = (unsigned long long *)(b + L.route_entry);
    pa.route_edge = (unsigned long long *)(b + L.route_edge);
    pa.route = (unsigned char *)(b + L.route);
    pa.cursor = (unsigned long long *)(b + L.cursor);
    pa.pending = (unsigned long long *)(b + L.pending);
    pa.pending_inv = (unsigned long long *)(b + L.pend_inv);
    pa.prio = (unsigned long long *)(b + L.prio);
    pa.alive = c->batch_mode != kBatchNone ? c->d_alive : nullptr;
    return pa;
}

// Partition rule (Sec. IV edge-balanced chunk partitioning, read with word-
// aligned bounds): starting at b, the partition ends at the largest multiple
// of 32 vertices e (or V) with off[e] - off[b] <= part_edges; if even the
// first 32 vertices hold more, it is those 32 alone.
void slots_forget(hytg_ctx *c);

void make_partitions(hytg_ctx *c) {
    slots_forget(c);
    const uint64_t V = c->V, pe = c->part_edges;
    const std::vector<uint64_t> &off = c->h_off;
    c->part_vb.assign(1, 0);
    uint64_t b = 0;
    while (b < V) {
        // binary search over aligned ends b + 32 j (and V)
        uint64_t lo = 0, hi = (V - b + 31) / 32;     // j in [1, hi] candidate; find largest ok
        auto end_of = [&](uint64_t j) { return std::min(V, b + 32 * j); };
        while (lo < hi) {
            uint64_t mid = (lo + hi + 1) / 2;
            if (off[end_of(mid)] - off[b] <= pe) lo = mid; else hi = mid - 1;
        }
        uint64_t e = lo == 0 ? end_of(1) : end_of(lo);
        c->part_vb.push_back(e);
        b = e;
    }
    if (V == 0) c->part_vb.push_back(0);
    const size_t N = c->part_vb.size() - 1;
    c->part_eb.resize(N + 1);
    c->part_wb.resize(N + 1);
    c->max_part_edges = 0;
    for (size_t i = 0; i <= N; ++i) {
        c->part_eb[i] = off[c->part_vb[i]];
        c->part_wb[i] = (uint32_t)((c->part_vb[i] + 31) / 32);
        if (i) c->max_part_edges = std::max(c->max_part_edges, c->part_eb[i] - c->part_eb[i - 1]);
    }
}

hytg_status upload_partitions(hytg_ctx *c) {
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    free_loop_graph(c);             // its body holds the arrays freed here
    dfree(c->d_part_wb); dfree(c->d_part_eb); dfree(c->d_sumbuf); dfree(c->d_round_part);
    for (int i = 0; i < 2; ++i) {
        if (c->h_sumbuf[i]) cudaFreeHost(c->h_sumbuf[i]);
        c->h_sumbuf[i] = nullptr;
    }
    CK(cudaMalloc(&c->d_part_wb, (N + 1) * sizeof(unsigned int)));
    CK(cudaMalloc(&c->d_part_eb, (N + 1) * sizeof(unsigned long long)));
    CK(cudaMemcpy(c->d_part_wb, c->part_wb.data(), (N + 1) * sizeof(unsigned int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_part_eb, c->part_eb.data(), (N + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice));
    {
        // round table for the planning kernels' partition lookup
        const uint64_t rounds = std::max<uint64_t>(1, c->n_words_alloc / 32);
        std::vector<uint32_t> rp(rounds);
        uint32_t p = 0;
        for (uint64_t r = 0; r < rounds; ++r) {
            const uint64_t w = r * 32;
            while (p + 1 < N && c->part_wb[p + 1] <= w) ++p;
            rp[r] = p;
        }
        CK(cudaMalloc(&c->d_round_part, rounds * sizeof(uint32_t)));
        CK(cudaMemcpy(c->d_round_part, rp.data(), rounds * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    SumLayout L = sum_layout(N);
    c->sum_dev_bytes = L.total;
    c->sum_host_bytes = L.host_end;
    CK(cudaMalloc(&c->d_sumbuf, L.total));
    CK(cudaMemset(c->d_sumbuf, 0, L.total));
    for (int i = 0; i < 2; ++i) CK(cudaHostAlloc(&c->h_sumbuf[i], L.host_end, cudaHostAllocDefault));
    c->carve = Carve();
    c->cache_filled_arrays = 0;
    return HYTG_OK;
}

// Split the budget (or `edge_budget` bytes of it, when serving keeps the
// rest for query frames) into staging slots (F), the compaction buffer (C)
// and the resident cache (the rest, whole partitions from id 0 upwards).
// The staging slots' contents are no longer known (new partitions, a new
// carve, or copies the host did not track).
void slots_forget(hytg_ctx *c) {
    for (auto &h : c->slot_held) h = hytg_ctx::SlotHeld();
}

hytg_status plan_carve(hytg_ctx *c, int n_arrays, uint64_t edge_budget = 0) {
    const uint64_t B = edge_budget ? edge_budget : c->budget;
    Carve &cv = c->carve;
    const uint64_t pe = c->part_edges;
    Carve n;
    n.n_arrays = n_arrays;
    n.budget = B;
    n.part_edges = pe;
    const uint64_t eb = 4ull * n_arrays;
    const uint64_t min_slot = std::max<uint64_t>(c->max_part_edges, 1);
    const uint64_t compact_min = std::max<uint64_t>(kTile, 1);
    if (B < (min_slot + compact_min) * eb)
        return fail(c, HYTG_ERR_BUDGET, "device budget " + std::to_string(B) +
                                            " B is below one staging slot of the largest partition (" +
                                            std::to_string(min_slot * eb) + " B) plus the minimum compaction buffer (" +
                                            std::to_string(compact_min * eb) + " B)");
    uint64_t stage_cap = std::max<uint64_t>((uint64_t)(B * c->staging_frac), min_slot * eb);
    stage_cap = std::min<uint64_t>(stage_cap, B - compact_min * eb);
    uint64_t slot_edges = std::max<uint64_t>((uint64_t)c->k * pe, min_slot);
    if (slot_edges * eb > stage_cap) slot_edges = std::max<uint64_t>(min_slot, stage_cap / eb);
    uint64_t n_slots = stage_cap / (slot_edges * eb);
    n_slots = std::max<uint64_t>(1, std::min<uint64_t>({n_slots, (uint64_t)(c->streams + c->prefetch_slots),
                                                        (uint64_t)kMaxSlots}));
    uint64_t rem = B - n_slots * slot_edges * eb;
    uint64_t compact_edges = std::max<uint64_t>(compact_min, (uint64_t)(B * c->compact_frac) / eb);
    compact_edges = std::min<uint64_t>(compact_edges, rem / eb);
    compact_edges = compact_edges / kTile * kTile;
    if (compact_edges < (uint64_t)kTile) compact_edges = kTile;
    rem -= compact_edges * eb;
    // cache: largest prefix of whole partitions that fits
    uint32_t n_cached = 0;
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    while (n_cached < N && c->part_eb[n_cached + 1] * eb <= rem) ++n_cached;
    n.slot_edges = slot_edges;
    n.n_slots = (uint32_t)n_slots;
    n.compact_edges = compact_edges;
    n.n_cached = n_cached;
    n.cache_edges = c->part_eb[n_cached];
    // addresses inside the pool (256-byte aligned pieces)
    auto align = [](uint64_t x) { return (x + 255) & ~uint64_t(255); };
    char *base = (char *)c->d_pool;
    uint64_t o = 0;
    n.cache_dst = (uint32_t *)(base + o); o = align(o + n.cache_edges * 4);
    if (n_arrays == 2) { n.cache_w = (uint32_t *)(base + o); o = align(o + n.cache_edges * 4); }
    for (uint32_t s = 0; s < n.n_slots; ++s) {
        n.slot_dst[s] = (uint32_t *)(base + o); o = align(o + slot_edges * 4);
        if (n_arrays == 2) { n.slot_w[s] = (uint32_t *)(base + o); o = align(o + slot_edges * 4); }
    }
    n.cmp_dst = (uint32_t *)(base + o); o = align(o + compact_edges * 4);
    if (n_arrays == 2) { n.cmp_w = (uint32_t *)(base + o); o = align(o + compact_edges * 4); }
    // at most 36 pieces, each padded by < 256 B: the pool holds budget + kPoolSlack
    if (o > B + kPoolSlack)
        return fail(c, HYTG_ERR_BUDGET, "internal: budget carve exceeds the pool");
    n.end = o;
    n.used = n.cache_edges * eb + n.n_slots * slot_edges * eb + compact_edges * eb;
    if (c->cache_filled_arrays != n_arrays || c->carve.cache_dst != n.cache_dst ||
        c->cache_filled_n != n.n_cached)
        c->cache_filled_arrays = 0;   // cache must be refilled
    bool same_slots = cv.n_slots == n.n_slots && cv.slot_edges == n.slot_edges;
    for (uint32_t s = 0; same_slots && s < n.n_slots; ++s)
        same_slots = cv.slot_dst[s] == n.slot_dst[s] && cv.slot_w[s] == n.slot_w[s];
    if (!same_slots) slots_forget(c);
    cv = n;
    return HYTG_OK;
}

cudaEvent_t pool_event(hytg_ctx *c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

int stream_index(const hytg_ctx *c, cudaStream_t s) {
    if (s == c->s_c) return 1;
    for (int i = 0; i < kMaxStreams; ++i)
        if (s == c->s_f[i]) return 2 + i;
    for (int i = 0; i < kMaxSlots; ++i)
        if (s == c->s_cp[i]) return 2 + kMaxStreams + i;
    return 0;
}

// NVTX range names of the launch kinds (index: HYTG_K_*, then the second
// pass), so that a profiler can select a route's launches; without a tool
// attached the NVTX calls do nothing.
const char *const kKindName[] = {"init", "count", "bin", "relax_cache", "relax_F", "gather_C", "relax_C",
                                 "relax_Z", "copy_F", "final", "cache_fill", "other", "second_pass"};

// CUDA-event interval of one launch (timing on); bytes, edges, vertices and
// the second-pass counter slot are filled in by the caller when they apply.
// Every host-issued launch is also an NVTX range named for its kind.
struct ScopedTime {
    hytg_ctx *c;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    uint64_t bytes = 0, edges = 0, vertices = 0;
    int sp_slot = -1;
    uint32_t part_first = 0, part_last = 0;
    bool pushed = false;
    ScopedTime(hytg_ctx *c_, int kind_, cudaStream_t s_, bool kernel = true) : c(c_), kind(kind_), s(s_) {
        const unsigned k = (kernel && kind != HYTG_K_COPY_F && kind != HYTG_K_CACHE_FILL) ? 1 : 0;
        if (c->capturing) {              // inside a graph body: counted per body run
            c->loop_kernels += k;
            return;
        }
        c->stats.kernel_launches += k;
        nvtxRangePushA(kind >= 0 && kind <= kKindSecondPass ? kKindName[kind] : "launch");
        pushed = true;
        if (c->timing != 0) {
            a = pool_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~ScopedTime() {
        if (pushed) nvtxRangePop();
        if (a) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, s);
            c->timed.push_back({kind, a, b, stream_index(c, s), bytes, edges, vertices, sp_slot, part_first,
                                part_last});
        }
    }
};

// A second pass is two launches (take, push); ScopedTime counted the first.
void count_second_launch(hytg_ctx *c) {
    if (c->capturing) c->loop_kernels += 1;
    else c->stats.kernel_launches += 1;
}

// Counter slot of the next host-issued second pass.
unsigned long long *next_sp_slot(hytg_ctx *c, int *slot) {
    const uint32_t k = std::min<uint32_t>(++c->sp_launches, kSpSlots - 1);
    *slot = (int)k;
    return c->d_sp + k;
}

GraphDev graph_dev(hytg_ctx *c) {
    GraphDev g;
    g.off = c->d_off;
    g.V = c->V;
    g.n_words_alloc = c->n_words_alloc;
    g.part_wb = c->d_part_wb;
    g.part_eb = c->d_part_eb;
    g.round_part = c->d_round_part;
    g.N = (unsigned int)(c->part_vb.size() - 1);
    return g;
}

// The second passes' scratch; their push values live in d_out, which holds
// nothing until the run's finalisation writes the result.
SecondPassScratch sp_scratch(hytg_ctx *c) {
    SecondPassScratch sc;
    sc.owner = c->d_sp_owner;
    sc.pay = (unsigned int *)c->d_out;
    sc.mask = c->d_sp_mask;
    return sc;
}

ListArrays list_arrays(hytg_ctx *c) {
    ListArrays l;
    l.ebase = c->d_ebase;
    l.soff = c->d_soff;
    l.pay = c->d_pay;
    l.tile_first = c->d_tiles;
    l.cap_entries = c->V;
    l.cap_tiles = c->n_tiles_alloc;
    l.err = c->d_err;
    l.pay64 = c->d_pay64;
    l.vid = c->d_vid;
    return l;
}

CostParams cost_params(hytg_ctx *c, int algo, uint32_t iteration) {
    CostParams p;
    auto q = [](double x) { return (unsigned long long)std::llround(x * (double)kParamDen); };
    p.alpha_num = q(c->alpha);
    p.beta_num = q(c->beta);
    p.gamma_num = q(c->gamma);
    p.m = (unsigned long long)c->m;
    p.MR = (unsigned long long)c->MR;
    p.d1 = (algo == kSSSP) ? 8 : 4;
    p.d2 = 8;
    p.n_cached = c->carve.n_cached;
    p.force_route = (int)c->force_route;
    p.seed = (unsigned long long)c->seed;
    p.iteration = iteration;
    return p;
}

AlgoState algo_state(hytg_ctx *c, int algo, unsigned int bucket_limit = 0xFFFFFFFFu) {
    AlgoState st;
    st.algo = algo;
    st.val = c->d_val;
    st.rank = (float *)c->d_val;
    st.delta = c->d_delta;
    st.damping = (float)c->pr_damping;
    st.eps = (float)c->pr_eps;
    st.bm_cur = c->d_bm[0];
    st.bm_next = c->d_bm[0];
    st.bucket_limit = bucket_limit;
    st.batch_mode = c->batch_mode;
    st.b_fr = c->bs.fr;
    st.b_fr32 = c->bs.fr32;
    st.src_work = c->d_src_work;
    st.overflow = c->d_overflow;
    st.n_arrays = (algo == kSSSP) ? 2 : 1;
    st.perm = c->d_perm;
    const bool pr = (algo == kPR || algo == kPPR);
    st.hub_rep = pr ? c->d_hub_rep : nullptr;
    st.n_hub_rep = pr && c->d_hub_rep ? c->n_hub_rep : 0;
    st.prio = pr && c->priority != 0 && c->batch_mode == kBatchNone;
    st.loop = nullptr;
    return st;
}

// Initial residual of a PPR seed: (1 - d) V, the total that PageRank starts
// with, so that the FP32 threshold eps bounds the same relative error (with
// 1 - d at the seed alone, eps = 1e-9 left an L1 error near 0.1 on 2^24
// vertices).  Results are normalised, so the scale cancels.
float ppr_seed_mass(const hytg_ctx *c) { return (float)((1.0 - c->pr_damping) * (double)c->V); }

// Copies ahead apply to single-source runs whose F iterations the host
// issues (batched runs and serving keep their F iterations in the graph or
// interleave queries, so a guess from the previous iteration does not hold).
bool ahead_on(const hytg_ctx *c) {
    return c->f_ahead > 0 && c->batch_mode == kBatchNone && !c->serving;
}

// Drop the copies ahead of the last iteration; the main stream (and so all
// later work of the run) waits for those still in flight, since the next
// user of their slots may be a graph node or a run with another carve.
cudaError_t ahead_join(hytg_ctx *c) {
    for (const hytg_ctx::AheadCopy &a : c->ahead) {
        cudaError_t e = cudaStreamWaitEvent(c->s_main, c->ev_copied[a.slot], 0);
        if (e != cudaSuccess) return e;
    }
    c->ahead.clear();
    return cudaSuccess;
}

// At the start of a run or a serving session: copies ahead left by a run
// that ended early (an error) finish before the slots can be carved again.
cudaError_t ahead_drop(hytg_ctx *c) {
    for (const hytg_ctx::AheadCopy &a : c->ahead) {
        cudaError_t e = cudaStreamSynchronize(c->s_cp[a.slot]);
        if (e != cudaSuccess) return e;
    }
    c->ahead.clear();
    c->ring_pos = 0;
    return cudaSuccess;
}

// "two_pass": 0 off, 1 PageRank/PPR only (default), 2 every algorithm; in
// batched runs (and serving) PPR only.
bool second_pass_on(const hytg_ctx *c, int algo) {
    if (c->two_pass == 0) return false;
    if (c->batch_mode != kBatchNone) return c->batch_mode == kBatchPPR;
    return c->two_pass == 2 || algo == kPR || algo == kPPR;
}

// The second pass over a resident range, single-source or batched PPR.
cudaError_t second_pass_any(hytg_ctx *c, const AlgoState &st, const unsigned int *dst, const unsigned int *w,
                            long long shift, unsigned long long src_len, unsigned long long vlo,
                            unsigned long long vhi, unsigned long long E0, unsigned long long E1,
                            unsigned long long *ctr, cudaStream_t s) {
    if (c->batch_mode == kBatchPPR) {
        BatchState b = c->bs;
        b.loop = st.loop;
        return launch_second_pass_batched(b, c->d_off, dst, shift, src_len, vlo, vhi, E0, E1, c->batch_K,
                                          (float)c->pr_damping, (float)c->pr_eps, sp_scratch(c), ctr,
                                          st.bm_cur, c->d_err, s);
    }
    return launch_second_pass(st, c->d_off, dst, w, shift, src_len, vlo, vhi, E0, E1, sp_scratch(c), ctr,
                              c->d_err, s);
}

// An F task's range gets its second pass only if it holds at least
// "two_pass_min_degree" edges per vertex: on ranges of low-degree vertices
// the pass mostly scans vertices (on R-MAT 24, tasks under 2 edges per vertex
// took 29 % of the second-pass time for 5 % of its edges), and the vertices
// it would take stay active for the next iteration instead.
bool range_second_pass(const hytg_ctx *c, uint64_t edges, uint64_t vertices) {
    return (double)edges >= c->two_pass_min_degree * (double)vertices;
}

// The cache range gets its second pass only when every cached partition is
// routed to the cache (always, under the cost model); a forced route could
// send a cached partition to F, whose own second pass would then overlap.
bool cache_second_pass_on(const hytg_ctx *c, int algo) {
    return second_pass_on(c, algo) && (c->force_route == -1 || c->force_route == 1);
}

cudaError_t relax_any(hytg_ctx *c, const AlgoState &st, const ListArrays &la, const Summary *sum,
                      const RelaxTask &t, int cap, cudaStream_t s) {
    if (c->batch_mode != kBatchNone) {
        BatchState b = c->bs;
        b.loop = st.loop;
        return launch_relax_batched(b, la, sum, t, cap, st.bm_cur, st.overflow, s);
    }
    return launch_relax(st, la, sum, t, cap, s);
}

// Device arrays of batched runs and serving that do not grow with the
// number of sources (masks, list payloads, result rows), allocated on first
// use and kept with the graph (vertex-side data, outside the budget).  Every
// frame pointer is cleared; attach_own_frames or the serving calls set them.
hytg_status ensure_batch(hytg_ctx *c, int mode, uint32_t out_rows) {
    const uint64_t V = c->V;
    if (!c->d_pay64) {
        CK(cudaMalloc(&c->d_pay64, V * 8));
        CK(cudaMalloc(&c->d_vid, V * 4));
    }
    if (c->bout_rows < out_rows) {
        dfree(c->d_bout);
        c->bout_rows = 0;
        CK(cudaMalloc(&c->d_bout, V * 4 * out_rows));
        c->bout_rows = out_rows;
    }
    if (mode == kBatchPPR) {
        if (!c->bs_alloc_ppr) {
            CK(cudaMalloc(&c->bs.fr32, V * 4));
            c->bs_alloc_ppr = true;
        }
    } else if (!c->bs_alloc_mask) {
        CK(cudaMalloc(&c->bs.fr, V * 8));
        CK(cudaMalloc(&c->bs.vis, V * 8));
        CK(cudaMalloc(&c->bs.nxt, V * 8));
        c->bs_alloc_mask = true;
    }
    c->bs.mode = mode;
    c->bs.alive = c->d_alive;
    c->bs.sparse_below = c->batch_sparse_below >= 0 ? (unsigned int)c->batch_sparse_below : 16u;
    for (auto &p : c->bs.val) p = nullptr;
    for (uint32_t g = 0; g < kMaxPprFrames; ++g) c->bs.delta[g] = c->bs.rank[g] = c->bs.msg[g] = nullptr;
    return HYTG_OK;
}

// Bytes of one frame of 8 sources: BFS/SSSP values, or PPR delta, rank, msg.
uint64_t frame_bytes(const hytg_ctx *c, int mode) {
    const uint64_t b = c->V * kFrameSources * 4ull * (mode == kBatchPPR ? 3 : 1);
    return (b + 255) & ~uint64_t(255);
}

// Point group g's frame at `mem` (nullptr: the group has no frame).
void set_group_frame(hytg_ctx *c, uint32_t g, char *mem) {
    const uint64_t blk = c->V * kFrameSources * 4ull;
    if (c->bs.mode == kBatchPPR) {
        c->bs.delta[g] = mem ? (float *)mem : nullptr;
        c->bs.rank[g] = mem ? (float *)(mem + blk) : nullptr;
        c->bs.msg[g] = mem ? (float *)(mem + 2 * blk) : nullptr;
    } else {
        c->bs.val[g] = mem ? (unsigned int *)mem : nullptr;
    }
}

// Serving: give group g's frame back once none of its slots holds a query.
void release_idle_frame(hytg_ctx *c, uint32_t g) {
    if (g >= kMaxFrames || c->serve_group_frame[g] < 0) return;
    if ((c->serve_busy >> (g * kFrameSources)) & 0xFFull) return;
    c->serve_frames_used &= ~(1u << c->serve_group_frame[g]);
    c->serve_group_frame[g] = -1;
    set_group_frame(c, g, nullptr);
}

// Frames of a batched hytg_run: one per 8 sources, owned by the context
// (outside the budget, like every batched run's per-source state).
hytg_status attach_own_frames(hytg_ctx *c, int mode, uint32_t K) {
    const uint32_t groups = (K + kFrameSources - 1) / kFrameSources;
    for (uint32_t g = 0; g < groups; ++g) {
        void **own = mode == kBatchPPR ? (void **)&c->own_ppr[g] : (void **)&c->own_val[g];
        if (!*own) CK(cudaMalloc(own, frame_bytes(c, mode)));
        set_group_frame(c, g, (char *)*own);
    }
    return HYTG_OK;
}

hytg_status issue_plan_tail(hytg_ctx *c, int algo, unsigned int bucket, cudaStream_t s, LoopCtl *loop,
                            int part = 0);

// Start mark of the next iteration record (timing on).
void iteration_mark(hytg_ctx *c) {
    if (c->timing == 0) return;
    cudaEvent_t e = pool_event(c);
    if (cudaEventRecord(e, c->s_main) == cudaSuccess) c->iter_ev.push_back({c->iters.size(), e});
}

// Issue planning for one iteration on s_main: counts, selection, summary
// copy (-> ev_sum[buf]) and, with work, binning (-> ev_bin) and the
// device-sized cache and zero-copy relaxes (issue_plan_tail).
hytg_status issue_plan(hytg_ctx *c, int algo, unsigned int bucket, uint32_t it, int buf, bool with_work) {
    if (with_work) iteration_mark(c);
    GraphDev g = graph_dev(c);
    AlgoState st = algo_state(c, algo, bucket);
    PartArrays pa = part_arrays(c);
    Summary *sum = (Summary *)c->d_sumbuf;
    const uint32_t N = g.N;
    if ((algo == kPR || algo == kPPR) && it > 0 && c->batch_mode == kBatchNone) {
        ScopedTime t(c, HYTG_K_OTHER, c->s_main);
        CK(launch_hub_reduce(st, c->s_main));
        CK(launch_pr_frontier(st, c->V, c->n_words_alloc, c->s_main));
    }
    if (algo == kCC && it > 0 && with_work) {
        ScopedTime t(c, HYTG_K_OTHER, c->s_main);
        CK(launch_cc_jump(st, c->n_words_alloc, c->s_main));
    }
    if (c->batch_mode != kBatchNone && with_work) CK(cudaMemsetAsync(c->d_alive, 0, 8, c->s_main));
    if (c->batch_mode == kBatchPPR && with_work) {
        ScopedTime t(c, HYTG_K_OTHER, c->s_main);
        CK(launch_b_take(c->bs, c->d_off, c->n_words_alloc, c->batch_K, (float)c->pr_damping,
                         (float)c->pr_eps, st.bm_cur, c->s_main));
    } else if (c->batch_mode != kBatchNone && (it > 0 || c->serving) && with_work) {
        ScopedTime t(c, HYTG_K_OTHER, c->s_main);
        CK(launch_b_commit(c->bs, c->V, c->n_words_alloc, it, st.bm_cur, c->s_main));
    }
    {
        const SumLayout L = sum_layout(N);
        CK(cudaMemsetAsync(pa.n_act, 0, L.zero_end - L.n_act, c->s_main));
    }
    { ScopedTime t(c, HYTG_K_COUNT, c->s_main); CK(launch_count(g, st, pa, (unsigned long long)c->m, c->s_main)); }
    { ScopedTime t(c, HYTG_K_COUNT, c->s_main); CK(launch_select(g, pa, cost_params(c, algo, it), sum, c->s_main)); }
    CK(cudaMemcpyAsync(c->h_sumbuf[buf], c->d_sumbuf, c->sum_host_bytes, cudaMemcpyDeviceToHost, c->s_main));
    CK(cudaEventRecord(c->ev_sum[buf], c->s_main));
    if (!with_work) return HYTG_OK;
    return issue_plan_tail(c, algo, bucket, c->s_main, nullptr);
}

// The device-sized part of an iteration once its routes are decided: k_bin,
// then the cache relax (and its second pass) and the zero-copy relax.
// `loop` is set when the launches are captured into the device loop's body:
// they then run only if k_loop_decide gave the iteration to the device.
// part: 0 everything; while capturing the device loop's body, 1 stops after
// k_bin and 2 issues only what follows it.
hytg_status issue_plan_tail(hytg_ctx *c, int algo, unsigned int bucket, cudaStream_t s, LoopCtl *loop,
                            int part) {
    GraphDev g = graph_dev(c);
    AlgoState st = algo_state(c, algo, bucket);
    st.loop = loop;
    PartArrays pa = part_arrays(c);
    ListArrays la = list_arrays(c);
    Summary *sum = (Summary *)c->d_sumbuf;
    if (part != 2) {
        { ScopedTime t(c, HYTG_K_BIN, s); CK(launch_bin(g, st, pa, la, sum, s)); }
        if (!c->capturing) CK(cudaEventRecord(c->ev_bin, s));
    }
    if (part == 1) return HYTG_OK;
    const int cap = 4 * (int)device_sms();
    if (c->capturing && c->batch_mode == kBatchNone && c->carve.n_cached > 0) {
        // device loop body: cache and zero-copy routes in one launch
        RelaxTask tc{}, tz{};
        tc.route = kRouteCache; tc.mode = kModeDevice; tc.dst = c->carve.cache_dst; tc.w = c->carve.cache_w;
        tc.shift = 0; tc.device_sized = true; tc.src_len = c->carve.cache_edges;
        tz.route = kRouteZ; tz.mode = kModeHost; tz.dst = c->m_dst; tz.w = c->m_w; tz.shift = 0;
        tz.device_sized = true; tz.src_len = c->E; tz.link_ctr = c->d_link_ctr + 2 * kRouteZ;
        {
            ScopedTime tm(c, HYTG_K_RELAX_Z, s);
            CK(launch_relax_pair(st, la, sum, tc, tz, cap, s));
        }
        if (cache_second_pass_on(c, algo)) {
            ScopedTime tm(c, kKindSecondPass, s);
            CK(second_pass_any(c, st, c->carve.cache_dst, c->carve.cache_w, 0, c->carve.cache_edges, 0,
                               c->part_vb[c->carve.n_cached], 0, c->part_eb[c->carve.n_cached], c->d_sp, s));
            count_second_launch(c);
        }
        return HYTG_OK;
    }
    if (c->carve.n_cached > 0) {
        RelaxTask t{};
        t.route = kRouteCache; t.mode = kModeDevice; t.dst = c->carve.cache_dst; t.w = c->carve.cache_w;
        t.shift = 0; t.device_sized = true; t.src_len = c->carve.cache_edges;
        {
            ScopedTime tm(c, HYTG_K_RELAX_CACHE, s);
            CK(relax_any(c, st, la, sum, t, cap, s));
        }
        if (cache_second_pass_on(c, algo)) {
            ScopedTime tm(c, kKindSecondPass, s);
            unsigned long long *ctr = next_sp_slot(c, &tm.sp_slot);
            tm.vertices = c->part_vb[c->carve.n_cached];
            CK(second_pass_any(c, st, c->carve.cache_dst, c->carve.cache_w, 0, c->carve.cache_edges, 0,
                               c->part_vb[c->carve.n_cached], 0, c->part_eb[c->carve.n_cached], ctr, s));
            count_second_launch(c);
            c->stats.second_pass_vertices += c->part_vb[c->carve.n_cached];
        }
    }
    {
        RelaxTask t{};
        t.route = kRouteZ; t.mode = kModeHost; t.dst = c->m_dst; t.w = c->m_w; t.shift = 0;
        t.device_sized = true; t.src_len = c->E; t.link_ctr = c->d_link_ctr + 2 * kRouteZ;
        ScopedTime tm(c, HYTG_K_RELAX_Z, s);
        CK(relax_any(c, st, la, sum, t, (int)c->z_blocks * (int)device_sms(), s));
    }
    return HYTG_OK;
}

// Device loop (plain runs): whether it applies, and its graph.  The body is
// captured once per configuration and replayed by one graph launch per
// stretch of device iterations.
bool loop_applies(const hytg_ctx *c) {
    return c->device_loop != 0 && c->force_route != 5 && !c->serving;
}

// F and C iterations can stay in the device loop: batched runs at "device_loop"
// 1, every run at 2; not with host compaction, forced random routes, more
// partitions than 1024 IF nodes, or a staging slot without room for one
// partition (plus 3 words of alignment slack when the copy kernel, not a
// memcpy node, moves it).
bool loop_fc_wanted(const hytg_ctx *c) {
    if (c->device_loop < 2 && c->batch_mode == kBatchNone) return false;
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    const uint64_t slack = c->loop_fc_copy == 1 ? 3 : 0;
    return c->compact_host == 0 && c->force_route != 5 && N >= 1 && N <= 1024 && c->carve.n_slots >= 1 &&
           c->carve.slot_edges >= c->max_part_edges + slack;
}

// One IF node per partition (copy the partition into the staging slot of its
// lane, relax it, and for PageRank/PPR its second pass), chained per slot so
// that a slot's next user starts after the previous one; one IF node for the
// C route (gather into the compaction buffer, relax).  k_loop_decide opens the
// nodes of the partitions it routed F and the C node when C fits the buffer.
hytg_status capture_loop_fc(hytg_ctx *c, int algo, cudaGraph_t cg, const std::vector<cudaGraphNode_t> &after_bin) {
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    Carve &cv = c->carve;
    const int n_arrays = (algo == kSSSP) ? 2 : 1;
    AlgoState st = algo_state(c, algo);
    st.loop = c->d_loop;
    PartArrays pa = part_arrays(c);
    ListArrays la = list_arrays(c);
    Summary *sum = (Summary *)c->d_sumbuf;
    const int cap = 8 * (int)device_sms();
    if (!c->d_loop_fh) return fail(c, HYTG_ERR_CUDA, "device loop: no handle array");
    c->loop_fh.assign(N, 0);
    const uint32_t S = cv.n_slots;
    std::vector<cudaGraphNode_t> lane(S, nullptr);
    auto add_if = [&](const std::vector<cudaGraphNode_t> &d, cudaGraphConditionalHandle *h, cudaGraphNode_t *node,
                      cudaGraph_t *body) -> cudaError_t {
        cudaError_t e = cudaGraphConditionalHandleCreate(h, cg, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return e;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = *h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        e = cudaGraphAddNode(node, cg, d.data(), nullptr, d.size(), &np);
        if (e == cudaSuccess) *body = np.conditional.phGraph_out[0];
        return e;
    };
    const uint32_t k_before = c->loop_kernels;
    c->loop_f_kernels = 0;
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t k_node = c->loop_kernels;
        const uint32_t L = i % S;
        std::vector<cudaGraphNode_t> d = lane[L] ? std::vector<cudaGraphNode_t>{lane[L]} : after_bin;
        cudaGraphConditionalHandle h;
        cudaGraphNode_t node;
        cudaGraph_t body;
        CK(add_if(d, &h, &node, &body));
        c->loop_fh[i] = (unsigned long long)h;
        lane[L] = node;
        const uint64_t eb = c->part_eb[i], ee = c->part_eb[i + 1];
        // the copy kernel reads from the 16-byte boundary at or below the
        // partition's first edge; a memcpy node copies the partition exactly
        const uint64_t e0 = c->loop_fc_copy == 1 ? (eb & ~uint64_t(3)) : eb;
        CK(cudaStreamBeginCaptureToGraph(c->s_cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        hytg_status r = HYTG_OK;
        cudaError_t e = cudaSuccess;
        if (ee > eb) {
            if (c->loop_fc_copy == 0) {
                e = cudaMemcpyAsync(cv.slot_dst[L], c->h_dst + eb, (ee - eb) * 4, cudaMemcpyHostToDevice, c->s_cap2);
                if (e == cudaSuccess && n_arrays == 2)
                    e = cudaMemcpyAsync(cv.slot_w[L], c->h_w + eb, (ee - eb) * 4, cudaMemcpyHostToDevice, c->s_cap2);
            } else {
                e = launch_copy_words(c->m_dst + e0, cv.slot_dst[L], ee - e0, c->d_loop, c->s_cap2);
                if (e == cudaSuccess && n_arrays == 2)
                    e = launch_copy_words(c->m_w + e0, cv.slot_w[L], ee - e0, c->d_loop, c->s_cap2);
                c->loop_kernels += n_arrays;
            }
            RelaxTask t{};
            t.route = kRouteF; t.mode = kModeDevice; t.dst = cv.slot_dst[L]; t.w = cv.slot_w[L];
            t.shift = (long long)e0; t.src_len = ee - e0;
            t.dev_edge = pa.route_edge + i; t.dev_len = pa.edges + i; t.dev_entry = pa.route_entry + i;
            if (e == cudaSuccess) {
                ScopedTime tm(c, HYTG_K_RELAX_F, c->s_cap2);
                e = relax_any(c, st, la, sum, t, cap, c->s_cap2);
            }
            if (e == cudaSuccess && second_pass_on(c, algo) &&
                range_second_pass(c, ee - eb, c->part_vb[i + 1] - c->part_vb[i])) {
                ScopedTime tm(c, kKindSecondPass, c->s_cap2);
                e = second_pass_any(c, st, cv.slot_dst[L], cv.slot_w[L], (long long)e0, ee - e0, c->part_vb[i],
                                    c->part_vb[i + 1], eb, ee, c->d_sp, c->s_cap2);
                count_second_launch(c);
            }
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(c->s_cap2, &captured);
        if (e != cudaSuccess) r = fail(c, HYTG_ERR_CUDA, std::string("F node of the device loop: ") + cudaGetErrorString(e));
        else if (e_end != cudaSuccess)
            r = fail(c, HYTG_ERR_CUDA, std::string("F node capture: ") + cudaGetErrorString(e_end));
        if (r != HYTG_OK) return r;
        if (c->loop_kernels > k_node && c->loop_f_kernels == 0) c->loop_f_kernels = c->loop_kernels - k_node;
    }
    c->loop_kernels = k_before;              // F-node kernels are counted per opened node
    {
        // the C route in one chunk of the compaction buffer
        cudaGraphConditionalHandle h;
        cudaGraphNode_t node;
        cudaGraph_t body;
        CK(add_if(after_bin, &h, &node, &body));
        c->loop_ch = (unsigned long long)h;
        CK(cudaStreamBeginCaptureToGraph(c->s_cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        RelaxTask gt{};
        gt.route = kRouteC; gt.mode = kModeHost; gt.dst = c->m_dst; gt.w = c->m_w; gt.shift = 0;
        gt.device_sized = true; gt.src_len = c->E; gt.link_ctr = c->d_link_ctr + 2 * kRouteC;
        cudaError_t e = launch_gather(la, sum, gt, cv.cmp_dst, n_arrays == 2 ? cv.cmp_w : nullptr, cap, c->s_cap2,
                                      c->d_loop);
        RelaxTask rt{};
        rt.route = kRouteC; rt.mode = kModeCompact; rt.dst = cv.cmp_dst; rt.w = cv.cmp_w; rt.shift = 0;
        rt.device_sized = true; rt.src_len = cv.compact_edges;
        if (e == cudaSuccess) e = relax_any(c, st, la, sum, rt, cap, c->s_cap2);
        cudaGraph_t captured = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(c->s_cap2, &captured);
        if (e != cudaSuccess || e_end != cudaSuccess)
            return fail(c, HYTG_ERR_CUDA, std::string("C node of the device loop: ") +
                                              cudaGetErrorString(e != cudaSuccess ? e : e_end));
        c->loop_c_kernels = 2;
    }
    return HYTG_OK;
}

hytg_status capture_loop_body(hytg_ctx *c, int algo, cudaStream_t s, unsigned long long handle) {
    GraphDev g = graph_dev(c);
    AlgoState st = algo_state(c, algo);
    st.loop = c->d_loop;
    PartArrays pa = part_arrays(c);
    Summary *sum = (Summary *)c->d_sumbuf;
    if (c->batch_mode != kBatchNone) {
        // per-iteration source bookkeeping, as the host loop does it
        BatchState b = c->bs;
        b.loop = c->d_loop;
        ScopedTime t(c, HYTG_K_OTHER, s);
        CK(launch_zero_u64(c->d_alive, 1, s));
        if (c->batch_mode == kBatchPPR)
            CK(launch_b_take(b, c->d_off, c->n_words_alloc, c->batch_K, (float)c->pr_damping,
                             (float)c->pr_eps, st.bm_cur, s));
        else
            CK(launch_b_commit(b, c->V, c->n_words_alloc, 0, st.bm_cur, s));
    } else if (algo == kPR || algo == kPPR) {
        ScopedTime t(c, HYTG_K_OTHER, s);
        CK(launch_hub_reduce(st, s));
        CK(launch_pr_frontier(st, c->V, c->n_words_alloc, s));
    } else if (algo == kCC) {
        ScopedTime t(c, HYTG_K_OTHER, s);
        CK(launch_cc_jump(st, c->n_words_alloc, s));
    }
    {
        const SumLayout L = sum_layout(g.N);
        ScopedTime t(c, HYTG_K_OTHER, s);
        CK(launch_zero_u64(pa.n_act, (L.zero_end - L.n_act) / 8, s));
    }
    { ScopedTime t(c, HYTG_K_COUNT, s); CK(launch_count(g, st, pa, (unsigned long long)c->m, s)); }
    { ScopedTime t(c, HYTG_K_COUNT, s); CK(launch_select(g, pa, cost_params(c, algo, 1), sum, s)); }
    { ScopedTime t(c, HYTG_K_OTHER, s); CK(launch_loop_decide(sum, c->d_loop, handle, s)); }
    return issue_plan_tail(c, algo, 0xFFFFFFFFu, s, c->d_loop, 1);
}

hytg_status ensure_loop_graph(hytg_ctx *c, int algo) {
    char key[512];
    std::snprintf(key, sizeof key, "%d|%d|%u|%p|%u|%llu|%d|%p|%u|%p|%p|%p|%g|%g|%g|%g|%g|%g|%g|%g|%g|%llu|%zu|%g|%g|%p",
                  algo, c->batch_mode, c->batch_K, (void *)c->carve.cache_dst, c->carve.n_cached,
                  (unsigned long long)c->carve.cache_edges, (int)second_pass_on(c, algo), (void *)c->d_hub_rep,
                  c->n_hub_rep, (void *)c->d_sumbuf, (void *)c->d_val, (void *)c->d_ebase, c->alpha, c->beta,
                  c->gamma, c->m, c->MR, c->force_route, c->pr_damping, c->pr_eps, c->priority,
                  (unsigned long long)c->n_words_alloc, c->part_vb.size(), c->hub_frac, c->batch_sparse_below,
                  (void *)c->bs.val[0]);
    {
        const size_t n = std::strlen(key);
        std::snprintf(key + n, sizeof key - n, "|fc%d.%d|%u|%p|%p|%llu", (int)c->loop_fc, c->loop_fc_copy,
                      c->carve.n_slots, (void *)c->carve.slot_dst[0], (void *)c->carve.cmp_dst,
                      (unsigned long long)c->carve.compact_edges);
    }
    if (c->loop_exec && c->loop_key == key) return HYTG_OK;
    free_loop_graph(c);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    c->loop_graph = g;
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // The body is captured in two pieces that meet at k_bin: planning up to
    // k_bin, then (from k_bin's node) the cache and zero-copy relaxes; the F
    // and C IF nodes are added to the finished body, also after k_bin, and
    // each IF node's own body is captured on the second capture stream.
    c->loop_kernels = 0;
    std::vector<cudaGraphNode_t> after_bin;
    for (int piece = 0; piece < 2; ++piece) {
        CK(cudaStreamBeginCaptureToGraph(c->s_cap, body, after_bin.empty() ? nullptr : after_bin.data(), nullptr,
                                         after_bin.size(), cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        hytg_status st = piece == 0 ? capture_loop_body(c, algo, c->s_cap, (unsigned long long)h)
                                    : issue_plan_tail(c, algo, 0xFFFFFFFFu, c->s_cap, c->d_loop, 2);
        if (st == HYTG_OK && piece == 0) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            if (cudaStreamGetCaptureInfo(c->s_cap, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess || nd == 0)
                st = fail(c, HYTG_ERR_CUDA, "device loop: no node after k_bin");
            else
                after_bin.assign(deps, deps + nd);
        }
        c->capturing = false;
        cudaGraph_t captured = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(c->s_cap, &captured);
        if (st != HYTG_OK) { free_loop_graph(c); return st; }
        if (e_end != cudaSuccess) {
            free_loop_graph(c);
            return fail(c, HYTG_ERR_CUDA, std::string("capture of the device loop: ") + cudaGetErrorString(e_end));
        }
    }
    if (c->loop_fc) {
        c->capturing = true;
        hytg_status st = capture_loop_fc(c, algo, body, after_bin);
        c->capturing = false;
        if (st != HYTG_OK) { free_loop_graph(c); return st; }
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e_in = cudaGraphInstantiate(&ex, g, 0);
    if (e_in != cudaSuccess) {
        free_loop_graph(c);
        return fail(c, HYTG_ERR_CUDA, std::string("instantiating the device loop: ") + cudaGetErrorString(e_in));
    }
    if (c->loop_fc && !c->loop_fh.empty())
        CK(cudaMemcpy(c->d_loop_fh, c->loop_fh.data(), c->loop_fh.size() * 8, cudaMemcpyHostToDevice));
    c->loop_exec = ex;
    c->loop_key = key;
    return HYTG_OK;
}

// The device loop with its F and C nodes when the run allows them: first
// with memcpy nodes for the F copies, then with a copy kernel, and if the
// installed driver accepts neither, without F and C nodes (such iterations
// then go to the host, as with "device_loop" 1).
hytg_status ensure_loop_graph_fc(hytg_ctx *c, int algo) {
    if (!loop_fc_wanted(c) || c->loop_fc_copy >= 2) {
        c->loop_fc = false;
        return ensure_loop_graph(c, algo);
    }
    for (;;) {
        c->loop_fc = true;
        hytg_status s = ensure_loop_graph(c, algo);
        if (s == HYTG_OK) return s;
        cudaGetLastError();
        c->loop_fc = false;
        if (++c->loop_fc_copy >= 2) return ensure_loop_graph(c, algo);
    }
}


hytg_status ensure_cache(hytg_ctx *c, int n_arrays) {
    Carve &cv = c->carve;
    if (c->cache_filled_arrays == n_arrays && c->cache_filled_n == cv.n_cached) return HYTG_OK;
    if (cv.cache_edges) {
        ScopedTime t(c, HYTG_K_CACHE_FILL, c->s_main);
        CK(cudaMemcpyAsync(cv.cache_dst, c->h_dst, cv.cache_edges * 4, cudaMemcpyHostToDevice, c->s_main));
        if (n_arrays == 2)
            CK(cudaMemcpyAsync(cv.cache_w, c->h_w, cv.cache_edges * 4, cudaMemcpyHostToDevice, c->s_main));
        c->stats.cache_fill_bytes += cv.cache_edges * 4 * n_arrays;
    }
    c->cache_filled_arrays = n_arrays;
    c->cache_filled_n = cv.n_cached;
    return HYTG_OK;
}

// The C route with the compaction done by host threads (the CPU-compaction
// form of ExpTM-C, Sec. III-B / Sec. V): the route's active list (row offset
// and route edge base per entry) comes back to the host, the worker threads
// copy each entry's edges from the pinned CSR into a pinned staging chunk at
// its route position, one explicit copy moves the chunk into the compaction
// buffer and the compact-mode relax runs on it.  Two staging chunks let the
// threads fill one while the other is copied and relaxed.
hytg_status host_compact(hytg_ctx *c, int algo, unsigned int bucket, const Summary *hs, int n_arrays) {
    Carve &cv = c->carve;
    const uint64_t nC = hs->route_entries[kRouteC];
    const uint64_t base = hs->route_entry_base[kRouteC];
    const uint64_t c_edges = hs->route_edges[kRouteC];
    const unsigned nt = (unsigned)c->compact_host;
    if (!c->pool || c->pool->size() != nt) {
        delete c->pool;
        c->pool = nullptr;
        c->pool = new HostPool(nt);
    }
    if (c->h_cstage_edges != cv.compact_edges) {
        for (int b = 0; b < 2; ++b) {
            if (c->h_cstage[b]) CK(cudaFreeHost(c->h_cstage[b]));
            c->h_cstage[b] = nullptr;
        }
        c->h_cstage_edges = 0;
        for (int b = 0; b < 2; ++b)
            if (cudaHostAlloc((void **)&c->h_cstage[b], cv.compact_edges * 8, cudaHostAllocDefault) != cudaSuccess)
                return fail(c, HYTG_ERR_HOSTMEM, "pinned staging for host compaction");
        c->h_cstage_edges = cv.compact_edges;
    }
    if (c->h_clist_cap < nC) {
        if (c->h_clist) CK(cudaFreeHost(c->h_clist));
        c->h_clist = nullptr;
        c->h_clist_cap = 0;
        uint64_t cap = 1024;
        while (cap < nC) cap *= 2;
        if (cudaHostAlloc((void **)&c->h_clist, cap * 16, cudaHostAllocDefault) != cudaSuccess)
            return fail(c, HYTG_ERR_HOSTMEM, "pinned list buffer for host compaction");
        c->h_clist_cap = cap;
    }
    unsigned long long *h_soff = c->h_clist, *h_ebase = c->h_clist + c->h_clist_cap;
    CK(cudaStreamWaitEvent(c->s_c, c->ev_bin, 0));
    CK(cudaMemcpyAsync(h_soff, c->d_soff + base, nC * 8, cudaMemcpyDeviceToHost, c->s_c));
    CK(cudaMemcpyAsync(h_ebase, c->d_ebase + base, nC * 8, cudaMemcpyDeviceToHost, c->s_c));
    CK(cudaEventRecord(c->ev_clist, c->s_c));
    CK(cudaEventSynchronize(c->ev_clist));
    const auto t0 = std::chrono::steady_clock::now();
    AlgoState st = algo_state(c, algo, bucket);
    ListArrays la = list_arrays(c);
    Summary *dsum = (Summary *)c->d_sumbuf;
    const uint32_t *hd = c->h_dst, *hw = c->h_w;
    const uint64_t E = c->E;
    std::atomic<int> bad{0};
    int chunk = 0;
    for (uint64_t cb = 0; cb < c_edges; cb += cv.compact_edges, ++chunk) {
        const uint64_t ce = std::min<uint64_t>(c_edges, cb + cv.compact_edges);
        const int b = chunk & 1;
        if (chunk >= 2) CK(cudaEventSynchronize(c->ev_cstage[b]));   // its copy two chunks ago
        uint32_t *sd = c->h_cstage[b], *sw = c->h_cstage[b] + cv.compact_edges;
        const std::function<void(unsigned)> job = [&](unsigned t) {
            // route edges [a, z) of this chunk, split evenly across the threads
            const uint64_t a = cb + (ce - cb) * t / nt, z = cb + (ce - cb) * (t + 1) / nt;
            if (a >= z) return;
            uint64_t i = (uint64_t)(std::upper_bound(h_ebase, h_ebase + nC, (unsigned long long)a) - h_ebase);
            if (i == 0) { bad = 1; return; }
            --i;
            for (uint64_t pos = a; pos < z; ++i) {
                if (i >= nC) { bad = 1; return; }
                const uint64_t e_hi = i + 1 < nC ? h_ebase[i + 1] : c_edges;
                const uint64_t take = std::min<uint64_t>(e_hi, z) - pos;
                const uint64_t src = h_soff[i] + (pos - h_ebase[i]);
                if (e_hi <= pos || src + take > E) { bad = 1; return; }
                std::memcpy(sd + (pos - cb), hd + src, take * 4);
                if (n_arrays == 2) std::memcpy(sw + (pos - cb), hw + src, take * 4);
                pos += take;
            }
        };
        c->pool->run(job);
        if (bad) return fail(c, HYTG_ERR_CUDA, "host compaction: active list out of range");
        {
            ScopedTime tm(c, HYTG_K_GATHER_C, c->s_c, false);
            tm.bytes = (ce - cb) * 4ull * n_arrays;
            CK(cudaMemcpyAsync(cv.cmp_dst, sd, (ce - cb) * 4, cudaMemcpyHostToDevice, c->s_c));
            if (n_arrays == 2)
                CK(cudaMemcpyAsync(cv.cmp_w, sw, (ce - cb) * 4, cudaMemcpyHostToDevice, c->s_c));
        }
        CK(cudaEventRecord(c->ev_cstage[b], c->s_c));
        RelaxTask r{};
        r.route = kRouteC; r.mode = kModeCompact; r.dst = cv.cmp_dst; r.w = cv.cmp_w;
        r.shift = (long long)cb; r.k_begin = cb; r.k_end = ce; r.first_entry = 0;
        r.device_sized = false;
        r.src_len = ce - cb;
        {
            ScopedTime tm(c, HYTG_K_RELAX_C, c->s_c);
            CK(relax_any(c, st, la, dsum, r, 8 * (int)device_sms(), c->s_c));
        }
    }
    c->stats.host_compact_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    CK(cudaEventRecord(c->ev_c, c->s_c));
    CK(cudaStreamWaitEvent(c->s_main, c->ev_c, 0));
    return HYTG_OK;
}

// Issue one iteration's route work after its summary reached the host:
// F tasks (task combination of Alg. 1, copy + relax per stream), the C
// route in chunks of the compaction buffer, and the per-iteration statistics.
// Leaves s_main waiting on every stream used.
hytg_status issue_work(hytg_ctx *c, int algo, unsigned int bucket, const char *hb, int n_arrays) {
    const SumLayout L = sum_layout((uint32_t)(c->part_vb.size() - 1));
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    const uint64_t ebytes = 4ull * n_arrays;
    const Summary *hs = (const Summary *)hb;
    Carve &cv = c->carve;
    std::vector<int> f_streams_used;
    const unsigned long long *p_edges = (const unsigned long long *)(hb + L.edges);
    const unsigned long long *p_rentry = (const unsigned long long *)(hb + L.route_entry);
    const unsigned long long *p_redge = (const unsigned long long *)(hb + L.route_edge);
    const unsigned char *p_route = (const unsigned char *)(hb + L.route);
    hytg_iter_record rec{};
    rec.active_vertices = hs->n_active;
    AlgoState st = algo_state(c, algo, bucket);
    ListArrays la = list_arrays(c);
    Summary *dsum = (Summary *)c->d_sumbuf;
    // --- F: task combination (Alg. 1, k consecutive partitions, slot capacity)
    std::vector<FTask> &tasks = c->f_tasks_buf;
    tasks.clear();
    const unsigned long long *p_prio = (const unsigned long long *)(hb + L.prio);
    const bool by_delta = algo_state(c, algo).prio != 0;
    uint32_t i = 0;
    while (i < N) {
        if (p_route[i] != kRouteF) { ++i; continue; }
        uint32_t j = i;
        uint64_t edges = c->part_eb[i + 1] - c->part_eb[i];
        uint64_t pr = by_delta ? p_prio[i] : 0;
        while (j + 1 < N && p_route[j + 1] == kRouteF && (j + 1 - i + 1) <= (uint32_t)c->k &&
               edges + (c->part_eb[j + 2] - c->part_eb[j + 1]) <= cv.slot_edges) {
            ++j;
            edges += c->part_eb[j + 1] - c->part_eb[j];
            if (by_delta) pr += p_prio[j];
        }
        tasks.push_back({i, j, edges, pr});
        i = j + 1;
    }
    // delta-driven priority (Sec. VI-A): the tasks whose partitions hold the
    // most pending delta go first; otherwise partition order, which puts the
    // hub partitions (hub sorting) first
    if (by_delta)
        std::stable_sort(tasks.begin(), tasks.end(),
                         [](const FTask &a, const FTask &b) { return a.prio > b.prio; });
    uint64_t f_bytes = 0;
    uint32_t n_tasks = 0;
    f_streams_used.clear();
    // Staging-slot reuse ("slot_reuse" 1): a task whose partitions a slot
    // still holds from an earlier iteration (the same combined range and
    // arrays; the edge arrays do not change during a run) runs from that slot
    // without a copy.  Those tasks go first, since they need no transfer; the
    // other tasks keep their order.  Off by default: on R-MAT 24 PageRank it
    // saved 16 % of the F bytes but took longer (343-357 ms against
    // 312-317), because the reused tasks' relaxes delay the copied tasks'
    // relaxes, and with them the slots the copies wait for.
    std::vector<int> &hit = c->f_hit_buf;
    std::vector<uint32_t> &order = c->f_order_buf;
    hit.assign(tasks.size(), -1);
    order.clear();
    uint32_t reserved = 0;                    // bit s: slot s serves a task of this iteration from memory
    // Copies ahead ("f_ahead" > 0; single-source runs on the host loop): the
    // end of the previous iteration copied its first tasks into slots, as a
    // guess at this iteration's first tasks, while the link would otherwise
    // idle through that iteration's last relaxes and this iteration's
    // planning.  A task found among them runs from its slot and keeps its
    // place in the order; until it is issued, copied tasks skip its slot.
    const bool ahead = ahead_on(c);
    uint32_t pending = 0;                     // bit s: slot s holds a copy ahead for a task not issued yet
    uint32_t missed = 0;                      // bit s: slot s holds a copy ahead that no task uses
    for (const hytg_ctx::AheadCopy &a : c->ahead) {
        bool used = false;
        if (ahead && c->ahead_seq == c->work_seq)
            for (size_t k = 0; k < tasks.size() && !used; ++k)
                if (hit[k] < 0 && a.n_arrays == n_arrays && tasks[k].i == a.i0 && tasks[k].j == a.j) {
                    hit[k] = (int)a.slot;
                    pending |= 1u << a.slot;
                    used = true;
                }
        if (!used) missed |= 1u << a.slot;
    }
    c->ahead.clear();
    if (ahead) {
        for (size_t k = 0; k < tasks.size(); ++k) order.push_back((uint32_t)k);
    } else if (c->slot_reuse != 0) {
        for (size_t k = 0; k < tasks.size(); ++k)
            for (uint32_t s = 0; s < cv.n_slots; ++s) {
                const hytg_ctx::SlotHeld &h = c->slot_held[s];
                if (!((reserved >> s) & 1u) && h.n_arrays == n_arrays && h.i0 == tasks[k].i && h.j == tasks[k].j) {
                    hit[k] = (int)s;
                    reserved |= 1u << s;
                    order.push_back((uint32_t)k);
                    break;
                }
            }
    }
    if (!ahead)
        for (size_t k = 0; k < tasks.size(); ++k)
            if (hit[k] < 0) order.push_back((uint32_t)k);
    // Tasks take the F compute streams in turn, and copied tasks take all the
    // slots in turn, reused ones included: those tasks were issued first, so
    // the copy into such a slot waits only for that task's relax, and the
    // ring keeps every slot for copying ahead.  There are more slots than
    // compute streams, and each slot has its own copy stream, so the copy of
    // a later task runs while earlier tasks' relaxes and second passes still
    // hold their slots.
    const uint32_t n_fs = std::max<uint32_t>(1, std::min<uint32_t>(cv.n_slots, (uint32_t)c->streams));
    uint32_t rr = ahead ? c->ring_pos : 0;
    int last_copied = -1;                     // slot of this iteration's last copy
    // An F copy by the copy engine moves the task's edges exactly; the copy
    // kernel ("f_copy" > 0) starts at the 16-byte boundary at or below the
    // first edge, so the slot then holds up to 3 words before it (when it has
    // room for them).  base_of gives the first edge a slot holds for a task.
    auto by_kernel = [&](uint64_t e0, uint64_t edges) {
        return c->f_copy > 0 && edges + (e0 & 3) <= cv.slot_edges;
    };
    auto base_of = [&](uint64_t e0, uint64_t edges) -> uint64_t {
        return by_kernel(e0, edges) ? (e0 & ~uint64_t(3)) : e0;
    };
    auto copy_task = [&](uint32_t slot, uint64_t e0, uint64_t edges, cudaStream_t cs) -> cudaError_t {
        cudaError_t e;
        if (by_kernel(e0, edges)) {
            const uint64_t ea = e0 & ~uint64_t(3);
            e = launch_stage_copy(c->m_dst + ea, cv.slot_dst[slot], e0 + edges - ea, (unsigned)c->f_copy, cs);
            if (e == cudaSuccess && n_arrays == 2)
                e = launch_stage_copy(c->m_w + ea, cv.slot_w[slot], e0 + edges - ea, (unsigned)c->f_copy, cs);
            c->stats.kernel_launches += n_arrays;
        } else {
            e = cudaMemcpyAsync(cv.slot_dst[slot], c->h_dst + e0, edges * 4, cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess && n_arrays == 2)
                e = cudaMemcpyAsync(cv.slot_w[slot], c->h_w + e0, edges * 4, cudaMemcpyHostToDevice, cs);
        }
        return e;
    };
    for (uint32_t k : order) {
        const FTask &ft = tasks[k];
        const uint32_t i0 = ft.i, j = ft.j;
        const uint64_t edges = ft.edges;
        const bool reuse = hit[k] >= 0;
        uint32_t slot;
        if (reuse) {
            slot = (uint32_t)hit[k];
            pending &= ~(1u << slot);
        } else {
            // at most f_ahead < n_slots slots are pending, so this ends
            do slot = rr++ % cv.n_slots;
            while ((pending >> slot) & 1u);
        }
        const uint32_t fi = n_tasks % n_fs;
        cudaStream_t fs = c->s_f[fi], cs = c->s_cp[slot];
        const uint64_t e0 = c->part_eb[i0];
        if (!reuse) {
            // the copy needs only the route decision (already on the host)
            // and the end of the slot's previous use, not the lists
            c->slot_held[slot] = hytg_ctx::SlotHeld();
            CK(cudaStreamWaitEvent(cs, c->ev_free[slot], 0));
            {
                ScopedTime t(c, HYTG_K_COPY_F, cs);
                t.bytes = (e0 + edges - base_of(e0, edges)) * ebytes;
                t.part_first = i0;
                t.part_last = j;
                CK(copy_task(slot, e0, edges, cs));
            }
            CK(cudaEventRecord(c->ev_copied[slot], cs));
            c->slot_held[slot] = {i0, j, n_arrays};
            last_copied = (int)slot;
        } else if (ahead) {
            // copied ahead: its bytes were counted when the copy was issued
            c->stats.f_ahead_hits += 1;
        } else {
            // the slot's last copy finished before the previous iteration
            // ended (its relax waited for it, and the main stream for that)
            c->stats.f_reused_tasks += 1;
            c->stats.f_reused_bytes += edges * ebytes;
        }
        if (std::find(f_streams_used.begin(), f_streams_used.end(), (int)fi) == f_streams_used.end()) {
            f_streams_used.push_back((int)fi);
            CK(cudaStreamWaitEvent(fs, c->ev_bin, 0));
        }
        // a copy ahead may still be in flight; a reused slot's copy is not
        if (!reuse || ahead) CK(cudaStreamWaitEvent(fs, c->ev_copied[slot], 0));
        const uint64_t ea = base_of(e0, edges);
        RelaxTask t{};
        t.route = kRouteF; t.mode = kModeDevice; t.dst = cv.slot_dst[slot]; t.w = cv.slot_w[slot];
        t.shift = (long long)ea;
        t.k_begin = p_redge[i0];
        t.k_end = p_redge[j] + p_edges[j];
        t.first_entry = p_rentry[i0];
        t.device_sized = false;
        t.src_len = e0 + edges - ea;
        {
            ScopedTime tm(c, HYTG_K_RELAX_F, fs);
            tm.edges = t.k_end - t.k_begin;
            tm.part_first = i0;
            tm.part_last = j;
            CK(relax_any(c, st, la, dsum, t, 8 * (int)device_sms(), fs));
        }
        if (second_pass_on(c, algo) && range_second_pass(c, edges, c->part_vb[j + 1] - c->part_vb[i0])) {
            ScopedTime tm(c, kKindSecondPass, fs);
            unsigned long long *ctr = next_sp_slot(c, &tm.sp_slot);
            tm.vertices = c->part_vb[j + 1] - c->part_vb[i0];
            tm.part_first = i0;
            tm.part_last = j;
            CK(second_pass_any(c, st, cv.slot_dst[slot], cv.slot_w[slot], (long long)ea, e0 + edges - ea,
                               c->part_vb[i0], c->part_vb[j + 1], e0, c->part_eb[j + 1], ctr, fs));
            count_second_launch(c);
            c->stats.second_pass_vertices += c->part_vb[j + 1] - c->part_vb[i0];
        }
        CK(cudaEventRecord(c->ev_free[slot], fs));
        if (!reuse) f_bytes += (e0 + edges - ea) * ebytes;
        ++n_tasks;
    }
    // --- C: gather active lists into the compaction buffer, relax, in chunks
    const uint64_t c_edges = hs->route_edges[kRouteC];
    if (c_edges && c->compact_host > 0) {
        hytg_status hs_c = host_compact(c, algo, bucket, hs, n_arrays);
        if (hs_c != HYTG_OK) return hs_c;
    } else if (c_edges) {
        CK(cudaStreamWaitEvent(c->s_c, c->ev_bin, 0));
        for (uint64_t cb = 0; cb < c_edges; cb += cv.compact_edges) {
            const uint64_t ce = std::min<uint64_t>(c_edges, cb + cv.compact_edges);
            RelaxTask g{};
            g.route = kRouteC; g.mode = kModeHost; g.dst = c->m_dst; g.w = c->m_w; g.shift = 0;
            g.k_begin = cb; g.k_end = ce; g.first_entry = 0; g.device_sized = false;
            g.src_len = c->E; g.link_ctr = c->d_link_ctr + 2 * kRouteC;
            {
                ScopedTime tm(c, HYTG_K_GATHER_C, c->s_c);
                CK(launch_gather(la, dsum, g, cv.cmp_dst, n_arrays == 2 ? cv.cmp_w : nullptr, 8 * (int)device_sms(), c->s_c));
            }
            RelaxTask r{};
            r.route = kRouteC; r.mode = kModeCompact; r.dst = cv.cmp_dst; r.w = cv.cmp_w;
            r.shift = (long long)cb; r.k_begin = cb; r.k_end = ce; r.first_entry = 0;
            r.device_sized = false;
            r.src_len = ce - cb;
            {
                ScopedTime tm(c, HYTG_K_RELAX_C, c->s_c);
                CK(relax_any(c, st, la, dsum, r, 8 * (int)device_sms(), c->s_c));
            }
        }
        CK(cudaEventRecord(c->ev_c, c->s_c));
        CK(cudaStreamWaitEvent(c->s_main, c->ev_c, 0));
    }
    for (int sl : f_streams_used) {
        CK(cudaEventRecord(c->ev_f[sl], c->s_f[sl]));
        CK(cudaStreamWaitEvent(c->s_main, c->ev_f[sl], 0));
    }
    // a copy ahead that no task used is still joined, so that the run's end
    // (and its device time) covers every copy it issued
    for (uint32_t sl = 0; sl < (uint32_t)kMaxSlots; ++sl)
        if ((missed >> sl) & 1u) CK(cudaStreamWaitEvent(c->s_main, c->ev_copied[sl], 0));
    // --- copies ahead for the next iteration: this iteration's first tasks,
    // into the least recently used slots of the ring.  Each waits for its
    // slot's last relax and for this iteration's last copy, so that it runs
    // in the gap that the iteration's last relaxes and the next planning
    // leave on the link, not among this iteration's copies; the main stream
    // does not wait for them.
    if (ahead && !tasks.empty()) {
        cudaEvent_t after = last_copied >= 0 ? c->ev_copied[last_copied] : nullptr;
        const uint32_t n_ahead = std::min<uint32_t>({(uint32_t)c->f_ahead, cv.n_slots - 1, (uint32_t)order.size()});
        for (uint32_t q = 0; q < n_ahead; ++q) {
            const FTask &ft = tasks[order[q]];
            const uint32_t slot = rr++ % cv.n_slots;
            const uint64_t e0 = c->part_eb[ft.i];
            cudaStream_t cs = c->s_cp[slot];
            c->slot_held[slot] = hytg_ctx::SlotHeld();
            CK(cudaStreamWaitEvent(cs, c->ev_free[slot], 0));
            if (after) CK(cudaStreamWaitEvent(cs, after, 0));
            const uint64_t words = e0 + ft.edges - base_of(e0, ft.edges);
            {
                ScopedTime t(c, HYTG_K_COPY_F, cs);
                t.bytes = words * ebytes;
                t.part_first = ft.i;
                t.part_last = ft.j;
                CK(copy_task(slot, e0, ft.edges, cs));
            }
            CK(cudaEventRecord(c->ev_copied[slot], cs));
            c->slot_held[slot] = {ft.i, ft.j, n_arrays};
            c->ahead.push_back({slot, ft.i, ft.j, n_arrays});
            c->stats.f_ahead_tasks += 1;
            f_bytes += words * ebytes;
        }
        c->ahead_seq = c->work_seq + 1;
    }
    if (ahead) c->ring_pos = rr % std::max<uint32_t>(1, cv.n_slots);
    ++c->work_seq;
    // --- statistics of this iteration
    uint64_t act_edges = 0;
    for (int r = 0; r < kRoutes; ++r) {
        act_edges += hs->route_edges[r];
        rec.route_partitions[r] = hs->route_parts[r];
        rec.route_edges[r] = hs->route_edges[r];
        c->stats.route_partitions[r] += hs->route_parts[r];
        c->stats.route_vertices[r] += hs->route_entries[r];
        c->stats.route_edges[r] += hs->route_edges[r];
    }
    const uint64_t zb = hs->route_lines[kRouteZ] * (uint64_t)c->m;
    // host compaction moves the active lists themselves plus their index
    // (soff, ebase) back to the host; the GPU gather reads 128-byte lines
    const uint64_t cbts = c->compact_host > 0
        ? hs->route_edges[kRouteC] * ebytes + hs->route_entries[kRouteC] * 16
        : hs->route_lines[kRouteC] * (uint64_t)c->m;
    c->stats.link_bytes[kRouteF] += f_bytes;
    c->stats.link_bytes[kRouteZ] += zb;
    c->stats.link_bytes[kRouteC] += cbts;
    c->stats.f_tasks += n_tasks;
    c->last_fc = n_tasks > 0 || c_edges > 0;
    c->stats.edges_relaxed += act_edges;
    c->stats.vertices_processed += hs->n_active;
    rec.active_edges = act_edges;
    rec.f_tasks = n_tasks;
    rec.link_bytes = f_bytes + zb + cbts;
    c->iters.push_back(rec);
    return HYTG_OK;
}

// One launch of the device loop from iteration `it`: uploads the control
// block, replays the graph, and folds the device iterations' records and
// totals into the run's statistics.  On return `it` and `bucket` are those
// of the iteration the loop stopped at and `status` says why it stopped.
// A run past its "run_timeout_ms" deadline stops at an iteration boundary:
// wait for everything already issued on the context's streams, so that the
// context is idle and the next call can use it, and report the timeout.
hytg_status run_timed_out(hytg_ctx *c, uint32_t it) {
    cudaStream_t all[2 + kMaxStreams + kMaxSlots] = {c->s_main, c->s_c};
    int n = 2;
    for (int i = 0; i < kMaxStreams; ++i) all[n++] = c->s_f[i];
    for (int i = 0; i < kMaxSlots; ++i) all[n++] = c->s_cp[i];
    for (int i = 0; i < n; ++i)
        if (all[i]) CK(cudaStreamSynchronize(all[i]));
    c->ahead.clear();
    c->have_result = false;
    c->stats.iterations = it;
    return fail(c, HYTG_ERR_TIMEOUT,
                "the run passed run_timeout_ms (" + std::to_string(c->run_timeout_ms) + " ms) at iteration " +
                    std::to_string(it) + "; its result is not available");
}

bool past_deadline(const hytg_ctx *c) {
    return c->has_deadline && std::chrono::steady_clock::now() >= c->run_deadline;
}

hytg_status run_device_loop(hytg_ctx *c, uint32_t &it, unsigned int &bucket, uint64_t delta, int &status) {
    LoopCtl &h = *c->h_loop;
    std::memset(&h, 0, sizeof(LoopCtl));
    h.status = kLoopRun;
    h.it = it;
    h.bucket = bucket;
    h.rec_cap = c->loop_rec_cap;
    h.delta = delta;
    h.max_it = (unsigned long long)c->max_iters;
    h.m = (unsigned long long)c->m;
    h.rec = c->d_loop_rec;
    if (c->loop_fc) {
        const PartArrays pa = part_arrays(c);
        h.f_handles = c->d_loop_fh;
        h.c_handle = c->loop_ch;
        h.c_cap = c->carve.compact_edges;
        h.route = pa.route;
        h.part_eb = c->d_part_eb;
        h.n_parts = (unsigned int)(c->part_vb.size() - 1);
        h.n_arrays = c->last_run_arrays;
    }
    h.cancel = c->has_deadline ? c->d_cancel : nullptr;
    if (c->loop_fc) {
        // the graph's F nodes copy into the slots: copies ahead end first
        // (the graph is launched on the main stream) and are dropped
        CK(ahead_join(c));
        slots_forget(c);
    }
    iteration_mark(c);
    CK(cudaMemcpyAsync(c->d_loop, c->h_loop, sizeof(LoopCtl), cudaMemcpyHostToDevice, c->s_main));
    CK(cudaGraphLaunch(c->loop_exec, c->s_main));
    CK(cudaMemcpyAsync(c->h_loop, c->d_loop, sizeof(LoopCtl), cudaMemcpyDeviceToHost, c->s_main));
    if (c->has_deadline) {
        // past the deadline the host sets the cancel word; k_loop_decide reads
        // it at the next iteration boundary and ends the loop, so the launch
        // still ends after at most one more iteration
        for (;;) {
            const cudaError_t q = cudaStreamQuery(c->s_main);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) CK(q);
            if (*(volatile unsigned int *)c->h_cancel == 0u && std::chrono::steady_clock::now() >= c->run_deadline) {
                *(volatile unsigned int *)c->h_cancel = 1u;
                std::atomic_thread_fence(std::memory_order_seq_cst);
            }
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    } else {
        CK(cudaStreamSynchronize(c->s_main));
    }
    const uint32_t n = std::min<uint32_t>(h.n_rec, c->loop_rec_cap);
    if (n) {
        const size_t base = c->iters.size();
        c->iters.resize(base + n);
        CK(cudaMemcpy(c->iters.data() + base, c->d_loop_rec, n * sizeof(hytg_iter_record), cudaMemcpyDeviceToHost));
    }
    for (int r = 0; r < kRoutes; ++r) {
        c->stats.route_partitions[r] += h.route_parts[r];
        c->stats.route_vertices[r] += h.route_entries[r];
        c->stats.route_edges[r] += h.route_edges[r];
    }
    c->stats.link_bytes[kRouteZ] += h.z_lines * (uint64_t)c->m;
    c->stats.link_bytes[kRouteF] += h.f_bytes;
    c->stats.link_bytes[kRouteC] += h.c_lines * (uint64_t)c->m;
    c->stats.f_tasks += h.f_parts;
    c->stats.edges_relaxed += h.edges;
    c->stats.vertices_processed += h.vertices;
    c->stats.graph_launches += 1;
    c->stats.graph_iterations += h.iterations;
    // every body run launches the whole body; gated kernels return at once
    c->stats.kernel_launches += (uint64_t)c->loop_kernels * ((uint64_t)(h.it - it) + 1) +
                                h.f_parts * c->loop_f_kernels + h.c_iters * c->loop_c_kernels;
    it = h.it;
    bucket = h.bucket;
    status = (int)h.status;
    return HYTG_OK;
}

}  // namespace

// ===================================================================== ABI
extern "C" {

const char *hytg_status_str(hytg_status s) {
    unsigned i = (unsigned)s;
    return i < sizeof(kStatusStr) / sizeof(kStatusStr[0]) ? kStatusStr[i] : "unknown status";
}

const char *hytg_last_error(hytg_ctx *c) { return c ? c->err.c_str() : "null context"; }

hytg_status hytg_create(hytg_ctx **out, int device) {
    if (!out) return HYTG_ERR_ARG;
    *out = nullptr;
    hytg_ctx *c = new (std::nothrow) hytg_ctx();
    if (!c) return HYTG_ERR_HOSTMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete c; return HYTG_ERR_CUDA; }
    hytg_status s = HYTG_OK;
    auto ck = [&](cudaError_t r) { if (r != cudaSuccess && s == HYTG_OK) s = HYTG_ERR_CUDA; };
    ck(cudaStreamCreateWithFlags(&c->s_main, cudaStreamNonBlocking));
    ck(cudaStreamCreateWithFlags(&c->s_c, cudaStreamNonBlocking));
    for (int i = 0; i < kMaxStreams; ++i) {
        ck(cudaStreamCreateWithFlags(&c->s_f[i], cudaStreamNonBlocking));
        ck(cudaEventCreateWithFlags(&c->ev_f[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < kMaxSlots; ++i) {
        ck(cudaStreamCreateWithFlags(&c->s_cp[i], cudaStreamNonBlocking));
        ck(cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < 2; ++i) ck(cudaEventCreateWithFlags(&c->ev_sum[i], cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&c->ev_bin, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&c->ev_c, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) ck(cudaEventCreateWithFlags(&c->ev_cstage[i], cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&c->ev_clist, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) ck(cudaEventCreate(&c->ev_run[i]));
    ck(cudaMalloc(&c->d_overflow, sizeof(unsigned int)));
    ck(cudaMalloc(&c->d_err, sizeof(unsigned int)));
    ck(cudaMemset(c->d_err, 0, sizeof(unsigned int)));
    ck(cudaMalloc(&c->d_prsums, 2 * sizeof(double)));
    ck(cudaMalloc(&c->d_src, 64 * sizeof(unsigned int)));
    ck(cudaMalloc(&c->d_src_work, sizeof(unsigned long long)));
    ck(cudaMalloc(&c->d_bsums, 64 * sizeof(double)));
    ck(cudaMalloc(&c->d_alive, sizeof(unsigned long long)));
    ck(cudaMalloc(&c->d_sp, kSpSlots * sizeof(unsigned long long)));
    ck(cudaMalloc(&c->d_link_ctr, 2 * kRoutes * sizeof(unsigned long long)));
    ck(cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking));
    ck(cudaStreamCreateWithFlags(&c->s_cap2, cudaStreamNonBlocking));
    ck(cudaMalloc(&c->d_loop_fh, 1024 * sizeof(unsigned long long)));
    ck(cudaMalloc(&c->d_loop, sizeof(LoopCtl)));
    ck(cudaMalloc(&c->d_loop_rec, (size_t)c->loop_rec_cap * sizeof(hytg_iter_record)));
    ck(cudaHostAlloc((void **)&c->h_loop, sizeof(LoopCtl), cudaHostAllocDefault));
    ck(cudaHostAlloc((void **)&c->h_cancel, sizeof(unsigned int), cudaHostAllocMapped));
    if (c->h_cancel) {
        *c->h_cancel = 0u;
        ck(cudaHostGetDevicePointer((void **)&c->d_cancel, c->h_cancel, 0));
    }
    if (s != HYTG_OK) { hytg_destroy(c); return s; }
    *out = c;
    return HYTG_OK;
}

hytg_status hytg_destroy(hytg_ctx *c) {
    if (!c) return HYTG_ERR_ARG;
    cudaSetDevice(c->device);
    if (c->s_main) cudaStreamSynchronize(c->s_main);
    free_graph(c);
    dfree(c->d_pool);
    dfree(c->d_overflow);
    dfree(c->d_err);
    dfree(c->d_prsums);
    dfree(c->d_src);
    dfree(c->d_src_work);
    dfree(c->d_bsums);
    dfree(c->d_alive);
    dfree(c->d_sp);
    dfree(c->d_link_ctr);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < kMaxStreams; ++i) {
        if (c->s_f[i]) cudaStreamDestroy(c->s_f[i]);
        if (c->ev_f[i]) cudaEventDestroy(c->ev_f[i]);
    }
    for (int i = 0; i < kMaxSlots; ++i) {
        if (c->s_cp[i]) cudaStreamDestroy(c->s_cp[i]);
        if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
        if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
    }
    for (int i = 0; i < 2; ++i) if (c->ev_sum[i]) cudaEventDestroy(c->ev_sum[i]);
    if (c->ev_bin) cudaEventDestroy(c->ev_bin);
    if (c->ev_c) cudaEventDestroy(c->ev_c);
    for (int i = 0; i < 2; ++i) if (c->ev_run[i]) cudaEventDestroy(c->ev_run[i]);
    free_loop_graph(c);
    dfree(c->d_loop);
    dfree(c->d_loop_rec);
    if (c->h_loop) cudaFreeHost(c->h_loop);
    if (c->h_cancel) cudaFreeHost(c->h_cancel);
    if (c->s_cap) cudaStreamDestroy(c->s_cap);
    if (c->s_cap2) cudaStreamDestroy(c->s_cap2);
    dfree(c->d_loop_fh);
    delete c->pool;
    for (int i = 0; i < 2; ++i) {
        if (c->h_cstage[i]) cudaFreeHost(c->h_cstage[i]);
        if (c->ev_cstage[i]) cudaEventDestroy(c->ev_cstage[i]);
    }
    if (c->h_clist) cudaFreeHost(c->h_clist);
    if (c->ev_clist) cudaEventDestroy(c->ev_clist);
    if (c->s_c) cudaStreamDestroy(c->s_c);
    if (c->s_main) cudaStreamDestroy(c->s_main);
    delete c;
    return HYTG_OK;
}

hytg_status hytg_load_csr(hytg_ctx *c, uint64_t V, uint64_t E, const uint64_t *offsets,
                          const uint32_t *dst, const uint32_t *weights) {
    if (!c) return HYTG_ERR_ARG;
    try {
        if (V == 0 || V > 0xFFFFFFFFull) return fail(c, HYTG_ERR_ARG, "V must be in [1, 2^32-1]");
        if (!offsets || (E > 0 && !dst)) return fail(c, HYTG_ERR_ARG, "null CSR array");
        if (offsets[0] != 0 || offsets[V] != E) return fail(c, HYTG_ERR_ARG, "offsets[0] must be 0 and offsets[V] must be E");
        bool ok = true;
        for (uint64_t v = 0; v < V && ok; ++v) ok = offsets[v] <= offsets[v + 1];
        if (!ok) return fail(c, HYTG_ERR_ARG, "offsets must be non-decreasing");
        {
            std::vector<char> bad(16, 0);
            std::atomic<bool> any_bad{false};
            parallel_chunks(E, [&](uint64_t lo, uint64_t hi) {
                for (uint64_t e = lo; e < hi; ++e)
                    if (dst[e] >= V) { any_bad = true; return; }
            });
            if (any_bad) return fail(c, HYTG_ERR_ARG, "dst entry out of range");
        }
        CK(cudaSetDevice(c->device));
        CK(cudaDeviceSynchronize());
        free_graph(c);
        if (getenv("HYTG_INJECT_HOSTMEM_FAIL") && atoi(getenv("HYTG_INJECT_HOSTMEM_FAIL")) != 0)
            return fail(c, HYTG_ERR_HOSTMEM, "pinned allocation failure injected by HYTG_INJECT_HOSTMEM_FAIL");
        const size_t eb = std::max<uint64_t>(E, 1) * 4;
        if (alloc_edge_array(c, 0, &c->h_dst, eb) != HYTG_OK)
            return fail(c, HYTG_ERR_HOSTMEM, "pinned allocation of the neighbour array failed");
        if (weights && alloc_edge_array(c, 1, &c->h_w, eb) != HYTG_OK) {
            free_graph(c);
            return fail(c, HYTG_ERR_HOSTMEM, "pinned allocation of the weight array failed");
        }
        if (c->hub_frac > 0.0) {
            // hub sorting: relabel so that the hubs are internal ids [0, n_hubs)
            c->h_perm.resize(V);
            uint64_t nh = 0;
            hytg_status hs = hytg_hub_order(V, offsets, dst, c->hub_frac, c->h_perm.data(), &nh);
            if (hs != HYTG_OK) { free_graph(c); return fail(c, hs, "hub ordering failed"); }
            c->h_inv.resize(V);
            for (uint64_t n = 0; n < V; ++n) c->h_inv[c->h_perm[n]] = (uint32_t)n;
            c->h_off.assign(V + 1, 0);
            for (uint64_t n = 0; n < V; ++n) {
                const uint64_t o = c->h_perm[n];
                c->h_off[n + 1] = c->h_off[n] + (offsets[o + 1] - offsets[o]);
            }
            const uint32_t *inv = c->h_inv.data();
            parallel_chunks(V, [&](uint64_t lo, uint64_t hi) {
                for (uint64_t n = lo; n < hi; ++n) {
                    const uint64_t o = c->h_perm[n], s0 = offsets[o], len = offsets[o + 1] - s0;
                    uint32_t *d = c->h_dst + c->h_off[n];
                    for (uint64_t j = 0; j < len; ++j) d[j] = inv[dst[s0 + j]];
                    if (weights) memcpy(c->h_w + c->h_off[n], weights + s0, len * 4);
                }
            });
            c->permuted = true;
            c->n_hubs = nh;
        } else {
            parallel_chunks(E, [&](uint64_t lo, uint64_t hi) {
                memcpy(c->h_dst + lo, dst + lo, (hi - lo) * 4);
                if (weights) memcpy(c->h_w + lo, weights + lo, (hi - lo) * 4);
            });
            c->h_off.assign(offsets, offsets + V + 1);
        }
        void *mp = nullptr;
        CK(cudaHostGetDevicePointer(&mp, c->h_dst, 0));
        c->m_dst = (const uint32_t *)mp;
        if (weights) {
            CK(cudaHostGetDevicePointer(&mp, c->h_w, 0));
            c->m_w = (const uint32_t *)mp;
        }
        c->V = V;
        c->E = E;
        c->weighted = weights != nullptr;
        c->part_edges = std::max<uint64_t>(1, (uint64_t)(c->part_bytes / 4));
        make_partitions(c);
        c->n_words_alloc = ((V + 31) / 32 + kBitmapPadWords - 1) / kBitmapPadWords * kBitmapPadWords;
        CK(cudaMalloc(&c->d_off, (V + 1) * 8));
        CK(cudaMemcpy(c->d_off, c->h_off.data(), (V + 1) * 8, cudaMemcpyHostToDevice));
        if (c->permuted) {
            CK(cudaMalloc(&c->d_perm, V * 4));
            CK(cudaMemcpy(c->d_perm, c->h_perm.data(), V * 4, cudaMemcpyHostToDevice));
            c->n_hub_rep = (unsigned int)std::min<uint64_t>(c->n_hubs, (uint64_t)c->hub_replicas);
            if (c->n_hub_rep) {
                CK(cudaMalloc(&c->d_hub_rep, (size_t)kHubReplicas * c->n_hub_rep * 4));
                CK(cudaMemset(c->d_hub_rep, 0, (size_t)kHubReplicas * c->n_hub_rep * 4));
            }
        }
        CK(cudaMalloc(&c->d_val, V * 4));
        CK(cudaMalloc(&c->d_delta, V * 4));
        CK(cudaMalloc(&c->d_out, V * 4));
        CK(cudaMalloc(&c->d_sp_owner, (E / kSpChunk + 2) * 4));
        CK(cudaMalloc(&c->d_sp_mask, c->n_words_alloc * 4));
        CK(cudaMalloc(&c->d_bm[0], c->n_words_alloc * 4));
        CK(cudaMemset(c->d_bm[0], 0, c->n_words_alloc * 4));
        CK(cudaMalloc(&c->d_ebase, V * 8));
        CK(cudaMalloc(&c->d_soff, V * 8));
        CK(cudaMalloc(&c->d_pay, V * 4));
        const uint64_t n_tiles = E / kTile + 8;
        CK(cudaMalloc(&c->d_tiles, n_tiles * 4));
        c->n_tiles_alloc = n_tiles;
        hytg_status s = upload_partitions(c);
        if (s != HYTG_OK) return s;
        c->vertex_bytes = (V + 1) * 8 + 3 * V * 4 + c->n_words_alloc * 4 + V * 20 + n_tiles * 4 +
                          c->sum_dev_bytes + (E / kSpChunk + 2) * 4 + c->n_words_alloc * 4;
        if (c->weighted) {
            // automatic SSSP bucket width: 8 x the mean edge weight (delta-stepping)
            long double sw = 0;
            for (uint64_t e = 0; e < E; e += std::max<uint64_t>(1, E / 4096)) sw += weights[e];
            const uint64_t ns = (E + std::max<uint64_t>(1, E / 4096) - 1) / std::max<uint64_t>(1, E / 4096);
            c->auto_delta = ns ? (uint64_t)std::max<long double>(1.0L, 8.0L * sw / ns) : 1;
        }
        c->loaded = true;
        return HYTG_OK;
    } catch (...) {
        return fail(c, HYTG_ERR_HOSTMEM, "host allocation failed");
    }
}

hytg_status hytg_set_device_budget(hytg_ctx *c, uint64_t bytes) {
    if (!c) return HYTG_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaDeviceSynchronize());
    dfree(c->d_pool);
    c->budget = 0;
    c->carve = Carve();
    c->cache_filled_arrays = 0;
    if (bytes == 0) return fail(c, HYTG_ERR_BUDGET, "zero budget");
    CK(cudaMalloc(&c->d_pool, bytes + kPoolSlack));
    c->budget = bytes;
    if (c->loaded) {
        hytg_status s = plan_carve(c, 1);
        if (s == HYTG_ERR_BUDGET) {
            // keep the pool; the error is reported again by hytg_run
            return s;
        }
    }
    return HYTG_OK;
}

hytg_status hytg_set_param(hytg_ctx *c, const char *key, double v) {
    if (!c || !key) return HYTG_ERR_ARG;
    std::string k(key);
    auto bad = [&]() { return fail(c, HYTG_ERR_ARG, "bad value for parameter " + k); };
    if (!std::isfinite(v)) return bad();
    if (k == "alpha") { if (v < 0 || v > 1000) return bad(); c->alpha = v; }
    else if (k == "beta") { if (v < 0 || v > 1000) return bad(); c->beta = v; }
    else if (k == "gamma") { if (v < 0 || v > 1) return bad(); c->gamma = v; }
    else if (k == "m") { if (v < 1 || v != std::floor(v)) return bad(); c->m = v; }
    else if (k == "MR") { if (v < 1 || v != std::floor(v)) return bad(); c->MR = v; }
    else if (k == "k") { if (v < 1 || v > 1024 || v != std::floor(v)) return bad(); c->k = v; c->carve = Carve(); }
    else if (k == "part_bytes") {
        if (v < 4 || v >= 64.0 * 1024 * 1024) return bad();   // < 2^24 edges per partition
        c->part_bytes = v;
        if (c->loaded) {
            CK(cudaSetDevice(c->device));
            c->part_edges = std::max<uint64_t>(1, (uint64_t)(v / 4));
            make_partitions(c);
            hytg_status s = upload_partitions(c);
            if (s != HYTG_OK) return s;
        }
    }
    else if (k == "streams") { if (v < 1 || v > kMaxStreams || v != std::floor(v)) return bad(); c->streams = v; c->carve = Carve(); }
    else if (k == "prefetch_slots") { if (v < 0 || v > 8 || v != std::floor(v)) return bad(); c->prefetch_slots = v; c->carve = Carve(); }
    else if (k == "staging_frac") { if (v <= 0 || v >= 1) return bad(); c->staging_frac = v; c->carve = Carve(); }
    else if (k == "compact_frac") { if (v <= 0 || v >= 1) return bad(); c->compact_frac = v; c->carve = Carve(); }
    else if (k == "force_route") { if (!(v == -1 || (v >= 1 && v <= 5)) || v != std::floor(v)) return bad(); c->force_route = v; }
    else if (k == "seed") { if (v < 0) return bad(); c->seed = v; }
    else if (k == "pr_damping") { if (v <= 0 || v >= 1) return bad(); c->pr_damping = v; }
    else if (k == "pr_eps") { if (v <= 0) return bad(); c->pr_eps = v; }
    else if (k == "max_iters") { if (v < 1) return bad(); c->max_iters = v; }
    else if (k == "run_timeout_ms") { if (v < 0) return bad(); c->run_timeout_ms = v; }
    else if (k == "slot_reuse") { if (v != 0 && v != 1) return bad(); c->slot_reuse = v; if (v == 0) slots_forget(c); }
    else if (k == "f_ahead") { if (v < 0 || v > kMaxSlots - 1 || v != std::floor(v)) return bad(); c->f_ahead = v; }
    else if (k == "f_copy") { if (v < 0 || v > 32 || v != std::floor(v)) return bad(); c->f_copy = v; slots_forget(c); }
    else if (k == "timing") { c->timing = v != 0 ? 1 : 0; }
    else if (k == "hub_frac") { if (v < 0 || v > 1) return bad(); c->hub_frac = v; }
    else if (k == "sssp_delta") { if (!(v == -1 || v >= 0) || v != std::floor(v) || v > 4e9) return bad(); c->sssp_delta = v; }
    else if (k == "two_pass") { if (v != 0 && v != 1 && v != 2) return bad(); c->two_pass = v; }
    else if (k == "two_pass_min_degree") { if (v < 0 || v > 1e6) return bad(); c->two_pass_min_degree = v; }
    else if (k == "hub_replicas") { if (v < 0 || v > 65536 || v != std::floor(v)) return bad(); c->hub_replicas = v; }
    else if (k == "compact_host") { if (v < 0 || v > 256 || v != std::floor(v)) return bad(); c->compact_host = v; }
    else if (k == "priority") { if (v != 0 && v != 1) return bad(); c->priority = v; }
    else if (k == "device_loop") { if (v != 0 && v != 1 && v != 2) return bad(); c->device_loop = v; }
    else if (k == "loop_after_fc") { if (v != 0 && v != 1) return bad(); c->loop_after_fc = v; }
    else if (k == "z_blocks") { if (v < 1 || v > 32 || v != std::floor(v)) return bad(); c->z_blocks = v; }
    else if (k == "host_huge") { if (v != 0 && v != 1) return bad(); c->host_huge = v; }
    else if (k == "serve_frames") { if (v < 0 || v > kMaxFrames || v != std::floor(v)) return bad(); c->serve_frames_param = v; }
    else if (k == "batch_sparse_below") { if (v < -1 || v > 65 || v != std::floor(v)) return bad(); c->batch_sparse_below = v; }
    else return fail(c, HYTG_ERR_ARG, "unknown parameter " + k);
    return HYTG_OK;
}

hytg_status hytg_get_param(hytg_ctx *c, const char *key, double *v) {
    if (!c || !key || !v) return HYTG_ERR_ARG;
    std::string k(key);
    if (k == "alpha") *v = c->alpha;
    else if (k == "beta") *v = c->beta;
    else if (k == "gamma") *v = c->gamma;
    else if (k == "m") *v = c->m;
    else if (k == "MR") *v = c->MR;
    else if (k == "k") *v = c->k;
    else if (k == "part_bytes") *v = c->part_bytes;
    else if (k == "streams") *v = c->streams;
    else if (k == "prefetch_slots") *v = c->prefetch_slots;
    else if (k == "staging_frac") *v = c->staging_frac;
    else if (k == "compact_frac") *v = c->compact_frac;
    else if (k == "force_route") *v = c->force_route;
    else if (k == "seed") *v = c->seed;
    else if (k == "pr_damping") *v = c->pr_damping;
    else if (k == "pr_eps") *v = c->pr_eps;
    else if (k == "max_iters") *v = c->max_iters;
    else if (k == "run_timeout_ms") *v = c->run_timeout_ms;
    else if (k == "slot_reuse") *v = c->slot_reuse;
    else if (k == "f_ahead") *v = c->f_ahead;
    else if (k == "f_copy") *v = c->f_copy;
    else if (k == "timing") *v = c->timing;
    else if (k == "hub_frac") *v = c->hub_frac;
    else if (k == "sssp_delta") *v = c->sssp_delta;
    else if (k == "two_pass") *v = c->two_pass;
    else if (k == "two_pass_min_degree") *v = c->two_pass_min_degree;
    else if (k == "hub_replicas") *v = c->hub_replicas;
    else if (k == "compact_host") *v = c->compact_host;
    else if (k == "priority") *v = c->priority;
    else if (k == "device_loop") *v = c->device_loop;
    else if (k == "loop_after_fc") *v = c->loop_after_fc;
    else if (k == "z_blocks") *v = c->z_blocks;
    else if (k == "host_huge") *v = c->host_huge;
    else if (k == "serve_frames") *v = c->serve_frames_param;
    else if (k == "batch_sparse_below") *v = c->batch_sparse_below;
    else return fail(c, HYTG_ERR_ARG, "unknown parameter " + k);
    return HYTG_OK;
}

hytg_status hytg_run(hytg_ctx *c, hytg_algo algo_in, const uint32_t *sources, uint32_t n_sources) {
    if (!c) return HYTG_ERR_ARG;
    const int algo = (int)algo_in;
    if (algo < 0 || algo > 4) return fail(c, HYTG_ERR_ARG, "unknown algorithm");
    if (!c->loaded) return fail(c, HYTG_ERR_STATE, "no graph loaded");
    if (!c->d_pool) return fail(c, HYTG_ERR_STATE, "no device budget set");
    if (c->serving) return fail(c, HYTG_ERR_STATE, "serving in progress (hytg_serve_end first)");
    const bool needs_src = (algo == kBFS || algo == kSSSP || algo == kPPR);
    uint32_t source = 0;
    uint32_t src_int[64] = {0};
    int bmode = kBatchNone;
    if (needs_src) {
        const uint32_t max_src = algo == kPPR ? 32u : 64u;
        if (!sources || n_sources < 1 || n_sources > max_src)
            return fail(c, HYTG_ERR_ARG, "BFS/SSSP take 1..64 sources, PPR 1..32 seeds");
        for (uint32_t i = 0; i < n_sources; ++i) {
            if (sources[i] >= c->V) return fail(c, HYTG_ERR_ARG, "source out of range");
            src_int[i] = c->permuted ? c->h_inv[sources[i]] : sources[i];
        }
        source = src_int[0];
        if (n_sources > 1) bmode = algo == kBFS ? kBatchBFS : algo == kSSSP ? kBatchSSSP : kBatchPPR;
    } else {
        n_sources = 1;
    }
    if (algo == kSSSP && !c->weighted) return fail(c, HYTG_ERR_ARG, "SSSP needs edge weights");
    try {
        if (algo == kCC) {
            // checked once per loaded graph, on the internal arrays (hub
            // sorting relabels vertices, which keeps symmetry)
            if (c->symmetric < 0) c->symmetric = csr_symmetric(c->h_off, c->h_dst, c->V) ? 1 : 0;
            if (!c->symmetric)
                return fail(c, HYTG_ERR_ARG,
                            "CC needs a symmetric CSR (every edge u->v with a reverse v->u of the same "
                            "multiplicity); symmetrise the graph first");
        }
        CK(cudaSetDevice(c->device));
        CK(ahead_drop(c));
        const auto t_start = std::chrono::steady_clock::now();
        c->has_deadline = c->run_timeout_ms > 0;
        if (c->has_deadline)
            c->run_deadline = t_start + std::chrono::microseconds((long long)(c->run_timeout_ms * 1000.0));
        *(volatile unsigned int *)c->h_cancel = 0u;
        c->have_result = false;
        c->stats = hytg_stats{};
        c->iters.clear();
        c->timed.clear();
        c->iter_ev.clear();
        c->ev_used = 0;
        c->batch_mode = kBatchNone;
        c->batch_K = 1;
        if (bmode != kBatchNone) {
            hytg_status bsx = ensure_batch(c, bmode, n_sources);
            if (bsx == HYTG_OK) bsx = attach_own_frames(c, bmode, n_sources);
            if (bsx != HYTG_OK) return bsx;
            c->batch_mode = bmode;
            c->batch_K = n_sources;
        }
        const int n_arrays = (algo == kSSSP) ? 2 : 1;
        c->last_run_arrays = n_arrays;
        CK(cudaEventRecord(c->ev_run[0], c->s_main));
        hytg_status s = plan_carve(c, n_arrays);
        if (s != HYTG_OK) return s;
        s = ensure_cache(c, n_arrays);
        if (s != HYTG_OK) return s;
        // delta-stepping bucket (SSSP only): eligible vertices have dist < bucket
        uint64_t delta = 0;
        if (algo == kSSSP && c->batch_mode == kBatchNone)
            delta = c->sssp_delta < 0 ? c->auto_delta : (uint64_t)c->sssp_delta;
        unsigned int bucket = delta ? (unsigned int)std::min<uint64_t>(delta, 0xFFFFFFFEull) : 0xFFFFFFFFu;
        CK(cudaMemsetAsync(c->d_err, 0, 4, c->s_main));
        CK(cudaMemsetAsync(c->d_sp, 0, kSpSlots * 8, c->s_main));
        CK(cudaMemsetAsync(c->d_link_ctr, 0, 2 * kRoutes * 8, c->s_main));
        c->sp_launches = 0;
        c->timeline.clear();
        if ((algo == kPR || algo == kPPR) && c->d_hub_rep && c->batch_mode == kBatchNone)
            CK(cudaMemsetAsync(c->d_hub_rep, 0, (size_t)kHubReplicas * c->n_hub_rep * 4, c->s_main));
        {
            AlgoState st = algo_state(c, algo);
            ScopedTime t(c, HYTG_K_INIT, c->s_main);
            if (c->batch_mode != kBatchNone) {
                CK(cudaMemcpyAsync(c->d_src, src_int, sizeof(src_int), cudaMemcpyHostToDevice, c->s_main));
                CK(cudaMemsetAsync(c->d_src_work, 0, 8, c->s_main));
                CK(cudaMemsetAsync(c->d_overflow, 0, 4, c->s_main));
                for (uint32_t g = 0; g * kFrameSources < c->batch_K; ++g)
                    CK(launch_frame_init(c->bs, c->V, g, c->s_main));
                CK(launch_b_init(c->bs, c->V, c->n_words_alloc, c->d_src, c->batch_K,
                                 ppr_seed_mass(c), st.bm_cur, c->s_main));
            } else {
                CK(launch_init(st, c->V, c->n_words_alloc, source, c->s_main));
            }
        }
        uint32_t it = 0;
        const bool use_loop = loop_applies(c);
        s = issue_plan(c, algo, bucket, it, 0, true);
        if (s != HYTG_OK) return s;
        for (;;) {
            const int buf = it & 1;
            CK(cudaEventSynchronize(c->ev_sum[buf]));
            const char *hb = (const char *)c->h_sumbuf[buf];
            const Summary *hs = (const Summary *)hb;
            if (hs->n_active != 0 && past_deadline(c)) return run_timed_out(c, it);
            if (hs->n_active == 0) {
                if (hs->pending == 0) break;
                // the current bucket is settled: open the next one at the
                // smallest pending distance (delta-stepping)
                const uint64_t nb = std::max<uint64_t>((uint64_t)bucket, hs->pending_min) + delta;
                bucket = (unsigned int)std::min<uint64_t>(nb, 0xFFFFFFFEull);
                if (hs->pending_min >= 0xFFFFFFFEull) bucket = 0xFFFFFFFFu;
                ++it;
                s = issue_plan(c, algo, bucket, it, it & 1, it < (uint32_t)c->max_iters);
                if (s != HYTG_OK) return s;
                continue;
            }
            if (it >= (uint32_t)c->max_iters) { c->stats.status = HYTG_OK; break; }
            s = issue_work(c, algo, bucket, hb, n_arrays);
            if (s != HYTG_OK) return s;
            // --- next iteration
            ++it;
            // In PageRank's dense phase an iteration with F or C work is
            // followed by another, so unless the graph holds F and C nodes
            // the host plans it at once: entering the device loop would only
            // plan it there, return, and put a host round trip between the
            // iterations.  After a cache/Z-only iteration the device loop
            // takes over.  (BFS, SSSP and CC have short F phases; their next
            // iteration is often cache/Z only and runs best in the graph.)
            const bool plan_on_host = (algo == kPR || algo == kPPR) && c->last_fc && c->loop_after_fc == 0 &&
                                      !loop_fc_wanted(c);
            if (use_loop && !c->loop_unavailable && !plan_on_host) {
                // captured after iteration 0 has run, so every launcher's
                // one-time set-up happened outside the capture; a CUDA driver that
                // cannot build the graph leaves this context on the host loop
                if (ensure_loop_graph_fc(c, algo) != HYTG_OK) {
                    c->loop_unavailable = true;
                    c->loop_error = c->err;
                    cudaGetLastError();
                }
            }
            if (use_loop && !c->loop_unavailable && !plan_on_host) {
                // iterations on the device until one needs the F or C route
                int status = 0;
                s = run_device_loop(c, it, bucket, delta, status);
                if (s != HYTG_OK) return s;
                if (status == kLoopCancel) return run_timed_out(c, it);
                if (status != kLoopHost) break;       // converged or at the cap
                const int nb = it & 1;
                iteration_mark(c);
                CK(cudaMemcpyAsync(c->h_sumbuf[nb], c->d_sumbuf, c->sum_host_bytes, cudaMemcpyDeviceToHost,
                                   c->s_main));
                CK(cudaEventRecord(c->ev_sum[nb], c->s_main));
                s = issue_plan_tail(c, algo, bucket, c->s_main, nullptr);
                if (s != HYTG_OK) return s;
                continue;
            }
            // at the cap only the plan runs (the loop then stops on it)
            s = issue_plan(c, algo, bucket, it, it & 1, it < (uint32_t)c->max_iters);
            if (s != HYTG_OK) return s;
        }
        c->stats.iterations = it;
        CK(ahead_join(c));
        // finalisation
        {
            AlgoState st = algo_state(c, algo);
            ScopedTime t(c, HYTG_K_FINAL, c->s_main);
            if (c->batch_mode != kBatchNone)
                CK(launch_b_finalize(c->bs, c->V, c->batch_K, c->d_perm, c->d_bout, c->d_bsums, c->s_main));
            else if (algo == kPR || algo == kPPR)
                CK(launch_pr_finalize(st, c->V, c->d_out, c->d_prsums, c->s_main));
            else if (algo == kCC)
                CK(launch_cc_final(st, c->V, c->d_pay, (unsigned int *)c->d_out, c->s_main));
            else
                CK(launch_to_original(st.perm, c->d_val, c->d_out, c->V, c->s_main));
        }
        unsigned int ovf = 0, ierr = 0;
        double prs[2] = {0, 0};
        CK(cudaMemcpyAsync(&ovf, c->d_overflow, 4, cudaMemcpyDeviceToHost, c->s_main));
        CK(cudaMemcpyAsync(&ierr, c->d_err, 4, cudaMemcpyDeviceToHost, c->s_main));
        if ((algo == kPR || algo == kPPR) && c->batch_mode == kBatchNone)
            CK(cudaMemcpyAsync(prs, c->d_prsums, 16, cudaMemcpyDeviceToHost, c->s_main));
        unsigned long long swork = 0, extra = 0;
        const uint32_t n_sp = std::min<uint32_t>(c->sp_launches + 1, kSpSlots);
        std::vector<unsigned long long> sp(n_sp, 0);
        unsigned long long lctr[2 * kRoutes] = {};
        CK(cudaMemcpyAsync(sp.data(), c->d_sp, n_sp * 8, cudaMemcpyDeviceToHost, c->s_main));
        CK(cudaMemcpyAsync(lctr, c->d_link_ctr, sizeof lctr, cudaMemcpyDeviceToHost, c->s_main));
        if (c->batch_mode != kBatchNone)
            CK(cudaMemcpyAsync(&swork, c->d_src_work, 8, cudaMemcpyDeviceToHost, c->s_main));
        CK(cudaEventRecord(c->ev_run[1], c->s_main));
        CK(cudaStreamSynchronize(c->s_main));
        CK(cudaGetLastError());
        const auto t_end = std::chrono::steady_clock::now();
        {
            float dms = 0;
            CK(cudaEventElapsedTime(&dms, c->ev_run[0], c->ev_run[1]));
            c->stats.device_ms = dms;
        }
        c->stats.wall_ms = std::chrono::duration<double, std::milli>(t_end - t_start).count();
        c->stats.pr_rank_sum = prs[0];
        c->stats.pr_residual_sum = prs[1];
        c->stats.n_sources = c->batch_K;
        for (unsigned long long x : sp) extra += x;
        c->stats.extra_edges = extra;
        for (int r = 0; r < kRoutes; ++r) {
            c->stats.link_sector_bytes[r] = lctr[2 * r] * 32ull;
            c->stats.link_line_bytes[r] = lctr[2 * r + 1] * 128ull;
        }
        // explicit copies move exactly their bytes (F; C compacted on the host)
        c->stats.link_sector_bytes[kRouteF] = c->stats.link_line_bytes[kRouteF] = c->stats.link_bytes[kRouteF];
        if (c->compact_host > 0)
            c->stats.link_sector_bytes[kRouteC] = c->stats.link_line_bytes[kRouteC] = c->stats.link_bytes[kRouteC];
        c->stats.source_edges = c->batch_mode != kBatchNone ? swork : c->stats.edges_relaxed;
        for (size_t i = 0; i + 1 < c->iter_ev.size(); ++i) {
            // host-issued iterations only: a mark and the next iteration's mark
            const size_t k = c->iter_ev[i].first;
            float ms = 0;
            if (k < c->iters.size() && c->iter_ev[i + 1].first == k + 1 &&
                cudaEventElapsedTime(&ms, c->iter_ev[i].second, c->iter_ev[i + 1].second) == cudaSuccess)
                c->iters[k].device_ms = ms;
        }
        {
            // busy time of each kernel kind and of each route's transfers:
            // the union of their intervals (relative to the run's start
            // event) over all streams
            constexpr int kKinds = kKindSecondPass + 1;
            std::vector<std::pair<float, float>> iv[kKinds];
            for (auto &tl : c->timed) {
                float t0 = 0, t1 = 0;
                if (tl.kind < 0 || tl.kind >= kKinds ||
                    cudaEventElapsedTime(&t0, c->ev_run[0], tl.a) != cudaSuccess ||
                    cudaEventElapsedTime(&t1, c->ev_run[0], tl.b) != cudaSuccess)
                    continue;
                iv[tl.kind].push_back({t0, t1});
            }
            double busy_of[kKinds] = {};
            for (int k = 0; k < kKinds; ++k) {
                std::sort(iv[k].begin(), iv[k].end());
                double busy = 0, lo = 0, hi = -1;
                for (auto &p : iv[k]) {
                    if (p.first > hi) {
                        if (hi > lo) busy += hi - lo;
                        lo = p.first;
                        hi = p.second;
                    } else if (p.second > hi) {
                        hi = p.second;
                    }
                }
                if (hi > lo) busy += hi - lo;
                busy_of[k] = busy;
                c->stats.kernel_busy_ms[k] = busy;
            }
            c->stats.route_busy_ms[kRouteF] = busy_of[HYTG_K_COPY_F];
            c->stats.route_busy_ms[kRouteC] = busy_of[HYTG_K_GATHER_C];
            c->stats.route_busy_ms[kRouteZ] = busy_of[HYTG_K_RELAX_Z];
        }
        c->timeline.reserve(c->timed.size());
        for (auto &tl : c->timed) {
            float t0 = 0, t1 = 0;
            if (cudaEventElapsedTime(&t0, c->ev_run[0], tl.a) != cudaSuccess ||
                cudaEventElapsedTime(&t1, c->ev_run[0], tl.b) != cudaSuccess)
                continue;
            hytg_timed_launch r{};
            r.kind = (uint32_t)tl.kind;
            r.stream = (uint32_t)tl.stream;
            r.start_ms = t0;
            r.end_ms = t1;
            r.bytes = tl.bytes;
            r.edges = tl.edges;
            r.vertices = tl.vertices;
            r.part_first = tl.part_first;
            r.part_last = tl.part_last;
            if (tl.sp_slot >= 0)
                r.edges = (uint32_t)tl.sp_slot < kSpSlots - 1 && (size_t)tl.sp_slot < sp.size() ? sp[tl.sp_slot]
                                                                                            : UINT64_MAX;
            c->timeline.push_back(r);
        }
        for (auto &tl : c->timed) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, tl.a, tl.b) == cudaSuccess) {
                if (tl.kind == kKindSecondPass) {
                    c->stats.second_pass_ms += ms;
                    c->stats.second_pass_count += 1;
                } else {
                    c->stats.kernel_ms[tl.kind] += ms;
                    c->stats.kernel_count[tl.kind] += 1;
                }
            }
        }
        cudaGetLastError();
        c->last_algo = algo;
        if (ierr) {
            c->stats.status = HYTG_ERR_CUDA;
            return fail(c, HYTG_ERR_CUDA, "internal index check failed (flags " + std::to_string(ierr) + ")");
        }
        if (ovf) {
            c->stats.status = HYTG_ERR_OVERFLOW;
            return fail(c, HYTG_ERR_OVERFLOW, "an SSSP distance does not fit in 32 bits");
        }
        c->have_result = true;
        c->stats.status = HYTG_OK;
        return HYTG_OK;
    } catch (...) {
        return fail(c, HYTG_ERR_HOSTMEM, "host allocation failed during the run");
    }
}

hytg_status hytg_serve_begin(hytg_ctx *c, hytg_algo algo_in, uint32_t n_slots) {
    if (!c) return HYTG_ERR_ARG;
    const int algo = (int)algo_in;
    if (algo != kBFS && algo != kSSSP && algo != kPPR)
        return fail(c, HYTG_ERR_ARG, "serving supports BFS, SSSP and PPR");
    if (n_slots < 1 || n_slots > (algo == kPPR ? 32u : 64u))
        return fail(c, HYTG_ERR_ARG, "BFS/SSSP serve 1..64 slots, PPR 1..32");
    if (!c->loaded) return fail(c, HYTG_ERR_STATE, "no graph loaded");
    if (!c->d_pool) return fail(c, HYTG_ERR_STATE, "no device budget set");
    if (algo == kSSSP && !c->weighted) return fail(c, HYTG_ERR_ARG, "SSSP needs edge weights");
    CK(cudaSetDevice(c->device));
    CK(ahead_drop(c));
    const int mode = algo == kBFS ? kBatchBFS : algo == kSSSP ? kBatchSSSP : kBatchPPR;
    hytg_status s = ensure_batch(c, mode, 1);
    if (s != HYTG_OK) return s;
    c->batch_mode = mode;
    c->batch_K = n_slots;
    c->have_result = false;
    c->stats = hytg_stats{};
    c->iters.clear();
    c->timed.clear();
    c->iter_ev.clear();
    c->ev_used = 0;
    const int n_arrays = algo == kSSSP ? 2 : 1;
    // The budget holds the edge-side carve and the queries' frames (8 queries
    // each): as many frames as the slots can use (at most "serve_frames"),
    // fewer if the budget cannot hold them beside the smallest edge carve.
    const uint64_t fb = frame_bytes(c, mode);
    const uint64_t pool_bytes = c->budget + kPoolSlack;
    uint32_t nf = (n_slots + kFrameSources - 1) / kFrameSources;
    if (c->serve_frames_param > 0) nf = std::min<uint32_t>(nf, (uint32_t)c->serve_frames_param);
    std::string why = "the budget is smaller than one frame";
    for (; nf >= 1; --nf) {
        if ((uint64_t)nf * fb + kPoolSlack >= c->budget) continue;
        const uint64_t eb = c->budget - (uint64_t)nf * fb - kPoolSlack;
        if (plan_carve(c, n_arrays, eb) != HYTG_OK) {
            why = c->err;
            continue;
        }
        const uint64_t base = (c->carve.end + 255) & ~uint64_t(255);
        if (base + (uint64_t)nf * fb > pool_bytes) continue;
        c->serve_frame_base = (char *)c->d_pool + base;
        c->serve_edge_budget = eb;
        break;
    }
    if (nf == 0) {
        c->batch_mode = kBatchNone;
        c->carve = Carve();
        return fail(c, HYTG_ERR_BUDGET, "the device budget holds no query frame (" + std::to_string(fb) +
                                            " B for 8 queries) beside the smallest edge-side carve; with one "
                                            "frame: " + why);
    }
    c->serve_frames = nf;
    c->serve_frame_bytes = fb;
    c->serve_frames_used = 0;
    for (auto &f : c->serve_group_frame) f = -1;
    s = ensure_cache(c, n_arrays);
    if (s != HYTG_OK) return s;
    CK(cudaMemsetAsync(c->d_err, 0, 4, c->s_main));
    CK(cudaMemsetAsync(c->d_overflow, 0, 4, c->s_main));
    CK(cudaMemsetAsync(c->d_src_work, 0, 8, c->s_main));
    CK(launch_b_init(c->bs, c->V, c->n_words_alloc, c->d_src, 0, 0.0f, c->d_bm[0], c->s_main));
    c->serving = true;
    c->serve_algo = algo;
    c->serve_it = 0;
    c->serve_busy = 0;
    c->serve_alive = 0;
    return HYTG_OK;
}

hytg_status hytg_serve_admit(hytg_ctx *c, uint32_t slot, uint32_t source) {
    if (!c) return HYTG_ERR_ARG;
    if (!c->serving) return fail(c, HYTG_ERR_STATE, "not serving");
    if (slot >= c->batch_K) return fail(c, HYTG_ERR_ARG, "slot out of range");
    if (c->serve_busy & (1ull << slot)) return fail(c, HYTG_ERR_STATE, "slot is busy");
    if (source >= c->V) return fail(c, HYTG_ERR_ARG, "source out of range");
    CK(cudaSetDevice(c->device));
    const uint32_t g = slot / kFrameSources;
    if (c->serve_group_frame[g] < 0) {
        // the slot's group of 8 needs a frame of device memory for its state
        int f = -1;
        for (uint32_t i = 0; i < c->serve_frames && f < 0; ++i)
            if (!((c->serve_frames_used >> i) & 1u)) f = (int)i;
        if (f < 0)
            return fail(c, HYTG_ERR_BUDGET, "no device memory free for the query's state: every frame of "
                                            "the budget is in use (admit it when a query finishes)");
        c->serve_frames_used |= 1u << f;
        c->serve_group_frame[g] = f;
        set_group_frame(c, g, c->serve_frame_base + (uint64_t)f * c->serve_frame_bytes);
        CK(launch_frame_init(c->bs, c->V, g, c->s_main));
    }
    const uint32_t src = c->permuted ? c->h_inv[source] : source;
    CK(launch_serve_admit(c->bs, c->V, slot, src, ppr_seed_mass(c), c->d_bm[0], c->s_main));
    c->serve_busy |= 1ull << slot;
    c->serve_admit_it[slot] = c->serve_it;
    return HYTG_OK;
}

hytg_status hytg_serve_step(hytg_ctx *c, uint64_t *finished, uint64_t *busy) {
    if (!c) return HYTG_ERR_ARG;
    if (!c->serving) return fail(c, HYTG_ERR_STATE, "not serving");
    CK(cudaSetDevice(c->device));
    try {
        const int algo = c->serve_algo;
        const int n_arrays = algo == kSSSP ? 2 : 1;
        const uint32_t it = c->serve_it;
        hytg_status s = issue_plan(c, algo, 0xFFFFFFFFu, it, it & 1, true);
        if (s != HYTG_OK) return s;
        CK(cudaEventSynchronize(c->ev_sum[it & 1]));
        const char *hb = (const char *)c->h_sumbuf[it & 1];
        const Summary *hs = (const Summary *)hb;
        c->serve_alive = hs->alive;
        if (hs->n_active > 0) {
            s = issue_work(c, algo, 0xFFFFFFFFu, hb, n_arrays);
            if (s != HYTG_OK) return s;
        }
        c->serve_it = it + 1;
        c->stats.iterations = c->serve_it;
        if (finished) *finished = c->serve_busy & ~c->serve_alive;
        if (busy) *busy = c->serve_busy;
        return HYTG_OK;
    } catch (...) {
        return fail(c, HYTG_ERR_HOSTMEM, "host allocation failed");
    }
}

hytg_status hytg_serve_fetch(hytg_ctx *c, uint32_t slot, void *out, uint64_t out_bytes) {
    if (!c || !out) return HYTG_ERR_ARG;
    if (!c->serving) return fail(c, HYTG_ERR_STATE, "not serving");
    if (slot >= c->batch_K) return fail(c, HYTG_ERR_ARG, "slot out of range");
    const uint64_t bit = 1ull << slot;
    if (!(c->serve_busy & bit) || (c->serve_alive & bit))
        return fail(c, HYTG_ERR_STATE, "slot has no finished query");
    if (out_bytes < c->V * 4) return fail(c, HYTG_ERR_ARG, "output buffer too small");
    CK(cudaSetDevice(c->device));
    CK(launch_serve_extract(c->bs, c->V, slot, c->d_perm, c->serve_admit_it[slot], c->d_bout,
                            c->d_bsums, c->s_main));
    CK(cudaMemcpyAsync(out, c->d_bout, c->V * 4, cudaMemcpyDeviceToHost, c->s_main));
    unsigned int ovf = 0, ierr = 0;
    CK(cudaMemcpyAsync(&ovf, c->d_overflow, 4, cudaMemcpyDeviceToHost, c->s_main));
    CK(cudaMemcpyAsync(&ierr, c->d_err, 4, cudaMemcpyDeviceToHost, c->s_main));
    CK(cudaStreamSynchronize(c->s_main));
    c->serve_busy &= ~bit;
    release_idle_frame(c, slot / kFrameSources);
    if (ierr) return fail(c, HYTG_ERR_CUDA, "internal index check failed");
    if (ovf) return fail(c, HYTG_ERR_OVERFLOW, "an SSSP distance does not fit in 32 bits");
    return HYTG_OK;
}

hytg_status hytg_serve_end(hytg_ctx *c) {
    if (!c) return HYTG_ERR_ARG;
    if (!c->serving) return fail(c, HYTG_ERR_STATE, "not serving");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->s_main));
    c->serving = false;
    c->serve_busy = 0;
    for (uint32_t g = 0; g < kMaxFrames; ++g) release_idle_frame(c, g);
    c->batch_mode = kBatchNone;
    return HYTG_OK;
}

hytg_status hytg_serve_get_info(hytg_ctx *c, hytg_serve_info *out) {
    if (!c || !out) return HYTG_ERR_ARG;
    if (!c->serving) return fail(c, HYTG_ERR_STATE, "not serving");
    hytg_serve_info i{};
    i.frames = c->serve_frames;
    i.frames_free = c->serve_frames - (uint32_t)__builtin_popcount(c->serve_frames_used);
    i.slots_per_frame = kFrameSources;
    i.frame_bytes = c->serve_frame_bytes;
    i.edge_budget_bytes = c->serve_edge_budget;
    i.busy_slots = c->serve_busy;
    *out = i;
    return HYTG_OK;
}

hytg_status hytg_fetch_result(hytg_ctx *c, void *out, uint64_t out_bytes) {
    if (!c || !out) return HYTG_ERR_ARG;
    if (!c->have_result) return fail(c, HYTG_ERR_STATE, "no completed run");
    const uint64_t need = c->V * 4 * (c->batch_mode != kBatchNone ? c->batch_K : 1);
    if (out_bytes < need) return fail(c, HYTG_ERR_ARG, "output buffer too small");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(out, c->batch_mode != kBatchNone ? c->d_bout : (void *)c->d_out, need,
                       cudaMemcpyDeviceToHost, c->s_main));
    CK(cudaStreamSynchronize(c->s_main));
    return HYTG_OK;
}

hytg_status hytg_fetch_pagerank_state(hytg_ctx *c, float *rank, float *delta, uint64_t V) {
    if (!c) return HYTG_ERR_ARG;
    if (!c->have_result || !(c->last_algo == kPR || c->last_algo == kPPR) || c->batch_mode != kBatchNone)
        return fail(c, HYTG_ERR_STATE, "no completed single-source PageRank run");
    if (V < c->V) return fail(c, HYTG_ERR_ARG, "buffers too small");
    CK(cudaSetDevice(c->device));
    // original vertex order; d_out (the normalised result) is rebuilt afterwards
    if (rank) {
        CK(launch_to_original(c->d_perm, c->d_val, c->d_out, c->V, c->s_main));
        CK(cudaMemcpyAsync(rank, c->d_out, c->V * 4, cudaMemcpyDeviceToHost, c->s_main));
    }
    if (delta) {
        CK(launch_to_original(c->d_perm, (const unsigned int *)c->d_delta, c->d_out, c->V, c->s_main));
        CK(cudaMemcpyAsync(delta, c->d_out, c->V * 4, cudaMemcpyDeviceToHost, c->s_main));
    }
    {
        AlgoState st = algo_state(c, c->last_algo);
        CK(launch_pr_finalize(st, c->V, c->d_out, c->d_prsums, c->s_main));
    }
    CK(cudaStreamSynchronize(c->s_main));
    return HYTG_OK;
}

hytg_status hytg_get_stats(hytg_ctx *c, hytg_stats *out) {
    if (!c || !out) return HYTG_ERR_ARG;
    *out = c->stats;
    return HYTG_OK;
}

hytg_status hytg_get_info(hytg_ctx *c, hytg_info *out) {
    if (!c || !out) return HYTG_ERR_ARG;
    hytg_info i{};
    i.V = c->V;
    i.E = c->E;
    i.weighted = c->weighted;
    i.n_parts = c->loaded ? (uint32_t)(c->part_vb.size() - 1) : 0;
    i.part_edges = c->part_edges;
    i.slot_edges = c->carve.slot_edges;
    i.n_slots = c->carve.n_slots;
    i.n_cached = c->carve.n_cached;
    i.budget_bytes = c->budget;
    i.budget_used_bytes = c->carve.used;
    i.compact_edges = c->carve.compact_edges;
    i.vertex_state_bytes = c->loaded ? c->vertex_bytes : 0;
    i.pinned_host_bytes = c->loaded ? std::max<uint64_t>(c->E, 1) * 4 * (c->weighted ? 2 : 1) : 0;
    *out = i;
    return HYTG_OK;
}

hytg_status hytg_get_partitions(hytg_ctx *c, uint64_t *vb, uint32_t cap, uint32_t *n_parts) {
    if (!c || !n_parts) return HYTG_ERR_ARG;
    if (!c->loaded) return fail(c, HYTG_ERR_STATE, "no graph loaded");
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    *n_parts = N;
    if (vb) {
        if (cap < N + 1) return fail(c, HYTG_ERR_ARG, "vbounds too small");
        std::copy(c->part_vb.begin(), c->part_vb.end(), vb);
    }
    return HYTG_OK;
}

hytg_status hytg_plan(hytg_ctx *c, hytg_algo algo_in, const uint8_t *active, uint8_t *routes,
                      uint64_t *counts, uint32_t cap) {
    if (!c || !active || !routes) return HYTG_ERR_ARG;
    const int algo = (int)algo_in;
    if (algo < 0 || algo > 4) return fail(c, HYTG_ERR_ARG, "unknown algorithm");
    if (!c->loaded) return fail(c, HYTG_ERR_STATE, "no graph loaded");
    if (!c->d_pool) return fail(c, HYTG_ERR_STATE, "no device budget set");
    const uint32_t N = (uint32_t)(c->part_vb.size() - 1);
    if (cap < N) return fail(c, HYTG_ERR_ARG, "output arrays too small");
    CK(cudaSetDevice(c->device));
    hytg_status s = plan_carve(c, algo == kSSSP ? 2 : 1);
    if (s != HYTG_OK) return s;
    std::vector<uint8_t> act_int;
    if (c->permuted) {
        act_int.resize(c->V);
        for (uint64_t n = 0; n < c->V; ++n) act_int[n] = active[c->h_perm[n]];
        active = act_int.data();
    }
    unsigned char *d_act = nullptr;
    CK(cudaMalloc(&d_act, c->V));
    cudaError_t e = cudaMemcpy(d_act, active, c->V, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_upload_bitmap(d_act, c->d_bm[0], c->V, c->n_words_alloc, c->s_main);
    if (e != cudaSuccess) { cudaFree(d_act); return fail(c, HYTG_ERR_CUDA, cudaGetErrorString(e)); }
    c->have_result = false;
    s = issue_plan(c, algo, 0xFFFFFFFFu, 0, 0, false);
    cudaStreamSynchronize(c->s_main);
    cudaFree(d_act);
    if (s != HYTG_OK) return s;
    CK(cudaGetLastError());
    const SumLayout L = sum_layout(N);
    const char *hb = (const char *)c->h_sumbuf[0];
    memcpy(routes, hb + L.route, N);
    if (counts) {
        const unsigned long long *na = (const unsigned long long *)(hb + L.n_act);
        const unsigned long long *ed = (const unsigned long long *)(hb + L.edges);
        const unsigned long long *ln = (const unsigned long long *)(hb + L.lines);
        for (uint32_t p = 0; p < N; ++p) {
            counts[3 * p] = na[p];
            counts[3 * p + 1] = ed[p];
            counts[3 * p + 2] = ln[p];
        }
    }
    CK(cudaMemset(c->d_bm[0], 0, c->n_words_alloc * 4));
    return HYTG_OK;
}

hytg_status hytg_probe_link(hytg_ctx *c, uint64_t bytes, uint32_t reps, double *memcpy_gbs,
                            double *zerocopy_gbs) {
    if (!c || bytes < 4096 || reps == 0) return HYTG_ERR_ARG;
    CK(cudaSetDevice(c->device));
    bytes &= ~uint64_t(511);
    void *h = nullptr, *d = nullptr;
    unsigned long long *sink = nullptr;
    if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HYTG_ERR_HOSTMEM, "probe pinned allocation failed");
    }
    memset(h, 1, bytes);
    cudaEvent_t a, b;
    hytg_status st = HYTG_OK;
    auto run = [&]() -> hytg_status {
        CK(cudaMalloc(&d, bytes));
        CK(cudaMalloc(&sink, 8));
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        void *mp = nullptr;
        CK(cudaHostGetDevicePointer(&mp, h, 0));
        float best = 1e30f;
        for (uint32_t r = 0; r < reps + 1; ++r) {
            CK(cudaEventRecord(a, c->s_main));
            CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->s_main));
            CK(cudaEventRecord(b, c->s_main));
            CK(cudaEventSynchronize(b));
            float ms;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (r > 0) best = std::min(best, ms);
        }
        if (memcpy_gbs) *memcpy_gbs = bytes / (best * 1e-3) / 1e9;
        best = 1e30f;
        for (uint32_t r = 0; r < reps + 1; ++r) {
            CK(cudaEventRecord(a, c->s_main));
            CK(launch_zc_probe((const uint4 *)mp, bytes / 16, sink, 8 * (int)device_sms(), c->s_main));
            CK(cudaEventRecord(b, c->s_main));
            CK(cudaEventSynchronize(b));
            float ms;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (r > 0) best = std::min(best, ms);
        }
        if (zerocopy_gbs) *zerocopy_gbs = bytes / (best * 1e-3) / 1e9;
        return HYTG_OK;
    };
    st = run();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (d) cudaFree(d);
    if (sink) cudaFree(sink);
    cudaFreeHost(h);
    return st;
}

hytg_status hytg_probe_atomics(hytg_ctx *c, uint64_t n, uint32_t reps, double *uniform_gops,
                               double *skewed_gops) {
    if (!c || n < 1024 || n > (1ull << 30) || reps == 0) return HYTG_ERR_ARG;
    CK(cudaSetDevice(c->device));
    unsigned int *idx = nullptr;
    float *d = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto run = [&]() -> hytg_status {
        CK(cudaMalloc(&idx, n * 4));
        CK(cudaMalloc(&d, (1ull << 24) * 4));
        CK(cudaMemset(d, 0, (1ull << 24) * 4));
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        for (int skew = 0; skew < 2; ++skew) {
            CK(launch_red_probe(idx, d, n, skew, true, c->s_main));
            float best = 1e30f;
            for (uint32_t r = 0; r < reps + 1; ++r) {
                CK(cudaEventRecord(a, c->s_main));
                CK(launch_red_probe(idx, d, n, skew, false, c->s_main));
                CK(cudaEventRecord(b, c->s_main));
                CK(cudaEventSynchronize(b));
                float ms;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (r > 0) best = std::min(best, ms);
            }
            double *out = skew ? skewed_gops : uniform_gops;
            if (out) *out = n / (best * 1e-3) / 1e9;
        }
        return HYTG_OK;
    };
    hytg_status st = run();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (idx) cudaFree(idx);
    if (d) cudaFree(d);
    return st;
}

hytg_status hytg_probe_atomics_hub(hytg_ctx *c, uint64_t n, uint32_t reps, uint32_t n_rep,
                                   double *plain_gops, double *replica_gops) {
    if (!c || n < 1024 || n > (1ull << 30) || reps == 0 || n_rep > (1u << 20)) return HYTG_ERR_ARG;
    CK(cudaSetDevice(c->device));
    unsigned int *idx = nullptr;
    float *d = nullptr, *rp = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto run = [&]() -> hytg_status {
        CK(cudaMalloc(&idx, n * 4));
        CK(cudaMalloc(&d, (1ull << 24) * 4));
        CK(cudaMemset(d, 0, (1ull << 24) * 4));
        if (n_rep) {
            CK(cudaMalloc(&rp, (size_t)kHubReplicas * n_rep * 4));
            CK(cudaMemset(rp, 0, (size_t)kHubReplicas * n_rep * 4));
        }
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(launch_red_probe(idx, d, n, 2, true, c->s_main));
        for (int with_rep = 0; with_rep < 2; ++with_rep) {
            float best = 1e30f;
            for (uint32_t r = 0; r < reps + 1; ++r) {
                CK(cudaEventRecord(a, c->s_main));
                CK(launch_red_probe(idx, d, n, 2, false, c->s_main, with_rep ? rp : nullptr,
                                    with_rep ? n_rep : 0));
                CK(cudaEventRecord(b, c->s_main));
                CK(cudaEventSynchronize(b));
                float ms;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (r > 0) best = std::min(best, ms);
            }
            double *out = with_rep ? replica_gops : plain_gops;
            if (out) *out = n / (best * 1e-3) / 1e9;
        }
        return HYTG_OK;
    };
    hytg_status st = run();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (idx) cudaFree(idx);
    if (d) cudaFree(d);
    if (rp) cudaFree(rp);
    return st;
}

hytg_status hytg_probe_frame_push(hytg_ctx *c, uint64_t n, uint32_t reps, uint32_t width, double *frame_gops) {
    if (!c || !frame_gops || n < 1024 || n > (1ull << 30) || reps == 0 || (width != 1 && width != 2 && width != 4))
        return HYTG_ERR_ARG;
    CK(cudaSetDevice(c->device));
    constexpr unsigned long long kVerts = 1ull << 24;
    unsigned int *idx = nullptr;
    float *d = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto run = [&]() -> hytg_status {
        CK(cudaMalloc(&idx, n * 4));
        CK(cudaMalloc(&d, kVerts * 8 * 4));
        CK(cudaMemset(d, 0, kVerts * 8 * 4));
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(launch_red_probe(idx, d, n, 0, true, c->s_main));        // uniform ids in [0, 2^24)
        float best = 1e30f;
        for (uint32_t r = 0; r < reps + 1; ++r) {
            CK(cudaEventRecord(a, c->s_main));
            CK(launch_frame_probe(idx, d, n, (int)width, c->s_main));
            CK(cudaEventRecord(b, c->s_main));
            CK(cudaEventSynchronize(b));
            float ms;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (r > 0) best = std::min(best, ms);
        }
        *frame_gops = n / (best * 1e-3) / 1e9;
        return HYTG_OK;
    };
    hytg_status st = run();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (idx) cudaFree(idx);
    if (d) cudaFree(d);
    return st;
}

hytg_status hytg_get_permutation(hytg_ctx *c, uint32_t *perm, uint64_t V) {
    if (!c || !perm) return HYTG_ERR_ARG;
    if (!c->loaded) return fail(c, HYTG_ERR_STATE, "no graph loaded");
    if (V < c->V) return fail(c, HYTG_ERR_ARG, "buffer too small");
    for (uint64_t n = 0; n < c->V; ++n) perm[n] = c->permuted ? c->h_perm[n] : (uint32_t)n;
    return HYTG_OK;
}

hytg_status hytg_get_timeline(hytg_ctx *c, hytg_timed_launch *out, uint32_t cap, uint32_t *n) {
    if (!c || !n) return HYTG_ERR_ARG;
    *n = (uint32_t)c->timeline.size();
    if (out) {
        const uint32_t k = std::min<uint32_t>(cap, *n);
        std::copy(c->timeline.begin(), c->timeline.begin() + k, out);
    }
    return HYTG_OK;
}

hytg_status hytg_get_iterations(hytg_ctx *c, hytg_iter_record *out, uint32_t cap, uint32_t *n) {
    if (!c || !n) return HYTG_ERR_ARG;
    *n = (uint32_t)c->iters.size();
    if (out) {
        const uint32_t k = std::min<uint32_t>(cap, *n);
        std::copy(c->iters.begin(), c->iters.begin() + k, out);
    }
    return HYTG_OK;
}

}  // extern "C"
