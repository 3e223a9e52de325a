// Initialisation, PageRank finalisation, frontier upload and the host-link
// probe kernel.
#include <atomic>

#include "common.cuh"

namespace hytg {

namespace {

// Initial values and frontier (Sec. II-A: traversals start from the source;
// CC and PageRank start with every vertex active).
__global__ void k_init(AlgoState st, unsigned long long V, unsigned long long n_words_alloc,
                       unsigned int source) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const float base = 1.0f - st.damping;
    for (unsigned long long v = t0; v < V; v += stride) {
        switch (st.algo) {
            case kBFS:
            case kSSSP: st.val[v] = (v == source) ? 0u : 0xFFFFFFFFu; break;
            case kCC: st.val[v] = (unsigned int)v; break;   // internal id, mapped at the end
            case kPR: st.rank[v] = 0.0f; st.delta[v] = base; break;
            // PPR: the seed holds the whole initial residual of PageRank,
            // (1 - d) V, so that eps bounds the same relative error
            default: st.rank[v] = 0.0f; st.delta[v] = (v == source) ? base * (float)V : 0.0f; break;
        }
    }
    const bool all = (st.algo == kCC || st.algo == kPR);
    const unsigned long long full_words = V >> 5;
    for (unsigned long long w = t0; w < n_words_alloc; w += stride) {
        unsigned int bits = 0;
        if (all) {
            if (w < full_words) bits = 0xFFFFFFFFu;
            else if (w == full_words && (V & 31)) bits = (1u << (V & 31)) - 1u;
        } else if (w == (source >> 5)) {
            bits = 1u << (source & 31);
        }
        st.bm_cur[w] = bits;
    }
    if (t0 == 0) *st.overflow = 0u;
}

// Delta-PageRank frontier: v is active iff delta[v] > eps (Sec. VI-A names
// delta-based PageRank without a threshold; eps is an FP32 residual on the
// unnormalised scale, where every vertex starts with delta = 1 - d).
// Inactive vertices always hold delta <= eps, so this equals "delta crossed
// eps during the iteration".
__global__ void k_pr_frontier(AlgoState st, unsigned long long V, unsigned long long n_words_alloc) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (unsigned long long base = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull;
         base < n_words_alloc * 32; base += stride) {
        const unsigned long long v = base + lane;
        const bool act = v < V && st.delta[v] > st.eps;
        const unsigned int bits = __ballot_sync(0xffffffffu, act);
        if (lane == 0) st.bm_cur[base >> 5] = bits;
    }
}

// CC pointer jumping over the vertices changed in the last iteration: a
// label is always the id of a vertex of the same component that is not
// larger than the vertex itself, so label[label[v]] is a valid, no larger
// label for v.  Jumping collapses label chains that min-label propagation
// alone would walk one edge per iteration on high-diameter graphs; the
// vertices it changes are already in the frontier and push their new label.
__global__ void k_cc_jump(AlgoState st, unsigned long long n_words_alloc) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         w < n_words_alloc; w += stride) {
        unsigned int bits = st.bm_cur[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const unsigned long long v = w * 32 + b;
            const unsigned int l0 = __ldcg(&st.val[v]);
            unsigned int l = l0;
            for (int hop = 0; hop < 64; ++hop) {
                const unsigned int l2 = __ldcg(&st.val[l]);
                if (l2 >= l) break;
                l = l2;
            }
            if (l < l0) atomicMin(&st.val[v], l);
        }
    }
}

// CC labels (smallest internal id of each component) to the smallest
// original id of the component, in original vertex order.
// tmp[label] = smallest original id with that label.  Most vertices share
// the giant component's label, so the lanes of a warp are grouped by label
// (isolated vertices form groups of one), each group reduces its ids, and
// one lane per group issues the atomic: one per distinct label instead of
// 32 to the same address.
__global__ void k_cc_min_orig(AlgoState st, unsigned long long V, unsigned int *tmp) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull;
         base < V; base += stride) {
        const unsigned long long v = base + lane;
        const bool in = v < V;
        const unsigned int lab = in ? st.val[v] : 0xFFFFFFFFu;
        const unsigned int orig = in ? (st.perm ? st.perm[v] : (unsigned int)v) : 0xFFFFFFFFu;
        const unsigned int grp = __match_any_sync(0xffffffffu, lab);
        const unsigned int m = __reduce_min_sync(grp, orig);
        if (in && lane == __ffs(grp) - 1) atomicMin(&tmp[lab], m);
    }
}
__global__ void k_cc_write(AlgoState st, unsigned long long V, const unsigned int *tmp,
                           unsigned int *out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride)
        out[st.perm ? st.perm[v] : v] = tmp[st.val[v]];
}

// Fold the per-SM hub replicas into delta and clear them.  A block takes 32
// consecutive hub ids; each of its 8 warps sums every 8th replica row of
// those ids (128-byte rows, eight loads in flight), and the first warp adds
// the 8 partial sums into delta.
__global__ void __launch_bounds__(256) k_hub_reduce(AlgoState st) {
    __shared__ float part[8][32];
    const unsigned int K = st.n_hub_rep;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (unsigned int v0 = blockIdx.x * 32u; v0 < K; v0 += gridDim.x * 32u) {
        const unsigned int v = v0 + lane;
        float s = 0.0f;
        if (v < K) {
#pragma unroll 8
            for (unsigned int r = wid; r < kHubReplicas; r += 8) {
                float *p = st.hub_rep + (size_t)r * K + v;
                s += *p;
                *p = 0.0f;
            }
        }
        part[wid][lane] = s;
        __syncthreads();
        if (wid == 0 && v < K) {
            float t = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) t += part[q][lane];
            st.delta[v] += t;
        }
        __syncthreads();
    }
}

__global__ void k_pr_sums(AlgoState st, unsigned long long V, double *sums) {
    __shared__ double s_rank[32], s_res[32];
    double r = 0.0, d = 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride) {
        r += st.rank[v];
        d += fabs((double)st.delta[v]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_rank[wid] = r; s_res[wid] = d; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        r = lane < nw ? s_rank[lane] : 0.0;
        d = lane < nw ? s_res[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r += __shfl_xor_sync(0xffffffffu, r, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) { atomicAdd(&sums[0], r); atomicAdd(&sums[1], d); }
    }
}

__global__ void k_pr_normalise(AlgoState st, unsigned long long V, const double *sums, float *out) {
    const double s = sums[0];
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride)
        out[st.perm ? st.perm[v] : v] = (float)((double)st.rank[v] * inv);
}

// Copy a per-vertex array from internal to original vertex order.
__global__ void k_to_original(const unsigned int *perm, const unsigned int *in, unsigned int *out,
                              unsigned long long V) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += stride)
        out[perm ? perm[v] : v] = in[v];
}

__global__ void k_upload_bitmap(const unsigned char *active, unsigned int *bm, unsigned long long V,
                                unsigned long long n_words_alloc) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         w < n_words_alloc; w += stride) {
        unsigned int bits = 0;
        for (int b = 0; b < 32; ++b) {
            const unsigned long long v = w * 32 + b;
            if (v < V && active[v]) bits |= 1u << b;
        }
        bm[w] = bits;
    }
}

// Reads n16 16-byte words (a warp covers 512 contiguous bytes = four
// 128-byte lines per step) and folds them into one word so the loads stay.
__global__ void k_zc_probe(const uint4 *src, unsigned long long n16, unsigned long long *sink) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int acc = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n16;
         i += stride) {
        const uint4 x = __ldg(src + i);
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

// F-route copy by the SMs ("f_copy" > 0), in place of the copy engine: the
// words [0, n) of mapped host memory into a staging slot, both 16-byte
// aligned, with 16-byte loads, four in flight per thread; the last n % 4
// words one at a time.
__global__ void __launch_bounds__(256) k_stage_copy(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                    unsigned long long n) {
    const unsigned long long n4 = n / 4;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long i = t0;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        const uint4 a = __ldg(src + i), b = __ldg(src + i + stride);
        const uint4 c = __ldg(src + i + 2 * stride), d = __ldg(src + i + 3 * stride);
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n4; i += stride) dst[i] = __ldg(src + i);
    if (t0 < n - n4 * 4)
        ((unsigned int *)dst)[n4 * 4 + t0] = __ldg((const unsigned int *)src + n4 * 4 + t0);
}

// L2 reduction probe: indices into a 2^24-float array, uniform or with the
// R-MAT in-degree skew (each of 24 bits set with probability 0.24), then
// n fire-and-forget float additions.
__device__ __forceinline__ unsigned long long probe_mix(unsigned long long x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
    return x;
}
__device__ __forceinline__ unsigned int binom24(unsigned int n, unsigned int r) {
    if (r > n) return 0u;
    unsigned long long x = 1;
    for (unsigned int i = 1; i <= r; ++i) x = x * (n - r + i) / i;
    return (unsigned int)x;
}
// The same skew after hub sorting: ids ordered by their probability, i.e.
// by popcount (fewer set bits first), and within one popcount by the
// combinatorial rank of the bit pattern.  Bijective on [0, 2^24).
__device__ __forceinline__ unsigned int hub_rank24(unsigned int v) {
    const unsigned int k = __popc(v);
    unsigned int off = 0;
    for (unsigned int i = 0; i < k; ++i) off += binom24(24, i);
    unsigned int rank = 0, seen = 0;
    for (unsigned int b = 0; b < 24; ++b)
        if ((v >> b) & 1u) rank += binom24(b, ++seen);
    return off + rank;
}

// skew 0: uniform over 2^24 floats; 1: R-MAT in-degree skew (each of 24
// index bits set with probability 0.24); 2: that skew with hub-sorted ids.
__global__ void k_probe_idx(unsigned int *idx, unsigned long long n, int skew) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned int v = 0;
        if (!skew) {
            v = (unsigned int)(probe_mix(i * 2654435761ull + 7) & 0xFFFFFFull);
        } else {
            for (int j = 0; j < 24; ++j)
                if ((probe_mix(i * 64 + j + 12345) & 0xFFFFFFFFull) < 1030792151ull) v |= 1u << j;
            if (skew == 2) v = hub_rank24(v);
        }
        idx[i] = v;
    }
}
__global__ void k_probe_red(const unsigned int *__restrict__ idx, unsigned long long n, float *d) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&d[__ldg(idx + i)], 1.0f);
}
// The relax kernels' scheme: additions to ids below n_rep go to this SM's
// row of per-SM replicas (not folded here).
__global__ void k_probe_red_rep(const unsigned int *__restrict__ idx, unsigned long long n, float *d,
                                float *rep, unsigned int n_rep) {
    unsigned int smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    float *row = rep + (size_t)(smid % kHubReplicas) * n_rep;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned int v = __ldg(idx + i);
        if (v < n_rep) atomicAdd(&row[v], 1.0f);
        else atomicAdd(&d[v], 1.0f);
    }
}

// Frame pushes, the batched PPR relax's access: each adds a frame of 8 floats
// (32 bytes, one sector) at a vertex given by idx, as 8 / W reductions of W
// floats each (W = 1: red.global.add.f32; 2, 4: the .v2 / .v4 forms).
template <int W>
__global__ void k_probe_frame(const unsigned int *__restrict__ idx, unsigned long long n, float *d) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float *p = d + (unsigned long long)__ldg(idx + i) * 8ull;
        if (W == 4) {
            atomicAdd((float4 *)p, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
            atomicAdd((float4 *)p + 1, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
        } else if (W == 2) {
#pragma unroll
            for (int j = 0; j < 4; ++j) atomicAdd((float2 *)p + j, make_float2(1.0f, 1.0f));
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(p + j, 1.0f);
        }
    }
}

inline unsigned int grid_for(unsigned long long n, unsigned int block) {
    unsigned long long g = (n + block - 1) / block;
    const unsigned long long cap = 32ull * device_sms();
    if (g > cap) g = cap;
    return g == 0 ? 1u : (unsigned int)g;
}

constexpr int kMaxDevices = 64;
std::atomic<unsigned int> g_sms[kMaxDevices];

}  // namespace

unsigned int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    unsigned int n = g_sms[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
        n = (unsigned int)v;
        g_sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t launch_init(const AlgoState &st, unsigned long long V, unsigned long long n_words_alloc,
                        unsigned int source, cudaStream_t s) {
    const unsigned long long n = V > n_words_alloc ? V : n_words_alloc;
    k_init<<<grid_for(n, 256), 256, 0, s>>>(st, V, n_words_alloc, source);
    return cudaGetLastError();
}

cudaError_t launch_pr_finalize(const AlgoState &st, unsigned long long V, float *out, double *sums,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_pr_sums<<<grid_for(V, 256), 256, 0, s>>>(st, V, sums);
    k_pr_normalise<<<grid_for(V, 256), 256, 0, s>>>(st, V, sums, out);
    return cudaGetLastError();
}

cudaError_t launch_hub_reduce(const AlgoState &st, cudaStream_t s) {
    if (!st.hub_rep || st.n_hub_rep == 0) return cudaSuccess;
    k_hub_reduce<<<(st.n_hub_rep + 31) / 32, 256, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_cc_jump(const AlgoState &st, unsigned long long n_words_alloc, cudaStream_t s) {
    k_cc_jump<<<grid_for(n_words_alloc, 256), 256, 0, s>>>(st, n_words_alloc);
    return cudaGetLastError();
}

cudaError_t launch_cc_final(const AlgoState &st, unsigned long long V, unsigned int *tmp,
                            unsigned int *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tmp, 0xFF, V * 4, s);
    if (e != cudaSuccess) return e;
    k_cc_min_orig<<<grid_for(V, 256), 256, 0, s>>>(st, V, tmp);
    k_cc_write<<<grid_for(V, 256), 256, 0, s>>>(st, V, tmp, out);
    return cudaGetLastError();
}

cudaError_t launch_pr_frontier(const AlgoState &st, unsigned long long V,
                               unsigned long long n_words_alloc, cudaStream_t s) {
    const unsigned long long n = n_words_alloc * 32;
    unsigned long long g = (n + 255) / 256;
    if (g > 16ull * device_sms()) g = 16ull * device_sms();
    k_pr_frontier<<<(unsigned int)g, 256, 0, s>>>(st, V, n_words_alloc);
    return cudaGetLastError();
}

cudaError_t launch_to_original(const unsigned int *perm, const unsigned int *in, float *out,
                               unsigned long long V, cudaStream_t s) {
    k_to_original<<<grid_for(V, 256), 256, 0, s>>>(perm, in, (unsigned int *)out, V);
    return cudaGetLastError();
}

cudaError_t launch_upload_bitmap(const unsigned char *active_dev, unsigned int *bm,
                                 unsigned long long V, unsigned long long n_words_alloc,
                                 cudaStream_t s) {
    k_upload_bitmap<<<grid_for(n_words_alloc, 256), 256, 0, s>>>(active_dev, bm, V, n_words_alloc);
    return cudaGetLastError();
}

cudaError_t launch_red_probe(unsigned int *idx, float *d, unsigned long long n, int skew, bool gen,
                             cudaStream_t s, float *rep, unsigned int n_rep) {
    if (gen) k_probe_idx<<<16 * device_sms(), 256, 0, s>>>(idx, n, skew);
    else if (rep && n_rep) k_probe_red_rep<<<32 * device_sms(), 256, 0, s>>>(idx, n, d, rep, n_rep);
    else k_probe_red<<<32 * device_sms(), 256, 0, s>>>(idx, n, d);
    return cudaGetLastError();
}

cudaError_t launch_frame_probe(const unsigned int *idx, float *d, unsigned long long n, int width,
                               cudaStream_t s) {
    const unsigned int grid = 32 * device_sms();
    if (width == 4) k_probe_frame<4><<<grid, 256, 0, s>>>(idx, n, d);
    else if (width == 2) k_probe_frame<2><<<grid, 256, 0, s>>>(idx, n, d);
    else if (width == 1) k_probe_frame<1><<<grid, 256, 0, s>>>(idx, n, d);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_zc_probe(const uint4 *src, unsigned long long n16, unsigned long long *sink,
                            int grid, cudaStream_t s) {
    k_zc_probe<<<grid, 256, 0, s>>>(src, n16, sink);
    return cudaGetLastError();
}

cudaError_t launch_stage_copy(const unsigned int *src, unsigned int *dst, unsigned long long n,
                              unsigned int blocks_per_sm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15) || blocks_per_sm == 0) return cudaErrorInvalidValue;
    unsigned long long blocks = (n / 4 + 255) / 256;
    const unsigned long long cap = (unsigned long long)blocks_per_sm * device_sms();
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_stage_copy<<<(unsigned int)blocks, 256, 0, s>>>((const uint4 *)src, (uint4 *)dst, n);
    return cudaGetLastError();
}

}  // namespace hytg
