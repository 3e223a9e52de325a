// hytg_plan_noalloc: the per-partition counting and engine selection of the
// planning kernels for a frontier that is already in device memory, for
// callers that must not allocate device memory (see include/hytg.h).  Its
// scratch (partition bounds in bitmap words and in edges) lives in a
// file-scope static device array; the caller passes every input and output.
#include <mutex>

#include "common.cuh"
#include "cost_model.cuh"
#include "hytg.h"

namespace hytg {
namespace {

constexpr unsigned int kNaMaxParts = HYTG_NOALLOC_MAX_PARTS;

struct NoAllocScratch {
    unsigned long long eb[kNaMaxParts + 1];   // partition bounds in edges
    unsigned int wb[kNaMaxParts + 1];         // partition bounds in bitmap words
};

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Bounds of every partition, and zeroed count outputs.
__global__ void k_na_bounds(const unsigned long long *off, unsigned long long V,
                            const unsigned long long *vb, unsigned int n_parts,
                            NoAllocScratch *sc, unsigned long long *counts) {
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int p = blockIdx.x * blockDim.x + threadIdx.x; p <= n_parts; p += stride) {
        unsigned long long v = vb[p];
        if (v > V) v = V;
        sc->eb[p] = off[v];
        sc->wb[p] = (unsigned int)((v + 31) / 32);
        if (p < n_parts) counts[3 * p] = counts[3 * p + 1] = counts[3 * p + 2] = 0ull;
    }
}

__device__ __forceinline__ unsigned int na_find_part(const unsigned int *wb, unsigned int N,
                                                     unsigned long long widx) {
    unsigned int lo = 0, hi = N;
    while (hi - lo > 1) {
        const unsigned int mid = (lo + hi) >> 1;
        if ((unsigned long long)wb[mid] <= widx) lo = mid; else hi = mid;
    }
    return lo;
}

// |A_i|, active edges and 128-byte lines per partition (footnote to Eq. 3),
// accumulated into counts[3 p + {0, 1, 2}].  One warp per 32 bitmap words.
__global__ void __launch_bounds__(256) k_na_count(const unsigned int *bm, unsigned long long V,
                                                  const unsigned long long *off,
                                                  const NoAllocScratch *sc, unsigned int n_parts,
                                                  unsigned int n_arrays, unsigned long long m,
                                                  unsigned long long *counts) {
    const int lane = threadIdx.x & 31;
    const unsigned long long n_words = (V + 31) / 32;
    const unsigned long long n_groups = (n_words + 31) / 32;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long grp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
         grp < n_groups; grp += nwarps) {
        const unsigned long long widx_l = grp * 32 + lane;
        unsigned int bits = widx_l < n_words ? bm[widx_l] : 0u;
        if (widx_l == n_words - 1 && (V & 31)) bits &= (1u << (V & 31)) - 1u;
        unsigned int nz = __ballot_sync(0xffffffffu, bits != 0);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            const unsigned int w = __shfl_sync(0xffffffffu, bits, src);
            const unsigned long long widx = grp * 32 + src;
            const unsigned int p = na_find_part(sc->wb, n_parts, widx);
            unsigned long long deg = 0, ln = 0;
            if ((w >> lane) & 1u) {
                const unsigned long long v = widx * 32 + lane;
                const unsigned long long o0 = off[v];
                deg = off[v + 1] - o0;
                ln = (unsigned long long)n_arrays * lines_spanned(o0 * 4ull, deg * 4ull, m);
            }
            const unsigned long long e_sum = warp_sum_u64(deg);
            const unsigned long long l_sum = warp_sum_u64(ln);
            if (lane == 0) {
                atomicAdd(&counts[3 * p], (unsigned long long)__popc(w));
                atomicAdd(&counts[3 * p + 1], e_sum);
                atomicAdd(&counts[3 * p + 2], l_sum);
            }
        }
    }
}

__global__ void k_na_select(const NoAllocScratch *sc, unsigned int n_parts,
                            const unsigned long long *counts, CostParams cp, unsigned char *routes) {
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_parts; p += stride)
        routes[p] = (unsigned char)decide_route_counts(p, sc->eb[p + 1] - sc->eb[p], counts[3 * p],
                                                       counts[3 * p + 1], counts[3 * p + 2], cp);
}

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
void *g_na_addr[kNaMaxDevices] = {};
unsigned int g_na_sms[kNaMaxDevices] = {};

}  // namespace
}  // namespace hytg

using namespace hytg;

extern "C" hytg_status hytg_plan_noalloc(hytg_algo algo, const uint32_t *frontier,
                                         const uint64_t *offsets, uint64_t V,
                                         const uint64_t *part_vbounds, uint32_t n_parts,
                                         uint32_t n_cached, const hytg_cost_params *params,
                                         uint8_t *routes, uint64_t *counts, void *stream) {
    const int a = (int)algo;
    if (a < 0 || a > 4 || !frontier || !offsets || !part_vbounds || !routes || !counts)
        return HYTG_ERR_ARG;
    if (V == 0 || V > 0xFFFFFFFFull) return HYTG_ERR_ARG;
    if (n_parts == 0 || n_parts > HYTG_NOALLOC_MAX_PARTS || n_cached > n_parts) return HYTG_ERR_ARG;
    hytg_cost_params prm = {0.8, 0.4, 0.625, 128, 256};
    if (params) prm = *params;
    if (prm.m == 0 || prm.MR == 0 || !(prm.gamma >= 0 && prm.gamma <= 1) || !(prm.alpha >= 0) ||
        !(prm.beta >= 0) || prm.alpha > 1000 || prm.beta > 1000)
        return HYTG_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return HYTG_ERR_CUDA;
    // an error left pending by earlier, unrelated work is not this call's to
    // report or to clear: queue nothing and leave it for its owner
    if (cudaPeekAtLastError() != cudaSuccess) return HYTG_ERR_CUDA;
    void *scratch = nullptr;
    unsigned int sms = 0;
    {
        // once per device, with that device current: the device address of
        // the static scratch array and the SM count that sizes the grid
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            int n = 0;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
                cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
                cudaGetLastError();
                return HYTG_ERR_CUDA;
            }
            g_na_sms[dev] = (unsigned int)n;
            g_na_addr[dev] = p;
        }
        scratch = g_na_addr[dev];
        sms = g_na_sms[dev];
    }
    CostParams cp;
    auto q = [](double x) { return (unsigned long long)((x * (double)kParamDen) + 0.5); };
    cp.alpha_num = q(prm.alpha);
    cp.beta_num = q(prm.beta);
    cp.gamma_num = q(prm.gamma);
    cp.m = prm.m;
    cp.MR = prm.MR;
    cp.d1 = (a == kSSSP) ? 8 : 4;
    cp.d2 = 8;
    cp.n_cached = n_cached;
    cp.force_route = -1;
    cp.seed = 0;
    cp.iteration = 0;
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocScratch *sc = (NoAllocScratch *)scratch;
    const unsigned int nb = (n_parts + 1 + 255) / 256;
    k_na_bounds<<<nb, 256, 0, s>>>((const unsigned long long *)offsets, V,
                                   (const unsigned long long *)part_vbounds, n_parts, sc,
                                   (unsigned long long *)counts);
    const unsigned long long n_groups = ((V + 31) / 32 + 31) / 32;
    unsigned long long blocks = (n_groups + 7) / 8;
    if (blocks > 16ull * sms) blocks = 16ull * sms;
    if (blocks == 0) blocks = 1;
    k_na_count<<<(unsigned int)blocks, 256, 0, s>>>(frontier, V, (const unsigned long long *)offsets, sc,
                                                    n_parts, a == kSSSP ? 2u : 1u, prm.m,
                                                    (unsigned long long *)counts);
    k_na_select<<<nb, 256, 0, s>>>(sc, n_parts, (const unsigned long long *)counts, cp, routes);
    return cudaGetLastError() == cudaSuccess ? HYTG_OK : HYTG_ERR_CUDA;
}
