// Kernels of the device-driven iteration loop.  The host captures one
// iteration (pre-step, counts, selection, k_loop_decide, binning, cache and
// zero-copy relax, and with "device_loop" 2 one IF node per partition that
// copies it into a staging slot and relaxes it, and an IF node for the C
// route) as the body of a CUDA-graph WHILE node; k_loop_decide ends the loop
// when the frontier is empty, when the iteration cap is reached, or when the
// selection (Sec. V-A) sent a partition to a route the body does not hold
// (F or C with "device_loop" 1; a C route larger than the compaction buffer),
// whose copies the host then issues, or when the host has set the cancel word
// (the run passed its deadline).  Iterations run in the body cost no host
// round trip.
#include "common.cuh"
#include "hytg.h"

namespace hytg {

namespace {

__global__ void k_zero_u64(unsigned long long *p, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        p[i] = 0ull;
}

__device__ void loop_decide_one(const Summary *sum, LoopCtl *ctl, cudaGraphConditionalHandle h);

// Thread 0: the host loop's decisions for the iteration just planned; then
// the block opens the IF nodes of the partitions routed F (each copies its
// partition into a staging slot and relaxes it) and of the C route.
__global__ void k_loop_decide(const Summary *sum, LoopCtl *ctl, cudaGraphConditionalHandle h) {
    __shared__ unsigned long long s_parts, s_bytes;
    if (threadIdx.x == 0) {
        s_parts = s_bytes = 0;
        loop_decide_one(sum, ctl, h);
    }
    __syncthreads();
    // every IF condition is set on every iteration (a value set once would
    // otherwise carry over to the next iteration of the loop), and left
    // closed when the device does not take the iteration
    const bool work = ctl->work != 0;
    if (ctl->f_handles) {
        unsigned long long np = 0, nb = 0;
        for (unsigned int i = threadIdx.x; i < ctl->n_parts; i += blockDim.x) {
            const bool f = work && ctl->route[i] == kRouteF;
            cudaGraphSetConditional((cudaGraphConditionalHandle)ctl->f_handles[i], f ? 1u : 0u);
            if (f) {
                ++np;
                nb += (ctl->part_eb[i + 1] - ctl->part_eb[i]) * 4ull * ctl->n_arrays;
            }
        }
        if (np) {
            atomicAdd(&s_parts, np);
            atomicAdd(&s_bytes, nb);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool c_on = work && sum->route_edges[kRouteC] != 0;
        if (ctl->c_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)ctl->c_handle, c_on ? 1u : 0u);
        if (work) {
            hytg_iter_record *r = (hytg_iter_record *)ctl->rec + (ctl->n_rec - 1);
            r->f_tasks = (unsigned int)s_parts;
            r->link_bytes += s_bytes;
            ctl->f_parts += s_parts;
            ctl->f_bytes += s_bytes;
            if (c_on && ctl->c_handle) {
                ++ctl->c_iters;
                ctl->c_lines += sum->route_lines[kRouteC];
                r->link_bytes += sum->route_lines[kRouteC] * ctl->m;
            }
        }
    }
}

// F copy inside the device loop without a memcpy node: 16-byte loads from
// mapped host memory, coalesced, into the staging slot.
__global__ void k_copy_words(const unsigned int *src, unsigned int *dst, unsigned long long n,
                             const LoopCtl *loop) {
    if (loop && !loop->work) return;
    const unsigned long long n4 = n / 4;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    for (unsigned long long i = t0; i < n4; i += stride)
        ((uint4 *)dst)[i] = __ldcs((const uint4 *)src + i);
    for (unsigned long long i = n4 * 4 + t0; i < n; i += stride) dst[i] = src[i];
}

__device__ void loop_decide_one(const Summary *sum, LoopCtl *ctl, cudaGraphConditionalHandle h) {
    ctl->work = 0;
    if (sum->n_active == 0) {
        if (sum->pending == 0) {
            ctl->status = kLoopDone;
            cudaGraphSetConditional(h, 0);
            return;
        }
        // the current bucket is settled: open the next one at the smallest
        // pending distance (delta-stepping), and plan again
        unsigned long long nb = (unsigned long long)(ctl->bucket > sum->pending_min ? ctl->bucket : sum->pending_min);
        nb += ctl->delta;
        ctl->bucket = nb < 0xFFFFFFFEull ? (unsigned int)nb : 0xFFFFFFFEu;
        if (sum->pending_min >= 0xFFFFFFFEu) ctl->bucket = 0xFFFFFFFFu;
        ++ctl->it;
        cudaGraphSetConditional(h, 1);
        return;
    }
    if ((unsigned long long)ctl->it >= ctl->max_it) {
        ctl->status = kLoopMaxIt;
        cudaGraphSetConditional(h, 0);
        return;
    }
    if (ctl->cancel && *ctl->cancel != 0u) {
        ctl->status = kLoopCancel;        // nothing of this iteration runs
        cudaGraphSetConditional(h, 0);
        return;
    }
    const bool f_host = sum->route_parts[kRouteF] != 0 && !ctl->f_handles;
    const bool c_host = sum->route_parts[kRouteC] != 0 &&
                        (!ctl->c_handle || sum->route_edges[kRouteC] > ctl->c_cap);
    if (f_host || c_host || ctl->n_rec >= ctl->rec_cap) {
        ctl->status = kLoopHost;          // the host takes this iteration from k_bin on
        cudaGraphSetConditional(h, 0);
        return;
    }
    hytg_iter_record *r = (hytg_iter_record *)ctl->rec + ctl->n_rec++;
    unsigned long long act = 0;
    for (int q = 0; q < kRoutes; ++q) {
        act += sum->route_edges[q];
        r->route_partitions[q] = sum->route_parts[q];
        r->route_edges[q] = sum->route_edges[q];
        ctl->route_parts[q] += sum->route_parts[q];
        ctl->route_entries[q] += sum->route_entries[q];
        ctl->route_edges[q] += sum->route_edges[q];
    }
    r->active_vertices = sum->n_active;
    r->active_edges = act;
    r->f_tasks = 0;
    r->link_bytes = sum->route_lines[kRouteZ] * ctl->m;
    r->device_ms = 0.0;
    ctl->z_lines += sum->route_lines[kRouteZ];
    ctl->vertices += sum->n_active;
    ctl->edges += act;
    ++ctl->iterations;
    ctl->work = 1;
    ++ctl->it;
    cudaGraphSetConditional(h, 1);
}

}  // namespace

cudaError_t launch_zero_u64(unsigned long long *p, unsigned long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned long long blocks = (n + 255) / 256;
    if (blocks > 4ull * device_sms()) blocks = 4ull * device_sms();
    k_zero_u64<<<(unsigned int)blocks, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_loop_decide(const Summary *sum, LoopCtl *ctl, unsigned long long cond_handle,
                               cudaStream_t s) {
    k_loop_decide<<<1, 256, 0, s>>>(sum, ctl, (cudaGraphConditionalHandle)cond_handle);
    return cudaGetLastError();
}

cudaError_t launch_copy_words(const unsigned int *src, unsigned int *dst, unsigned long long n,
                              const LoopCtl *loop, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (((uintptr_t)src | (uintptr_t)dst) & 15) return cudaErrorInvalidValue;
    unsigned long long blocks = (n / 4 + 255) / 256;
    if (blocks > 4ull * device_sms()) blocks = 4ull * device_sms();
    if (blocks == 0) blocks = 1;
    k_copy_words<<<(unsigned int)blocks, 256, 0, s>>>(src, dst, n, loop);
    return cudaGetLastError();
}

}  // namespace hytg
