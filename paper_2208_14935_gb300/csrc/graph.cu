// Kernels of the device-driven iteration loop.  The host captures one
// iteration (pre-step, counts, selection, k_loop_decide, binning, cache and
// zero-copy relax) as the body of a CUDA-graph WHILE node; k_loop_decide
// ends the loop when the frontier is empty, when the iteration cap is
// reached, or when the selection (Sec. V-A) sent a partition to the F or C
// route, whose copies the host issues (Sec. V-B task combination and
// Sec. VI-B multi-stream scheduling stay on the host).  Iterations that use
// only the resident cache and zero-copy routes (the long tails of tiny
// frontiers on high-diameter graphs) then cost no host round trip.
#include "common.cuh"
#include "hytg.h"

namespace hytg {

namespace {

__global__ void k_zero_u64(unsigned long long *p, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        p[i] = 0ull;
}

// One thread: the host loop's decisions for the iteration just planned.
__global__ void k_loop_decide(const Summary *sum, LoopCtl *ctl, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
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
    if (sum->route_parts[kRouteF] != 0 || sum->route_parts[kRouteC] != 0 || ctl->n_rec >= ctl->rec_cap) {
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
    k_loop_decide<<<1, 32, 0, s>>>(sum, ctl, (cudaGraphConditionalHandle)cond_handle);
    return cudaGetLastError();
}

}  // namespace hytg
