// Tile set-up shared by the load-balanced relax, gather and batched relax
// kernels: a block takes kTile consecutive edges of a route's edge space,
// finds the list entries that own them (the first from the tile index
// written by k_bin), marks each entry's first edge in shared memory and fills
// the gaps with a max-scan, so every slot knows its owner entry in O(1).
#pragma once

#include "common.cuh"

namespace hytg {

__device__ __forceinline__ unsigned int sm_id() {
    unsigned int id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

constexpr unsigned int kInf = 0xFFFFFFFFu;

template <bool BATCH> struct TileSmem;
template <> struct TileSmem<false> {
    long long delta[kTile + 1];          // edge address = k + delta
    unsigned int pay[kTile + 1];         // value pushed by the entry
    unsigned short sid[kTile];           // owner entry (tile-relative) of each slot
    unsigned int wmax[kRelaxBlock / 32];
};
template <> struct TileSmem<true> {
    long long delta[kTile + 1];
    unsigned long long pay[kTile + 1];   // per-source frontier word of the entry
    unsigned int vid[kTile + 1];         // the entry's vertex (internal id)
    unsigned short sid[kTile];
    unsigned int wmax[kRelaxBlock / 32];
};

// Edge range [kb, ke) of a task in its route's edge space: the host's bounds,
// the whole route (device_sized), or one partition's slice of the F route
// read on the device (dev_edge; its first list entry goes to t.first_entry).
__device__ __forceinline__ void task_range(RelaxTask &t, const Summary *sum, unsigned long long &kb,
                                           unsigned long long &ke) {
    if (t.dev_edge) {
        kb = *t.dev_edge;
        ke = kb + *t.dev_len;
        t.first_entry = *t.dev_entry;
    } else if (t.device_sized) {
        kb = 0;
        ke = sum->route_edges[t.route];
    } else {
        kb = t.k_begin;
        ke = t.k_end;
    }
}

// Set up one tile; returns the number of edges (0 if nothing to do).
template <bool BATCH>
__device__ __forceinline__ int tile_setup(TileSmem<BATCH> &sm, const ListArrays &la, const Summary *sum,
                                          const RelaxTask &t, unsigned long long tile,
                                          unsigned long long kb, unsigned long long ke,
                                          unsigned long long *k0_out) {
    const int r = t.route;
    const unsigned long long rbase = sum->route_entry_base[r];
    const unsigned long long tbase = sum->route_tile_base[r];
    const unsigned long long n_ent = sum->route_entries[r];
    const unsigned long long route_edges = sum->route_edges[r];
    const unsigned long long tstart = tile * kTile;
    const unsigned long long k0 = tstart > kb ? tstart : kb;
    const unsigned long long tend = tstart + kTile;
    const unsigned long long k1 = tend < ke ? tend : ke;
    const unsigned long long i0 = (k0 == tstart) ? la.tile_first[tbase + tile] : t.first_entry;
    const unsigned long long last_tile = (route_edges - 1) / kTile;
    const unsigned long long i_last = (tile < last_tile) ? la.tile_first[tbase + tile + 1] : n_ent - 1;
    const long long n_e_ll = (long long)i_last - (long long)i0 + 1;
    if (n_e_ll < 1 || n_e_ll > kTile + 1 || i0 >= n_ent || i_last >= n_ent || k1 <= k0) {
        // inconsistent tile index: record it and skip the tile (block-uniform)
        if (threadIdx.x == 0) atomicOr(la.err, 1u);
        *k0_out = k0;
        return 0;
    }
    const int n_e = (int)n_e_ll;
    const int n_slots = (int)(k1 - k0);
    for (int j = threadIdx.x; j < kTile; j += kRelaxBlock) sm.sid[j] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n_e; j += kRelaxBlock) {
        const unsigned long long i = rbase + i0 + j;
        const unsigned long long eb = la.ebase[i];
        long long d;
        if (t.mode == kModeCompact) d = -t.shift;
        else d = (long long)la.soff[i] - (long long)eb - t.shift;
        sm.delta[j] = d;
        if constexpr (BATCH) {
            sm.pay[j] = la.pay64[i];
            sm.vid[j] = la.vid[i];
        } else {
            sm.pay[j] = la.pay[i];
        }
        if (j > 0) {
            const long long head = (long long)eb - (long long)k0;
            if (head > 0 && head < n_slots) sm.sid[head] = (unsigned short)j;
            else if (head <= 0) atomicOr(la.err, 4u);
        }
    }
    __syncthreads();
    // inclusive max-scan of sid over the tile (8 consecutive slots per thread)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int base = threadIdx.x * kRelaxIPT;
    unsigned int mx = 0;
#pragma unroll
    for (int q = 0; q < kRelaxIPT; ++q) {
        unsigned int x = sm.sid[base + q];
        mx = x > mx ? x : mx;
        sm.sid[base + q] = (unsigned short)mx;
    }
    unsigned int inc = mx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = y > inc ? y : inc;
    }
    if (lane == 31) sm.wmax[wid] = inc;
    __syncthreads();
    unsigned int carry = 0;
    for (int q = 0; q < wid; ++q) carry = sm.wmax[q] > carry ? sm.wmax[q] : carry;
    unsigned int excl = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane > 0) carry = excl > carry ? excl : carry;
    if (carry) {
#pragma unroll
        for (int q = 0; q < kRelaxIPT; ++q)
            if (sm.sid[base + q] < carry) sm.sid[base + q] = (unsigned short)carry;
    }
    __syncthreads();
    *k0_out = k0;
    return n_slots;
}

// Host-link reads of one tile, for routes that read mapped host memory: the
// distinct 32-byte sectors and 128-byte lines that the tile's edges occupy in
// one 4-byte edge array (base 256-byte aligned, so edge e sits in sector e / 8
// and line e / 32).  A tile's edges are at increasing addresses, so a sector
// (line) is new where it differs from the previous slot's; the first slot of
// a tile always counts, so a sector shared with the previous tile is counted
// twice (at most one per 2,048 edges).  Adds n_arrays times the counts to
// ctr[0] (sectors) and ctr[1] (lines).
template <bool BATCH>
__device__ __forceinline__ void count_link_reads(const TileSmem<BATCH> &sm, unsigned long long k0, int n,
                                                 unsigned int n_arrays, unsigned long long *ctr) {
    unsigned int sec = 0, ln = 0;
#pragma unroll
    for (int j = 0; j < kRelaxIPT; ++j) {
        const int slot = threadIdx.x + j * kRelaxBlock;
        if (slot < n) {
            const long long e = (long long)(k0 + slot) + sm.delta[sm.sid[slot]];
            if (slot == 0) {
                ++sec;
                ++ln;
            } else {
                const long long p = (long long)(k0 + slot - 1) + sm.delta[sm.sid[slot - 1]];
                sec += (e >> 3) != (p >> 3);
                ln += (e >> 5) != (p >> 5);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sec += __shfl_xor_sync(0xffffffffu, sec, o);
        ln += __shfl_xor_sync(0xffffffffu, ln, o);
    }
    if ((threadIdx.x & 31) == 0 && sec) {
        atomicAdd(&ctr[0], (unsigned long long)sec * n_arrays);
        atomicAdd(&ctr[1], (unsigned long long)ln * n_arrays);
    }
}

}  // namespace hytg
