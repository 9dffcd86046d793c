// Block-level helpers: exclusive scan and an LSD radix sort of keys staged in
// shared memory.
#pragma once

#include "wl_common.cuh"

namespace wl {

// Padded shared-memory index: one spare word every 32 removes the bank
// conflicts of thread-strided access to blocked arrangements.
__device__ __forceinline__ int pad(int p) { return p + (p >> 5); }

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Exclusive prefix sum of one value per thread over the block; returns the
// thread's prefix and writes the block total to *total (shared).
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = (lane < kWarps) ? warp_tot[lane] : 0;
        const int ti = warp_incl_scan(t);
        if (lane < kWarps) warp_tot[lane] = ti - t;
        if (lane == kWarps - 1) *total = ti;
    }
    __syncthreads();
    const int r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

// Exclusive scan in place of arr[0..n), n <= 2 * kThreads.
__device__ __forceinline__ void block_scan_array(int* arr, int n, int* warp_tot, int* total) {
    const int i0 = 2 * threadIdx.x, i1 = i0 + 1;
    const int a0 = (i0 < n) ? arr[i0] : 0, a1 = (i1 < n) ? arr[i1] : 0;
    const int p = block_excl_scan(a0 + a1, warp_tot, total);
    if (i0 < n) arr[i0] = p;
    if (i1 < n) arr[i1] = p + a0;
    __syncthreads();
}

// Ascending LSD radix sort (4-bit digits) of the keys at padded positions
// 0 .. kThreads*TPT of `keys`, comparing the low `nbits` bits.  Thread i owns
// the blocked range [i*TPT, (i+1)*TPT).  `cnt` holds 16 * kThreads uint16.
// Stable, so equal keys keep their position order.
template <int TPT>
__device__ void block_radix_sort(uint32_t* keys, uint16_t* cnt, int nbits, int* warp_tot,
                                 int* total) {
    const int tid = threadIdx.x;
    for (int sh = 0; sh < nbits; sh += 4) {
        uint32_t k[TPT];
        uint16_t rank[TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) k[j] = keys[pad(tid * TPT + j)];
#pragma unroll
        for (int d = 0; d < 16; ++d) cnt[d * kThreads + tid] = 0;
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int d = (k[j] >> sh) & 15;
            rank[j] = cnt[d * kThreads + tid];
            cnt[d * kThreads + tid] = rank[j] + 1;
        }
        __syncthreads();
        // exclusive scan over the 16 * kThreads counters in digit-major order
        int loc[16];
        int s = 0;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            loc[e] = s;
            s += cnt[tid * 16 + e];
        }
        const int base = block_excl_scan(s, warp_tot, total);
#pragma unroll
        for (int e = 0; e < 16; ++e) cnt[tid * 16 + e] = (uint16_t)(base + loc[e]);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int d = (k[j] >> sh) & 15;
            keys[pad(cnt[d * kThreads + tid] + rank[j])] = k[j];
        }
        __syncthreads();
    }
}

}  // namespace wl
