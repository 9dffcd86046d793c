// Device building blocks of the WarpLDA sampler: Philox4x32-10, the FP32
// acceptance and mixture tests, and the per-segment count tables.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wl {

constexpr int kThreads = 256;          // threads of every sampler block
constexpr int kWarps = kThreads / 32;
constexpr int kSegsMax = 512;          // segments (documents / words) per block batch
constexpr int kHashCountBits = 12;     // packed hash entry: (topic + 1) << 12 | count
constexpr int kMaxBatchTokens = 4095;  // count of a packed entry stays below 2^12

enum Phase : uint32_t { kPhaseInit = 0, kPhaseDoc = 1, kPhaseWord = 2 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor bijection with the Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The sampler's block for (token t, iteration, phase, MH step i, stream).
__device__ __forceinline__ uint4 draw(uint32_t t, uint32_t iter, uint32_t phase, uint32_t step,
                                      uint32_t stream, uint32_t k0, uint32_t k1) {
    return philox(make_uint4(t, iter, (phase << 8) | step, stream), k0, k1);
}

// u = (r >> 8) * 2^-24, exact in FP32.
__device__ __forceinline__ float u24(uint32_t r) {
    return __fmul_rn(__uint2float_rn(r >> 8), 5.9604644775390625e-8f);
}

// Dice(n): (r * n) >> 32.
__device__ __forceinline__ uint32_t dice(uint32_t r, uint32_t n) { return __umulhi(r, n); }

// One Eq. 7 acceptance test from s to t (t != s): accept iff
//   u * ((C_s + g) * ckb_t) < (C_t + g) * ckb_s,
// ckb_k = (float)c_k + beta_bar.  Every operation is one FP32 RN operation.
__device__ __forceinline__ bool accept(uint32_t r0, int Cs, int Ct, float g, float ckb_s,
                                       float ckb_t) {
    const float num = __fmul_rn(__fadd_rn(__int2float_rn(Ct), g), ckb_s);
    const float den = __fmul_rn(__fadd_rn(__int2float_rn(Cs), g), ckb_t);
    return __fmul_rn(u24(r0), den) < num;
}

// Mixture coin of Eq. 6 (Sec. 2.2): p_A branch iff u * (L + G) < L.
__device__ __forceinline__ bool coin(uint32_t r1, float Lf, float LG) {
    return __fmul_rn(u24(r1), LG) < Lf;
}

// ---------------------------------------------------------------------------
// Per-segment count tables in shared memory (Sec. 5.4).  A segment's table is
// either dense (ceil(K/2) words, two 16-bit counts per word) or an
// open-addressing hash with linear probing and the `and` hash, capacity the
// smallest power of two above min(K, 2L), entries packed as
// (topic + 1) << 12 | count.  Dense is used whenever it is no larger.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t pow2_above(uint32_t x) {
    uint32_t c = 1;
    while (c <= x) c <<= 1;
    return c;
}

// Words of shared memory and the hash capacity (0 = dense) for a segment.
__host__ __device__ __forceinline__ void table_shape(uint32_t L, uint32_t K, uint32_t* words,
                                                     uint32_t* cap) {
    const uint32_t dense = (K + 1) / 2;
    if (L == 0) { *words = 0; *cap = 0; return; }
    const uint32_t h = pow2_above(L * 2 < K ? L * 2 : K);
    if (dense <= h) { *words = dense; *cap = 0; }
    else { *words = h; *cap = h; }
}

__device__ __forceinline__ void table_add(uint32_t* tab, uint32_t cap, uint32_t k) {
    if (cap == 0) {
        atomicAdd(&tab[k >> 1], (k & 1) ? 65536u : 1u);
        return;
    }
    const uint32_t tag = (k + 1) << kHashCountBits;
    uint32_t h = k & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        uint32_t v = tab[h];
        if (v == 0) {
            const uint32_t old = atomicCAS(&tab[h], 0u, tag | 1u);
            if (old == 0) return;
            v = old;
        }
        if ((v & ~((1u << kHashCountBits) - 1)) == tag) {
            atomicAdd(&tab[h], 1u);
            return;
        }
        h = (h + 1) & (cap - 1);
    }
    // unreachable: capacity exceeds the segment's token count
}

__device__ __forceinline__ int table_get(const uint32_t* tab, uint32_t cap, uint32_t k) {
    if (cap == 0) return (int)((tab[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu);
    const uint32_t tag = (k + 1) << kHashCountBits;
    uint32_t h = k & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const uint32_t v = tab[h];
        if (v == 0) return 0;
        if ((v & ~((1u << kHashCountBits) - 1)) == tag) return (int)(v & ((1u << kHashCountBits) - 1));
        h = (h + 1) & (cap - 1);
    }
    return 0;
}

// Parameters shared by the sampler kernels of one phase.
struct PhaseArgs {
    int32_t* z;              // [N] word-major topics
    int32_t* prop;           // [N*M] word-major proposals
    const int32_t* perm;     // [N] doc-major position -> word-major index
    const int32_t* seg_off;  // [S+1] token offsets of documents (doc-major) or words
    const float* ckb;        // [K] (float)c_k + beta_bar, frozen for the phase
    int32_t* ck;             // [K] c_k, receives this phase's deltas
    int32_t K, M;
    float g;                 // alpha (document phase) or beta (word phase)
    float G;                 // alpha_bar or K*beta: mixture weight L / (L + G)
    uint32_t iter, k0, k1;   // iteration and Philox key
    int32_t stage_ck;        // 1: c_k table and deltas in shared memory
};

}  // namespace wl
