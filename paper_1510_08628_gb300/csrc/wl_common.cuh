// Device building blocks of the WarpLDA sampler: Philox4x32-10, the FP32
// acceptance and mixture tests, and the per-segment count tables.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wl {

constexpr int kThreads = 256;          // threads of every sampler block
constexpr int kWarps = kThreads / 32;
constexpr int kSegsMax = 512;          // segments (documents / words) per block batch
constexpr int kDocSegs = 128;          // documents per batch of the pipelined document kernel
constexpr int kHashCountBits = 12;     // packed hash entry: (topic + 1) << 12 | count
constexpr int kMaxBatchTokens = 4093;  // count of a packed entry stays below 2^12
constexpr int kDenseMaxK = 2048;       // dense 16-bit count tables up to this K, hash above

enum Phase : uint32_t { kPhaseInit = 0, kPhaseDoc = 1, kPhaseWord = 2 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor bijection.  The Weyl key schedule is precomputed on the host
// (round_keys) and passed in the kernel parameters, so a round costs two
// 32x32->64 multiplies and two 3-input xors.
// ---------------------------------------------------------------------------
struct RoundKeys { uint32_t k[20]; };   // (k0, k1) of rounds 0..9

__host__ __device__ inline RoundKeys round_keys(uint64_t seed) {
    RoundKeys r;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        r.k[2 * i] = k0;
        r.k[2 * i + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return r;
}

__device__ __forceinline__ uint4 philox(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

// The sampler's block for (token t, iteration, phase, MH step i, stream).
__device__ __forceinline__ uint4 draw(uint32_t t, uint32_t iter, uint32_t phase, uint32_t step,
                                      uint32_t stream, const RoundKeys& rk) {
    return philox(make_uint4(t, iter, (phase << 8) | step, stream), rk);
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
    const int32_t* sperm;    // document batches: word-major indices of each batch's tokens,
                             // ascending within the batch (same position range as the batch)
    const uint32_t* sinfo;   // (segment slot << 16) | position within the batch, per sperm entry
    const int32_t* seg_off;  // [S+1] token offsets of documents (doc-major) or words
    const float* ckb;        // [K] (float)c_k + beta_bar, frozen for the phase
    int32_t K, M;
    float g;                 // alpha (document phase) or beta (word phase)
    float G;                 // alpha_bar or K*beta: mixture weight L / (L + G)
    uint32_t iter;           // iteration
    RoundKeys rk;            // Philox key schedule
    int32_t* ck;             // [K] c_k; with stage_ck it receives the phase's deltas
    int32_t word_storage;    // word proposals by positioning in storage order (else j-th smallest)
    int32_t stage_ck;        // 1 (dense tables): c_k table and deltas in shared memory;
                             // 0: kernels leave c_k alone, a histogram pass rebuilds it
    int32_t ck_delta;        // 1 (K above a shared-memory row): kernels add each changed
                             // token's -1 / +1 to c_k in global memory (no histogram pass)
    int64_t N;               // tokens
    int64_t nseg_total;      // documents (document phase) or words (word phase)
    int32_t* fault;          // index-check record {kernel site, 0, check bits, 0}
};

// Work of the multi-pass tier: pieces {count row, segment, first position,
// length} grouped into ranges of consecutive tokens (range r = pieces
// [range_off[r], range_off[r+1])), handed to blocks by a work counter.
struct HugeWork {
    const int4* pieces;
    const int32_t* range_off;
    int nranges, npieces, nrows;
    int guide_bits;          // word draw: log2 of the rank guide table size
    int* counter;
};

// Index checks.  Indices a kernel takes from its work lists (batches, chunks,
// segment table layouts) are validated once per work item; a failed check
// replaces the item by a safe empty one and sets the check's bit in a
// per-thread mask.  Per-token indices (token pointers, topics read back from
// z and the proposals) are in range by construction -- every topic a kernel
// stores is a phase-start topic, a proposal, or a draw in [0, K) -- and are
// validated the same way only in checked builds (-DWL_CHECKED), where a bad
// one is replaced by 0.  Each thread publishes its mask once, when it
// finishes: a.fault = {first kernel site, 0, OR of the masks}; the host reads
// the record at the next synchronising call and reports it as an error.
#ifdef WL_CHECKED
constexpr bool kTokenChecks = true;
#else
constexpr bool kTokenChecks = false;
#endif

struct Checks {
    uint32_t bad = 0;
    __device__ __forceinline__ bool operator()(bool ok, int bit) {
        bad |= ok ? 0u : (1u << bit);
        return ok;
    }
    // per-token check (checked builds)
    __device__ __forceinline__ bool tok(bool ok, int bit) {
        return kTokenChecks ? (*this)(ok, bit) : true;
    }
    // per-token topic: k, or 0 if a checked build finds it outside [0, K)
    __device__ __forceinline__ int topic(int k, int K, int bit) {
        if (!kTokenChecks) return k;
        const bool ok = (uint32_t)k < (uint32_t)K;
        bad |= ok ? 0u : (1u << bit);
        return ok ? k : 0;
    }
    __device__ __forceinline__ void publish(int32_t* fault, int kernel_site) const {
        if (bad != 0) {
            atomicCAS(fault, 0, kernel_site);
            atomicOr(reinterpret_cast<unsigned int*>(fault + 2), bad);
        }
    }
};

// Kernel sites of the check record.
enum : int {
    kSiteDocBatch = 1, kSiteWordBatch = 2, kSiteHugeHist = 3, kSiteHugeAccept = 4,
    kSiteHugeDraw = 5, kSiteDocWarp = 6, kSiteLoglik = 7, kSiteFoldin = 8, kSiteWordCluster = 9
};

}  // namespace wl
