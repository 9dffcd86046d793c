// Token store build on the device (Sec. 5.2): the word-major order of the
// tokens and the pointer array P between the two orders, and the document
// batches' lists of their tokens in word-major order.
//
//   word_check_kernel     the first token whose word id is outside [0, V).
//   radix_count_kernel /  one pass of a stable LSD radix sort (digits of up
//   radix_scatter_kernel  to 9 bits; two passes for up to 2^18 words) of
//                         (word id, doc-major position) pairs: per-tile
//                         digit counts, a device-wide exclusive scan in
//                         digit-major order, then each tile writes its pairs
//                         at their digit's offset plus their stable rank.
//                         After the passes the positions are in word-major
//                         order, ties (same word) in doc-major order.
//   word_starts_kernel    the first word-major index of each word present
//                         (the word offsets, read off the sorted word ids).
//   perm_kernel           perm[p] = word-major index of doc-major position p.
//   batch_lists_kernel    one block per document batch: the batch's word-major
//                         indices sorted ascending (block radix sort) with
//                         (document slot << 16 | position within the batch).
#include <algorithm>

#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

constexpr int kSortItems = 16;                      // items per thread of a tile
constexpr int kSortTile = kThreads * kSortItems;    // 4096 pairs per tile
constexpr int kScanChunk = kThreads * 16;           // entries per block of the scan
constexpr int kDigitBitsMax = 9;
constexpr int kBinsMax = 1 << kDigitBitsMax;

// The first position whose word id is outside [0, V) goes to *bad
// (initialised to INT_MAX by the caller).
__global__ void word_check_kernel(const int32_t* __restrict__ w, int64_t N, int32_t V, int32_t* __restrict__ bad) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        if ((uint32_t)w[t] >= (uint32_t)V) atomicMin(bad, (int32_t)t);
}

// start[w] = first index of word w in the sorted word ids (start is -1 for
// words without tokens; set by the caller).
__global__ void word_starts_kernel(const int32_t* __restrict__ keys, int64_t N, int32_t V,
                                   int32_t* __restrict__ start) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = keys[i];
        if ((i == 0 || keys[i - 1] != w) && (uint32_t)w < (uint32_t)V) start[w] = (int32_t)i;
    }
}

// tile_cnt[digit * ntiles + tile] = the tile's keys with that digit.
__global__ void __launch_bounds__(kThreads) radix_count_kernel(const int32_t* __restrict__ keys, int64_t n,
                                                               int shift, int bits, int32_t* __restrict__ tile_cnt,
                                                               int64_t ntiles) {
    __shared__ int h[kBinsMax];
    const int nbins = 1 << bits;
    const uint32_t mask = (uint32_t)nbins - 1u;
    for (int d = threadIdx.x; d < nbins; d += kThreads) h[d] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = t0 + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[((uint32_t)keys[i] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += kThreads) tile_cnt[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Exclusive scan of int32 data in place, in chunks of kScanChunk: chunk sums,
// a scan of the sums (one block, or recursively), then the chunks.
__global__ void __launch_bounds__(kThreads) scan_sums_kernel(const int32_t* __restrict__ d, int64_t n,
                                                             int32_t* __restrict__ sums) {
    __shared__ int warp_tot[kWarps];
    __shared__ int total;
    const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
    int s = 0;
    for (int j = threadIdx.x; j < kScanChunk; j += kThreads) {
        const int64_t i = c0 + j;
        if (i < n) s += d[i];
    }
    block_excl_scan(s, warp_tot, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) scan_chunks_kernel(int32_t* __restrict__ d, int64_t n,
                                                               const int32_t* __restrict__ offs) {
    __shared__ int warp_tot[kWarps];
    __shared__ int total;
    const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
    // thread i scans the 16 consecutive entries [16i, 16i + 16) of the chunk
    int v[16];
    int s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int64_t i = c0 + threadIdx.x * 16 + j;
        v[j] = i < n ? d[i] : 0;
        s += v[j];
    }
    int run = block_excl_scan(s, warp_tot, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int64_t i = c0 + threadIdx.x * 16 + j;
        if (i < n) d[i] = run;
        run += v[j];
    }
}

static cudaError_t scan_exclusive(int32_t* d, int64_t n, int32_t* tmp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb == 1) {
        scan_chunks_kernel<<<1, kThreads, 0, st>>>(d, n, nullptr);
        return cudaGetLastError();
    }
    scan_sums_kernel<<<(unsigned)nb, kThreads, 0, st>>>(d, n, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive(tmp, nb, tmp + nb, st);   // the sums' own scratch follows them
    if (e != cudaSuccess) return e;
    scan_chunks_kernel<<<(unsigned)nb, kThreads, 0, st>>>(d, n, tmp);
    return cudaGetLastError();
}

// Scratch words the scan of n entries needs (all recursion levels).
static int64_t scan_scratch(int64_t n) {
    int64_t s = 0;
    while (n > 1) {
        n = (n + kScanChunk - 1) / kScanChunk;
        s += n;
    }
    return s + 1;
}

// Stable scatter of one pass.  A tile's pairs go in 16 rounds of 256 (pair
// index = tile * 4096 + round * 256 + thread, so rounds, warps and lanes are
// in index order); within a warp, lanes with the same digit rank by lane;
// per-warp digit counts become per-warp bases by a scan over the warps, and
// a per-digit running base carries across rounds.
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const int32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n, int shift, int bits,
    const int32_t* __restrict__ tile_off, int64_t ntiles, int32_t* __restrict__ kout, int32_t* __restrict__ vout) {
    __shared__ int wc[kWarps][kBinsMax];
    __shared__ int wb[kWarps][kBinsMax];
    __shared__ int run[kBinsMax];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbins = 1 << bits;
    const uint32_t mask = (uint32_t)nbins - 1u;
    for (int d = tid; d < nbins; d += kThreads) {
        for (int w = 0; w < kWarps; ++w) wc[w][d] = 0;
        run[d] = tile_off[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = t0 + r * kThreads + tid;
        const bool ok = i < n;
        const int32_t key = ok ? kin[i] : 0;
        const int32_t val = ok ? (vin ? vin[i] : (int32_t)i) : 0;
        const int d = ok ? (int)(((uint32_t)key >> shift) & mask) : nbins + lane;   // padding matches nothing
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int wrank = __popc(peers & lt);
        if (ok && wrank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        for (int dd = tid; dd < nbins; dd += kThreads) {
            int acc = run[dd];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int c = wc[w][dd];
                wb[w][dd] = acc;
                wc[w][dd] = 0;
                acc += c;
            }
            run[dd] = acc;
        }
        __syncthreads();
        if (ok) {
            const int pos = wb[warp][d] + wrank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

__global__ void perm_kernel(const int32_t* __restrict__ pos_sorted, int64_t N, int32_t* __restrict__ perm) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        perm[pos_sorted[t]] = (int32_t)t;
}

// One block per document batch {first doc, end doc, table words, 0}: its
// tokens occupy doc-major positions [doc_off[x], doc_off[y]) and the same
// range of sperm / sinfo.
template <int kTPT>
__global__ void __launch_bounds__(kThreads) batch_lists_kernel(
    const int4* __restrict__ batches, int nb, const int32_t* __restrict__ doc_off, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ pos_sorted, int nbits, int32_t* __restrict__ sperm, uint32_t* __restrict__ sinfo,
    int32_t* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned char bsm[];
    uint32_t* keys = reinterpret_cast<uint32_t*>(bsm);
    uint16_t* cnt = reinterpret_cast<uint16_t*>(bsm + (kThreads * kTPT + (kThreads * kTPT >> 5) + 4) * 4);
    __shared__ int warp_tot[kWarps];
    __shared__ int total;
    const int tid = threadIdx.x;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int4 br = batches[b];
        const int x = br.x, y = br.y;
        const int b0 = doc_off[x], b1 = doc_off[y];
        const int n = b1 - b0;
        if (n < 0 || n > kThreads * kTPT || y - x > kSegsMax) {   // built on the host; never taken
            if (tid == 0) atomicMin(bad, b);
            continue;
        }
        for (int p = tid; p < kThreads * kTPT; p += kThreads)
            keys[pad(p)] = p < n ? (uint32_t)perm[b0 + p] : 0xFFFFFFFFu;
        __syncthreads();
        block_radix_sort<kTPT>(keys, cnt, nbits, warp_tot, &total);
        __syncthreads();
        for (int p = tid; p < n; p += kThreads) {
            const int t = (int)keys[pad(p)];
            const int q = pos_sorted[t];          // doc-major position of the token
            int lo = x, hi = y - 1;               // its document: last d with doc_off[d] <= q
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (doc_off[mid] <= q) lo = mid; else hi = mid - 1;
            }
            sperm[b0 + p] = t;
            sinfo[b0 + p] = ((uint32_t)(lo - x) << 16) | (uint32_t)(q - b0);
        }
        __syncthreads();
    }
}

int64_t token_sort_scratch(int64_t N) {
    const int64_t ntiles = std::max<int64_t>(1, (N + kSortTile - 1) / kSortTile);
    return kBinsMax * ntiles + scan_scratch(kBinsMax * ntiles) + 4;
}

cudaError_t launch_scan_exclusive(int32_t* d, int64_t n, int32_t* tmp, cudaStream_t st) {
    return scan_exclusive(d, n, tmp, st);
}

int64_t scan_scratch_words(int64_t n) { return scan_scratch(n); }

cudaError_t launch_word_check(const int32_t* w, int64_t N, int32_t V, int32_t* bad, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (N <= 0) return cudaSuccess;
    const int64_t g = std::min<int64_t>((N + kThreads - 1) / kThreads, 152 * 16);
    word_check_kernel<<<(unsigned)g, kThreads, 0, st>>>(w, N, V, bad);
    return cudaGetLastError();
}

cudaError_t launch_word_starts(const int32_t* keys_sorted, int64_t N, int32_t V, int32_t* start, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    cudaError_t e = cudaMemsetAsync(start, 0xFF, sizeof(int32_t) * (size_t)V, st);
    if (e != cudaSuccess || N <= 0) return e;
    const int64_t g = std::min<int64_t>((N + kThreads - 1) / kThreads, 152 * 16);
    word_starts_kernel<<<(unsigned)g, kThreads, 0, st>>>(keys_sorted, N, V, start);
    return cudaGetLastError();
}

static int key_bits(int64_t V) {
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < V) ++bits;
    return std::max(1, bits);
}

int token_sort_passes(int64_t V) { return (key_bits(V) + kDigitBitsMax - 1) / kDigitBitsMax; }

cudaError_t launch_token_sort(int32_t* keys_a, int32_t* vals_a, int32_t* keys_b, int32_t* vals_b, int64_t N,
                              int32_t V, int32_t* scratch, int32_t** pos_sorted, int32_t** keys_sorted,
                              cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    *pos_sorted = nullptr;
    *keys_sorted = nullptr;
    if (N <= 0) return cudaSuccess;
    const int64_t ntiles = (N + kSortTile - 1) / kSortTile;
    const int passes = token_sort_passes(V);
    // the key bits split evenly over the passes (the last takes what is left)
    const int bits = (key_bits(V) + passes - 1) / passes;
    int32_t* tile = scratch;
    int32_t* tmp = scratch + kBinsMax * ntiles;
    const int32_t* kin = keys_a;
    const int32_t* vin = nullptr;   // first pass: values are the positions
    int32_t* kout = keys_b;
    int32_t* vout = vals_b;
    for (int p = 0; p < passes; ++p) {
        const int shift = bits * p, pb = std::min(bits, key_bits(V) - shift);
        radix_count_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(kin, N, shift, pb, tile, ntiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if ((e = scan_exclusive(tile, ((int64_t)1 << pb) * ntiles, tmp, st)) != cudaSuccess) return e;
        radix_scatter_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(kin, vin, N, shift, pb, tile, ntiles, kout, vout);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *pos_sorted = vout;
        *keys_sorted = kout;
        // next pass reads what this one wrote
        int32_t* nk = (kout == keys_b) ? keys_a : keys_b;
        int32_t* nv = (vout == vals_b) ? vals_a : vals_b;
        kin = kout;
        vin = vout;
        kout = nk;
        vout = nv;
    }
    return cudaSuccess;
}

cudaError_t launch_perm(const int32_t* pos_sorted, int64_t N, int32_t* perm, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (N <= 0) return cudaSuccess;
    const int64_t g = std::min<int64_t>((N + kThreads - 1) / kThreads, 152 * 16);
    perm_kernel<<<(unsigned)g, kThreads, 0, st>>>(pos_sorted, N, perm);
    return cudaGetLastError();
}

template <int kTPT>
static cudaError_t batch_lists_tpt(const int4* batches, int nb, const int32_t* doc_off, const int32_t* perm,
                                   const int32_t* pos_sorted, int nbits, int32_t* sperm, uint32_t* sinfo,
                                   int32_t* bad, cudaStream_t st) {
    const int smem = (kThreads * kTPT + ((kThreads * kTPT) >> 5) + 4) * 4 + 16 * kThreads * 2;
    cudaError_t e = cudaFuncSetAttribute(batch_lists_kernel<kTPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    batch_lists_kernel<kTPT><<<(unsigned)std::min(nb, 152 * 8), kThreads, smem, st>>>(
        batches, nb, doc_off, perm, pos_sorted, nbits, sperm, sinfo, bad);
    return cudaGetLastError();
}

cudaError_t launch_batch_lists(const int4* batches, int nb, int max_tokens, const int32_t* doc_off,
                               const int32_t* perm, const int32_t* pos_sorted, int64_t N, int32_t* sperm,
                               uint32_t* sinfo, int32_t* bad, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nb <= 0) return cudaSuccess;
    int nbits = 1;
    while (nbits < 32 && ((int64_t)1 << nbits) <= N) ++nbits;   // 2^nbits - 1 >= N > every key
    // the block sorts 256 * TPT keys: the smallest TPT that holds a batch
    if (max_tokens <= kThreads * 4)
        return batch_lists_tpt<4>(batches, nb, doc_off, perm, pos_sorted, nbits, sperm, sinfo, bad, st);
    if (max_tokens <= kThreads * 8)
        return batch_lists_tpt<8>(batches, nb, doc_off, perm, pos_sorted, nbits, sperm, sinfo, bad, st);
    return batch_lists_tpt<16>(batches, nb, doc_off, perm, pos_sorted, nbits, sperm, sinfo, bad, st);
}

}  // namespace wl
