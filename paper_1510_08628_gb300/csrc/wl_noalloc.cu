// warplda_loglik_noalloc: the joint log-likelihood (Sec. 6.1) of caller-held
// device buffers, for callers that cannot allocate device memory -- code that
// runs inside a host framework which owns every device allocation (a caching
// allocator or a fixed arena that forbids raw cudaMalloc), or a long-running
// serving process with a fixed device-memory budget where an allocation could
// fail or stall the device.  It needs no context (creating a context
// allocates) and calls no allocating routine.
//
// Its scratch -- the topic-count vector c_k, one FP64 partial sum per block
// and a token counter -- lives in the file-scope array below, which every GPU
// that loads this library holds until the process exits (kNaScratchBytes,
// about 66 KB).
//
// Cost: every document and word clears and scans a K-entry histogram in
// shared memory, so a call does O((D + V) K) shared-memory work besides its
// O(N) reads -- at K = 16384 on a 400K-segment corpus about 6.5G operations.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/warplda.h"
#include "wl_common.cuh"
#include "wl_kernels.h"

namespace {

constexpr int kNaMaxK = 16384;         // largest K this entry point accepts
constexpr int kNaBlocks = 256;         // blocks, one FP64 partial sum each
constexpr size_t kNaScratchBytes =
    (size_t)kNaMaxK * sizeof(int32_t) + (size_t)kNaBlocks * sizeof(double) + 2 * sizeof(unsigned long long);

// [c_k: kNaMaxK int32][partial sums: kNaBlocks double][word tokens: uint64, pad]
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

// failures are reported through warplda_last_error()
int na_fail(int code, const std::string& msg) { return wl::record_error(code, msg.c_str()); }

// Device address of g_na_scratch on the current device (the host-side
// symbol is only a stand-in, not a device address).  Looked up on every call:
// it allocates nothing, and a cached address would go stale if the device's
// context were reset and the module loaded again elsewhere.
int na_scratch(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p)
        return na_fail(WARPLDA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return WARPLDA_OK;
}

__device__ __forceinline__ double na_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// Clears the scratch c_k, partial sums and word-token counter of this call.
__global__ void na_clear_kernel(int32_t* ck, double* part, unsigned long long* wtok, int K) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) ck[i] = 0;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < kNaBlocks; i += blockDim.x) part[i] = 0.0;
        if (threadIdx.x == 0) *wtok = 0ull;
    }
}

// One block per segment at a time (documents 0..D-1, then words): the
// segment's topic histogram in shared memory, then
//   documents: lnG(abar) - lnG(abar + L_d) + sum_k [lnG(alpha + C_dk) - lnG(alpha)]
//   words:     sum_k [lnG(beta + C_wk) - lnG(beta)]
// Document tokens also add into the scratch c_k, and the words' token counts
// into the word-token counter.  Each block writes its own partial sum;
// nothing is accumulated across blocks in floating point.
__global__ void __launch_bounds__(wl::kThreads) na_segments_kernel(
    int64_t D, int64_t V, int K, double alpha, double beta, double abar,
    const int64_t* __restrict__ doc_ptr, const int32_t* __restrict__ z_doc,
    const int64_t* __restrict__ word_ptr, const int32_t* __restrict__ z_word,
    int32_t* __restrict__ ck, double* __restrict__ part, unsigned long long* __restrict__ wtok) {
    extern __shared__ int hist[];
    __shared__ double red[wl::kWarps];
    const double la = lgamma(alpha), lb = lgamma(beta), lab = lgamma(abar);
    double acc = 0.0;
    unsigned long long words = 0;
    for (int64_t s = blockIdx.x; s < D + V; s += gridDim.x) {
        const bool doc = s < D;
        const int64_t b = doc ? doc_ptr[s] : word_ptr[s - D];
        const int64_t e = doc ? doc_ptr[s + 1] : word_ptr[s - D + 1];
        const int32_t* z = doc ? z_doc : z_word;
        for (int k = threadIdx.x; k < K; k += blockDim.x) hist[k] = 0;
        __syncthreads();
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            const int k = z[p];
            if ((uint32_t)k >= (uint32_t)K) {   // not a topic: the result becomes NaN
                acc = __longlong_as_double(0x7FF8000000000000ll);
                continue;
            }
            atomicAdd(&hist[k], 1);
            if (doc) atomicAdd(&ck[k], 1);
        }
        __syncthreads();
        const double g = doc ? alpha : beta, lg = doc ? la : lb;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const int c = hist[k];
            if (c) acc += lgamma(g + c) - lg;
        }
        if (doc && threadIdx.x == 0) acc += lab - lgamma(abar + (double)(e - b));
        if (!doc && threadIdx.x == 0) words += (unsigned long long)(e - b);
        __syncthreads();
    }
    const double tot = na_block_sum(acc, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        if (words) atomicAdd(wtok, words);
    }
}

// Topic terms sum_k [lnG(bbar) - lnG(bbar + C_k)] plus the block partials, in
// a fixed order; one block.  The document tokens (sum of c_k) and the word
// tokens must both equal N, else the result is NaN.
__global__ void na_final_kernel(const int32_t* __restrict__ ck, const double* __restrict__ part,
                                const unsigned long long* __restrict__ wtok, int K, int64_t N,
                                double bbar, double* __restrict__ out) {
    __shared__ double red[wl::kWarps];
    const double lbb = lgamma(bbar);
    double acc = 0.0, ntok = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        acc += lbb - lgamma(bbar + (double)ck[k]);
        ntok += (double)ck[k];   // exact: integers below 2^53
    }
    for (int i = threadIdx.x; i < kNaBlocks; i += blockDim.x) acc += part[i];
    const double tot = na_block_sum(acc, red);
    const double n = na_block_sum(ntok, red);
    if (threadIdx.x == 0)
        *out = (n == (double)N && *wtok == (unsigned long long)N) ? tot : __longlong_as_double(0x7FF8000000000000ll);
}

}  // namespace

extern "C" int warplda_loglik_noalloc(int64_t D, int64_t V, int64_t N, int32_t K, float alpha,
                                      float beta, const int64_t* doc_ptr_dev,
                                      const int32_t* z_docmajor_dev, const int64_t* word_ptr_dev,
                                      const int32_t* z_wordmajor_dev, double* out_dev,
                                      void* cuda_stream) try {
    if (D < 0 || V < 1 || N < 0 || N > (int64_t)0x7FFFFFF0)
        return na_fail(WARPLDA_EINVAL, "need D >= 0, V >= 1 and 0 <= N < 2^31");
    if (K < 1 || K > kNaMaxK)
        return na_fail(WARPLDA_EINVAL, "K must be in [1, " + std::to_string(kNaMaxK) +
                                           "] for warplda_loglik_noalloc (its scratch holds that many topic counts)");
    if (!(alpha > 0.0f) || !(beta > 0.0f) || !std::isfinite(alpha) || !std::isfinite(beta))
        return na_fail(WARPLDA_EINVAL, "alpha and beta must be > 0");
    if (!doc_ptr_dev || !word_ptr_dev || !out_dev || (N > 0 && (!z_docmajor_dev || !z_wordmajor_dev)))
        return na_fail(WARPLDA_EINVAL, "null device pointer");
    void* scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc) return rc;
    int32_t* ck = reinterpret_cast<int32_t*>(scratch);
    double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) +
                                             (size_t)kNaMaxK * sizeof(int32_t));
    unsigned long long* wtok = reinterpret_cast<unsigned long long*>(part + kNaBlocks);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double a = alpha, b = beta;
    const int smem = K * (int)sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(na_segments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        na_clear_kernel<<<16, wl::kThreads, 0, st>>>(ck, part, wtok, K);
        na_segments_kernel<<<kNaBlocks, wl::kThreads, smem, st>>>(D, V, K, a, b, (double)K * a, doc_ptr_dev,
                                                                  z_docmajor_dev, word_ptr_dev,
                                                                  z_wordmajor_dev, ck, part, wtok);
        na_final_kernel<<<1, wl::kThreads, 0, st>>>(ck, part, wtok, K, N, (double)V * b, out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return na_fail(WARPLDA_ECUDA, std::string("warplda_loglik_noalloc: ") + cudaGetErrorString(e));
    return WARPLDA_OK;
} catch (...) {
    // only the error messages allocate on the host; no exception crosses the C ABI
    return wl::record_error(WARPLDA_ENOMEM, "warplda_loglik_noalloc: host allocation failed");
}
