// Initialisation (Alg. 2: z = Dice(K), proposals = z), the global topic
// count vector c_k (Sec. 2.1; reduced once per phase), token-order export,
// range checks, and the joint log-likelihood of Sec. 6.1.
#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

static int grid_for(int64_t n, int per_block = kThreads, int cap = 152 * 16) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

__global__ void init_z_kernel(int32_t* z, int32_t* prop, int64_t N, int K, int M, RoundKeys rk) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = draw((uint32_t)t, 0u, kPhaseInit, 0u, 0u, rk);
        const int k = (int)dice(r.x, (uint32_t)K);
        z[t] = k;
        for (int i = 0; i < M; ++i) prop[t * M + i] = k;
    }
}

cudaError_t launch_init_z(int32_t* z, int32_t* prop, int64_t N, int K, int M, uint64_t seed,
                          cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (N <= 0) return cudaSuccess;
    init_z_kernel<<<grid_for(N), kThreads, 0, st>>>(z, prop, N, K, M, round_keys(seed));
    return cudaGetLastError();
}

// c_k = histogram of z: per-block histograms in shared memory over 128-bit
// loads, added into c_k once per block.
__global__ void __launch_bounds__(kThreads) topic_hist_kernel(const int32_t* __restrict__ z, int64_t N,
                                                              int32_t* __restrict__ ck, int K) {
    extern __shared__ int h[];
    for (int k = threadIdx.x; k < K; k += blockDim.x) h[k] = 0;
    __syncthreads();
    // topics are in [0, K) by construction; the clamp keeps a corrupt
    // value from addressing outside the histogram
    const uint32_t km = (uint32_t)K - 1u;
    auto add = [&](int v) { atomicAdd(&h[min((uint32_t)v, km)], 1); };
    const int4* zv = reinterpret_cast<const int4*>(z);
    const int64_t n4 = N >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + stride < n4; i += 2 * stride) {
        const int4 a = zv[i], b = zv[i + stride];
        add(a.x); add(a.y); add(a.z); add(a.w);
        add(b.x); add(b.y); add(b.z); add(b.w);
    }
    for (; i < n4; i += stride) {
        const int4 a = zv[i];
        add(a.x); add(a.y); add(a.z); add(a.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < (N & 3)) add(z[(n4 << 2) + threadIdx.x]);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (h[k]) atomicAdd(&ck[k], h[k]);
}

// above this K the histogram is kept in global memory
constexpr int kTopicHistSmemMaxK = 24 * 1024;

int topic_hist_blocks_per_sm(int K) {
    if (K > kTopicHistSmemMaxK) return 8;
    const int smem = K * 4;
    if (cudaFuncSetAttribute(topic_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, topic_hist_kernel, kThreads, smem) != cudaSuccess)
        return 0;
    return n;
}

// c_k = histogram of z for K too large for a shared-memory histogram: global
// atomics (topics are spread over K addresses).
__global__ void topic_hist_global_kernel(const int32_t* __restrict__ z, int64_t N, int32_t* __restrict__ ck, int K) {
    const uint32_t km = (uint32_t)K - 1u;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&ck[min((uint32_t)z[t], km)], 1);
}

cudaError_t launch_topic_hist(const int32_t* z, int64_t N, int32_t* ck, int K, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    cudaError_t e = cudaMemsetAsync(ck, 0, sizeof(int32_t) * K, st);
    if (e != cudaSuccess || N <= 0) return e;
    if (K > kTopicHistSmemMaxK) {
        topic_hist_global_kernel<<<grid_for(N), kThreads, 0, st>>>(z, N, ck, K);
        return cudaGetLastError();
    }
    const int smem = K * 4;
    e = cudaFuncSetAttribute(topic_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    topic_hist_kernel<<<grid, kThreads, smem, st>>>(z, N, ck, K);
    return cudaGetLastError();
}

// ckb[k] = (float)c_k + beta_bar (one FP32 RN add), and the block-batch
// counters of the next phase return to zero.
__global__ void finalize_ck_kernel(const int32_t* ck, float* ckb, int K, float beta_bar,
                                   int32_t* counters, int ncounters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) ckb[i] = __fadd_rn(__int2float_rn(ck[i]), beta_bar);
    if (i < ncounters) counters[i] = 0;
}

cudaError_t launch_finalize_ck(const int32_t* ck, float* ckb, int K, float beta_bar,
                               int32_t* counters, int ncounters, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    const int n = K > ncounters ? K : ncounters;
    finalize_ck_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(ck, ckb, K, beta_bar,
                                                                           counters, ncounters);
    return cudaGetLastError();
}

__global__ void zero_kernel(int4* p, int64_t n4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_int4(0, 0, 0, 0);
}

// n must be a multiple of 4 and p 16-byte aligned (row arrays are padded).
cudaError_t launch_zero(int32_t* p, int64_t n, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (n <= 0) return cudaSuccess;
    zero_kernel<<<grid_for(n / 4), kThreads, 0, st>>>(reinterpret_cast<int4*>(p), n / 4);
    return cudaGetLastError();
}

__global__ void gather_kernel(const int32_t* z, const int32_t* perm, int64_t N, int32_t* out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = z[perm[p]];
}

cudaError_t launch_gather_docmajor(const int32_t* z, const int32_t* perm, int64_t N, int32_t* out,
                                   cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (N <= 0) return cudaSuccess;
    gather_kernel<<<grid_for(N), kThreads, 0, st>>>(z, perm, N, out);
    return cudaGetLastError();
}

__global__ void check_range_kernel(const int32_t* v, int64_t n, int K, int32_t* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (v[i] < 0 || v[i] >= K) atomicAdd(bad, 1);
}

cudaError_t launch_check_range(const int32_t* v, int64_t n, int K, int32_t* bad, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (n <= 0) return cudaSuccess;
    check_range_kernel<<<grid_for(n), kThreads, 0, st>>>(v, n, K, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Log-likelihood (Sec. 6.1), FP64:
//   sum_d [lnG(abar) - lnG(abar + L_d)] + sum_{d,k: C_dk>0} [lnG(alpha + C_dk) - lnG(alpha)]
// + sum_k [lnG(bbar) - lnG(bbar + C_k)] + sum_{w,k: C_wk>0} [lnG(beta + C_wk) - lnG(beta)]
// The per-segment count terms reuse the block batches (tables in shared
// memory) and, for long segments, the count rows of the multi-pass tier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kWarps; ++i) s += red[i];
    __syncthreads();
    return s;
}

int loglik_smem_bytes(int region_words) { return (3 * kSegsMax + 4 + region_words) * 4; }

__global__ void __launch_bounds__(kThreads) loglik_batch_kernel(bool doc, const int32_t* z, const int32_t* perm,
                                                                const int32_t* seg_off, const int4* batches,
                                                                int nbatch, int K, double g, int region_words,
                                                                int64_t N, int64_t nseg_total, int32_t* fault,
                                                                double* out) {
    extern __shared__ __align__(16) int lsm[];
    int* seg_tok = lsm;
    int* seg_reg = seg_tok + kSegsMax + 1;
    int* seg_cap = seg_reg + kSegsMax;
    uint32_t* region = reinterpret_cast<uint32_t*>(seg_cap + kSegsMax + 3);
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total;
    __shared__ double red[kWarps];
    const int tid = threadIdx.x;
    const double lg0 = lgamma(g);
    double acc = 0.0;
    Checks chk;
    for (int b = blockIdx.x; b < nbatch; b += gridDim.x) {
        int4 br = batches[b];
        if (!chk(br.x >= 0 && br.y > br.x && br.y - br.x <= kSegsMax && br.y <= nseg_total, 0))
            br = make_int4(0, 0, 0, 0);
        const int nseg = br.y - br.x;
        const int base = seg_off[br.x];
        int end = seg_off[br.y];
        for (int s = tid; s < nseg; s += kThreads) {
            const int o0 = seg_off[br.x + s], o1 = seg_off[br.x + s + 1];
            uint32_t w, cap;
            table_shape((uint32_t)(o1 - o0), (uint32_t)K, &w, &cap);
            seg_tok[s] = o0 - base;
            seg_reg[s] = (int)w;
            seg_cap[s] = (int)cap;
        }
        if (tid == 0) seg_tok[nseg] = end - base;
        __syncthreads();
        block_scan_array(seg_reg, nseg, warp_tot, &s_total);
        int used = s_total;
        if (!chk(used <= region_words, 1)) {
            used = 0;   // the batch's tables do not fit: skip it
            end = base;
        }
        for (int i = tid; i < used; i += kThreads) region[i] = 0u;
        __syncthreads();
        for (int p = base + tid; p < end; p += kThreads) {
            const int t = doc ? perm[p] : p;
            if (!chk.tok(t >= 0 && t < N, 2)) continue;
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_tok[mid] <= p - base) lo = mid; else hi = mid - 1;
            }
            table_add(region + seg_reg[lo], (uint32_t)seg_cap[lo], (uint32_t)chk.topic(z[t], K, 3));
        }
        __syncthreads();
        // every table word: dense halves or packed hash entries
        for (int s = 0; s < nseg; ++s) {
            const int r0 = seg_reg[s];
            const int r1 = (s + 1 < nseg) ? seg_reg[s + 1] : used;
            const bool dense = seg_cap[s] == 0;
            for (int i = r0 + tid; i < r1; i += kThreads) {
                const uint32_t v = region[i];
                if (dense) {
                    const int c0 = (int)(v & 0xFFFFu), c1 = (int)(v >> 16);
                    if (c0) acc += lgamma(g + c0) - lg0;
                    if (c1) acc += lgamma(g + c1) - lg0;
                } else if (v) {
                    acc += lgamma(g + (int)(v & ((1u << kHashCountBits) - 1))) - lg0;
                }
            }
        }
        __syncthreads();
    }
    const double s = block_sum(acc, red);
    if (tid == 0) atomicAdd(out, s);
    chk.publish(fault, kSiteLoglik);
}

cudaError_t launch_loglik_batches(bool doc, const int32_t* z, const int32_t* perm,
                                  const int32_t* seg_off, const int4* batches, int nbatch, int K,
                                  double g, int region_words, int64_t N, int64_t nseg_total,
                                  int32_t* fault, double* out, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nbatch <= 0) return cudaSuccess;
    const int smem = loglik_smem_bytes(region_words);
    cudaError_t e = cudaFuncSetAttribute(loglik_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    loglik_batch_kernel<<<grid, kThreads, smem, st>>>(doc, z, perm, seg_off, batches, nbatch, K, g,
                                                      region_words, N, nseg_total, fault, out);
    return cudaGetLastError();
}

__global__ void loglik_rows_kernel(const int32_t* rows, int64_t n, double g, double* out) {
    __shared__ double red[kWarps];
    const double lg0 = lgamma(g);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = rows[i];
        if (c) acc += lgamma(g + c) - lg0;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

cudaError_t launch_loglik_rows(const int32_t* rows, int64_t nrows, int K, double g, double* out,
                               cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    const int64_t n = nrows * K;
    if (n <= 0) return cudaSuccess;
    loglik_rows_kernel<<<grid_for(n), kThreads, 0, st>>>(rows, n, g, out);
    return cudaGetLastError();
}

__global__ void loglik_lengths_kernel(const int32_t* seg_off, int64_t nseg, double abar,
                                      double* out) {
    __shared__ double red[kWarps];
    const double la = lgamma(abar);
    double acc = 0.0;
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < nseg;
         d += (int64_t)gridDim.x * blockDim.x)
        acc += la - lgamma(abar + (double)(seg_off[d + 1] - seg_off[d]));
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

cudaError_t launch_loglik_lengths(const int32_t* seg_off, int64_t nseg, double abar, double* out,
                                  cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nseg <= 0) return cudaSuccess;
    loglik_lengths_kernel<<<grid_for(nseg), kThreads, 0, st>>>(seg_off, nseg, abar, out);
    return cudaGetLastError();
}

__global__ void loglik_topics_kernel(const int32_t* ck, int K, double bbar, double* out) {
    __shared__ double red[kWarps];
    const double lb = lgamma(bbar);
    double acc = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
        acc += lb - lgamma(bbar + (double)ck[k]);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

cudaError_t launch_loglik_topics(const int32_t* ck, int K, double bbar, double* out,
                                 cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    loglik_topics_kernel<<<grid_for(K), kThreads, 0, st>>>(ck, K, bbar, out);
    return cudaGetLastError();
}

}  // namespace wl
