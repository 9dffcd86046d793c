// Multi-pass tier of the document and word phases for segments with more
// tokens than one block batch holds (the paper's intra-word parallelism for
// frequent words, Sec. 5.4).  The segment's tokens are split into chunks that
// many blocks process concurrently; the per-segment count row (K ints) lives
// in global memory (L2-resident) and is completed between passes:
//   hist   : row_pre  = histogram of the phase-start z of the segment
//   accept : M chained MH steps per token against row_pre (Eq. 7), z written;
//            word phase also builds row_post = histogram of the new z
//   draw   : M proposals per token from Eq. 6 -- positioning through perm
//            over the post-acceptance document, or the j-th smallest
//            post-acceptance topic of the word (inverse CDF of row_post).
// The draw pass recomputes the Philox blocks of the accept pass.
#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

// Warp-aggregated increment of h[k]: lanes holding the same k add once.
__device__ __forceinline__ void agg_add(int* h, int k) {
    const unsigned act = __activemask();
    const unsigned m = __match_any_sync(act, k);
    const int lane = threadIdx.x & 31;
    if (lane == __ffs(m) - 1) atomicAdd(&h[k], __popc(m));
}

int huge_smem_bytes(int K, int stage_ck, int pass, bool doc) {
    // pass 0 hist: K; pass 1 accept: row + (word) hist + staged ck; pass 2 draw: K+1 prefix
    int words = 0;
    if (pass == 0) words = K;
    else if (pass == 1) words = K + (doc ? 0 : K) + (stage_ck ? 2 * K : 0);
    else words = doc ? 0 : K + 1;
    return ((words * 4) + 15) & ~15;
}

template <bool kDoc>
__global__ void __launch_bounds__(kThreads) huge_hist_kernel(PhaseArgs a, const int4* __restrict__ chunks,
                                                             int nchunks, int32_t* __restrict__ rows) {
    extern __shared__ __align__(16) int hist[];
    const int K = a.K, tid = threadIdx.x;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        for (int k = tid; k < K; k += kThreads) hist[k] = 0;
        __syncthreads();
        for (int p = ch.z + tid; p < ch.z + ch.w; p += kThreads) {
            const int t = kDoc ? a.perm[p] : p;
            agg_add(hist, a.z[t]);
        }
        __syncthreads();
        int32_t* row = rows + (int64_t)ch.x * K;
        for (int k = tid; k < K; k += kThreads)
            if (hist[k] != 0) atomicAdd(&row[k], hist[k]);
        __syncthreads();
    }
}

template <bool kDoc, int M>
__global__ void __launch_bounds__(kThreads) huge_accept_kernel(PhaseArgs a, const int4* __restrict__ chunks,
                                                               int nchunks, const int32_t* __restrict__ rows_pre,
                                                               int32_t* __restrict__ rows_post) {
    extern __shared__ __align__(16) int sm[];
    const int K = a.K, tid = threadIdx.x;
    int* row = sm;
    int* hist = sm + K;                                    // word phase only
    float* ckb_s = reinterpret_cast<float*>(sm + (kDoc ? K : 2 * K));
    int* dck_s = sm + (kDoc ? 2 * K : 3 * K);
    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        const int32_t* rp = rows_pre + (int64_t)ch.x * K;
        for (int k = tid; k < K; k += kThreads) {
            row[k] = rp[k];
            if (!kDoc) hist[k] = 0;
        }
        __syncthreads();
        for (int p = ch.z + tid; p < ch.z + ch.w; p += kThreads) {
            const int t = kDoc ? a.perm[p] : p;
            const int z0 = a.z[t];
            int pr[M];
#pragma unroll
            for (int i = 0; i < M; ++i) pr[i] = a.prop[(int64_t)t * M + i];
            int s = z0;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const int tp = pr[i];
                if (tp != s) {
                    const uint4 r = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.k0, a.k1);
                    const float cs = a.stage_ck ? ckb_s[s] : __ldg(a.ckb + s);
                    const float ct = a.stage_ck ? ckb_s[tp] : __ldg(a.ckb + tp);
                    if (accept(r.x, row[s], row[tp], a.g, cs, ct)) s = tp;
                }
            }
            if (s != z0) {
                a.z[t] = s;
                if (a.stage_ck) {
                    atomicSub(&dck_s[z0], 1);
                    atomicAdd(&dck_s[s], 1);
                } else {
                    atomicSub(&a.ck[z0], 1);
                    atomicAdd(&a.ck[s], 1);
                }
            }
            if (!kDoc) agg_add(hist, s);
        }
        __syncthreads();
        if (!kDoc) {
            int32_t* rq = rows_post + (int64_t)ch.x * K;
            for (int k = tid; k < K; k += kThreads)
                if (hist[k] != 0) atomicAdd(&rq[k], hist[k]);
        }
        __syncthreads();
    }
    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads)
            if (dck_s[k] != 0) atomicAdd(&a.ck[k], dck_s[k]);
    }
}

template <bool kDoc, int M>
__global__ void __launch_bounds__(kThreads) huge_draw_kernel(PhaseArgs a, const int4* __restrict__ chunks,
                                                             int nchunks, const int32_t* __restrict__ rows_post) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total;
    const int K = a.K, tid = threadIdx.x;
    int* P = sm;   // word phase: exclusive prefix of row_post, P[K] = L_w
    const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        const int sb = a.seg_off[ch.y];
        const int Ls = a.seg_off[ch.y + 1] - sb;
        if (!kDoc) {
            const int32_t* rq = rows_post + (int64_t)ch.x * K;
            int carry = 0;
            for (int k0 = 0; k0 < K; k0 += kThreads) {
                const int k = k0 + tid;
                const int v = (k < K) ? rq[k] : 0;
                const int e = block_excl_scan(v, warp_tot, &s_total);
                if (k < K) P[k] = carry + e;
                carry += s_total;
            }
            if (tid == 0) P[K] = carry;
        }
        __syncthreads();
        const float Lf = __int2float_rn(Ls);
        const float LG = __fadd_rn(Lf, a.G);
        for (int p = ch.z + tid; p < ch.z + ch.w; p += kThreads) {
            const int t = kDoc ? a.perm[p] : p;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const uint4 r = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.k0, a.k1);
                int k;
                if (coin(r.y, Lf, LG)) {
                    const int j = (int)dice(r.z, (uint32_t)Ls);
                    if (kDoc) {
                        k = a.z[a.perm[sb + j]];
                    } else {
                        // largest k with P[k] <= j: the j-th smallest topic
                        int lo = 0, hi = K - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (P[mid] <= j) lo = mid; else hi = mid - 1;
                        }
                        k = lo;
                    }
                } else {
                    k = (int)dice(r.z, (uint32_t)a.K);
                }
                a.prop[(int64_t)t * M + i] = k;
            }
        }
        __syncthreads();
    }
}

template <typename F>
static cudaError_t set_smem(F f, int smem) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_huge_hist(bool doc, const PhaseArgs& a, const int4* chunks, int nchunks,
                             int32_t* rows, int grid, cudaStream_t st) {
    if (nchunks <= 0) return cudaSuccess;
    const int smem = huge_smem_bytes(a.K, a.stage_ck, 0, doc);
    if (doc) {
        cudaError_t e = set_smem(huge_hist_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        huge_hist_kernel<true><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows);
    } else {
        cudaError_t e = set_smem(huge_hist_kernel<false>, smem);
        if (e != cudaSuccess) return e;
        huge_hist_kernel<false><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows);
    }
    return cudaGetLastError();
}

#define WL_M_SWITCH(...)          \
    switch (a.M) {                \
        case 1: { constexpr int MM = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int MM = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int MM = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int MM = 4; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;           \
    }

cudaError_t launch_huge_accept(bool doc, const PhaseArgs& a, const int4* chunks, int nchunks,
                               const int32_t* rows_pre, int32_t* rows_post, int grid,
                               cudaStream_t st) {
    if (nchunks <= 0) return cudaSuccess;
    const int smem = huge_smem_bytes(a.K, a.stage_ck, 1, doc);
    cudaError_t e = cudaSuccess;
    if (doc) {
        WL_M_SWITCH({
            e = set_smem(huge_accept_kernel<true, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_accept_kernel<true, MM><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows_pre, rows_post);
        })
    } else {
        WL_M_SWITCH({
            e = set_smem(huge_accept_kernel<false, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_accept_kernel<false, MM><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows_pre, rows_post);
        })
    }
    return cudaGetLastError();
}

cudaError_t launch_huge_draw(bool doc, const PhaseArgs& a, const int4* chunks, int nchunks,
                             const int32_t* rows_post, int grid, cudaStream_t st) {
    if (nchunks <= 0) return cudaSuccess;
    const int smem = huge_smem_bytes(a.K, a.stage_ck, 2, doc);
    cudaError_t e = cudaSuccess;
    if (doc) {
        WL_M_SWITCH({
            e = set_smem(huge_draw_kernel<true, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_draw_kernel<true, MM><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows_post);
        })
    } else {
        WL_M_SWITCH({
            e = set_smem(huge_draw_kernel<false, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_draw_kernel<false, MM><<<grid, kThreads, smem, st>>>(a, chunks, nchunks, rows_post);
        })
    }
    return cudaGetLastError();
}

int huge_blocks_per_sm(int K, int stage_ck, int pass, bool doc, int M) {
    const int smem = huge_smem_bytes(K, stage_ck, pass, doc);
    const void* f = nullptr;
    if (pass == 0) f = doc ? (const void*)huge_hist_kernel<true> : (const void*)huge_hist_kernel<false>;
#define WL_P(P, KER)                                                                   \
    if (pass == P) {                                                                   \
        if (M == 1) f = doc ? (const void*)KER<true, 1> : (const void*)KER<false, 1>;  \
        if (M == 2) f = doc ? (const void*)KER<true, 2> : (const void*)KER<false, 2>;  \
        if (M == 3) f = doc ? (const void*)KER<true, 3> : (const void*)KER<false, 3>;  \
        if (M == 4) f = doc ? (const void*)KER<true, 4> : (const void*)KER<false, 4>;  \
    }
    WL_P(1, huge_accept_kernel)
    WL_P(2, huge_draw_kernel)
#undef WL_P
    if (!f) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace wl
