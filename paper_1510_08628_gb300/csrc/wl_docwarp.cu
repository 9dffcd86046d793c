// Warp tier of the document phase (Sec. 4.4): one warp per document of at
// most 32 * TPL tokens.  Each lane holds up to TPL of the document's tokens in
// registers; the document's count table c_d (dense 16-bit counts, or the
// paper's open-addressing hash, Sec. 5.4) and its post-acceptance topics live
// in the warp's own slice of shared memory, so the only synchronisation is
// __syncwarp.  Per token: M chained MH steps with pi^word (Eq. 7) against c_d
// and the phase-start c_k, then M doc proposals by random positioning over the
// post-acceptance document (Sec. 4.3, Eq. 6).  Tokens are reached through perm
// (Sec. 5.2) in the caller's document order, so the positions are the
// oracle's.  The counts of the current state are carried across the chained
// steps instead of being looked up again.
#include <algorithm>

#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

constexpr int kDocsPerGrab = 8;   // documents a warp takes from the work counter at once

int docwarp_table_words(int K, int tpl, int dense) {
    const int w = dense ? (K + 1) / 2 : (int)pow2_above((uint32_t)std::min(64 * tpl, K));
    return (w + 3) & ~3;
}

// words of the staged c_k table and deltas, kept a multiple of 4 so that
// every warp's slice starts 16-byte aligned
__host__ __device__ inline int docwarp_ck_words(int K, int stage_ck) {
    return stage_ck ? ((2 * K + 3) & ~3) : 0;
}

int docwarp_smem_bytes(int K, int stage_ck, int tpl, int dense) {
    return (docwarp_ck_words(K, stage_ck) + kWarps * (docwarp_table_words(K, tpl, dense) + 32 * tpl)) * 4;
}

template <int TPL>
constexpr int docwarp_min_blocks() { return TPL <= 8 ? 4 : 2; }

template <int TPL, int M, bool kDense>
__global__ void __launch_bounds__(kThreads, (docwarp_min_blocks<TPL>())) doc_warp_kernel(
    PhaseArgs a, const int32_t* __restrict__ docs, int ndocs, int* __restrict__ counter,
    int tab_words) {
    extern __shared__ __align__(16) uint32_t dsm[];
    const int K = a.K, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Checks chk;
    float* ckb_s = reinterpret_cast<float*>(dsm);
    int* dck_s = reinterpret_cast<int*>(dsm) + K;   // c_k deltas (with stage_ck)
    uint32_t* wbase = dsm + docwarp_ck_words(K, a.stage_ck) + warp * (tab_words + 32 * TPL);
    uint32_t* tab = wbase;                  // the document's count table
    uint32_t* zst = wbase + tab_words;      // post-acceptance topics, document order
    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    __syncthreads();

    for (;;) {
        int d0 = 0;
        if (lane == 0) d0 = atomicAdd(counter, kDocsPerGrab);
        d0 = __shfl_sync(0xFFFFFFFFu, d0, 0);
        if (d0 >= ndocs) break;
        const int d1 = min(d0 + kDocsPerGrab, ndocs);
        for (int di = d0; di < d1; ++di) {
            int d = docs[di];
            if (!chk(d >= 0 && (int64_t)d < a.nseg_total, 0)) d = 0;
            const int base = a.seg_off[d];
            int L = a.seg_off[d + 1] - base;
            if (!chk(L >= 0 && L <= 32 * TPL, 1)) L = 0;
            const uint32_t cap = kDense ? 0u : pow2_above((uint32_t)min(2 * L, K));
            const int words = kDense ? tab_words : (int)cap;
            for (int i = lane; i < (words >> 2); i += 32)
                reinterpret_cast<uint4*>(tab)[i] = make_uint4(0u, 0u, 0u, 0u);
            for (int i = (words & ~3) + lane; i < words; i += 32) tab[i] = 0u;
            __syncwarp();

            int tk[TPL], zz[TPL];
            int pp[TPL][M];
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
                if (32 * m >= L) break;
                const int j = 32 * m + lane;
                tk[m] = -1;
                if (j < L) {
                    int t = a.perm[base + j];
                    if (!chk.tok((uint32_t)t < (uint32_t)a.N, 2)) t = 0;
                    tk[m] = t;
                    zz[m] = chk.topic(a.z[t], K, 3);
                    if (M == 2) {
                        const int2 x = *reinterpret_cast<const int2*>(a.prop + (int64_t)t * 2);
                        pp[m][0] = x.x;
                        pp[m][1 % M] = x.y;
                    } else {
#pragma unroll
                        for (int i = 0; i < M; ++i) pp[m][i] = a.prop[(int64_t)t * M + i];
                    }
#pragma unroll
                    for (int i = 0; i < M; ++i) pp[m][i] = chk.topic(pp[m][i], K, 4);
                }
            }
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
                if (32 * m >= L) break;
                if (32 * m + lane < L) {
                    if (kDense) atomicAdd(&tab[(uint32_t)zz[m] >> 1], ((uint32_t)zz[m] & 1) ? 65536u : 1u);
                    else table_add(tab, cap, (uint32_t)zz[m]);
                }
            }
            __syncwarp();

            const float Lf = __int2float_rn(L);
            const float LG = __fadd_rn(Lf, a.G);
#pragma unroll
            for (int m = 0; m < TPL; ++m) {
                if (32 * m >= L) break;
                const int j = 32 * m + lane;
                if (j >= L) continue;
                const int z0 = zz[m];
                int s = z0;
                int cs = kDense ? (int)((tab[(uint32_t)s >> 1] >> (((uint32_t)s & 1) * 16)) & 0xFFFFu)
                                : table_get(tab, cap, (uint32_t)s);
                float ks = a.stage_ck ? ckb_s[s] : __ldg(a.ckb + s);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const uint4 r = draw((uint32_t)tk[m], a.iter, kPhaseDoc, (uint32_t)(i + 1), 0u, a.rk);
                    const int t = pp[m][i];
                    if (t != s) {
                        const int ct = kDense ? (int)((tab[(uint32_t)t >> 1] >> (((uint32_t)t & 1) * 16)) & 0xFFFFu)
                                              : table_get(tab, cap, (uint32_t)t);
                        const float kt = a.stage_ck ? ckb_s[t] : __ldg(a.ckb + t);
                        if (accept(r.x, cs, ct, a.g, ks, kt)) {
                            s = t;
                            cs = ct;
                            ks = kt;
                        }
                    }
                    pp[m][i] = coin(r.y, Lf, LG) ? -(int)(dice(r.z, (uint32_t)L) + 1)
                                                 : (int)dice(r.z, (uint32_t)K);
                }
                if (a.stage_ck && s != z0) {
                    atomicSub(&dck_s[z0], 1);
                    atomicAdd(&dck_s[s], 1);
                } else if (a.ck_delta && s != z0) {
                    atomicSub(&a.ck[z0], 1);
                    atomicAdd(&a.ck[s], 1);
                }
                zz[m] = s;
                zst[j] = (uint32_t)s;
            }
            __syncwarp();

#pragma unroll
            for (int m = 0; m < TPL; ++m) {
                if (32 * m >= L) break;
                if (32 * m + lane >= L) continue;
                int out[M];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const int pk = pp[m][i];
                    out[i] = pk < 0 ? (int)zst[-pk - 1] : pk;
                }
                const int t = tk[m];
                if (M == 2) {
                    *reinterpret_cast<int2*>(a.prop + (int64_t)t * 2) = make_int2(out[0], out[1 % M]);
                } else {
#pragma unroll
                    for (int i = 0; i < M; ++i) a.prop[(int64_t)t * M + i] = out[i];
                }
                a.z[t] = zz[m];
            }
            __syncwarp();
        }
    }

    if (a.stage_ck) {
        __syncthreads();
        for (int k = tid; k < K; k += kThreads) {
            const int dv = dck_s[k];
            if (dv != 0) atomicAdd(&a.ck[k], dv);
        }
    }
    chk.publish(a.fault, kSiteDocWarp);
}

template <int TPL, int M, bool kDense>
static const void* dw_ptr() {
    return (const void*)doc_warp_kernel<TPL, M, kDense>;
}

static const void* docwarp_pick(int tpl, int M, bool dense) {
#define WL_D(T, DN)                                                 \
    if (tpl == T && dense == DN) {                                  \
        switch (M) {                                                \
            case 1: return dw_ptr<T, 1, DN>();                      \
            case 2: return dw_ptr<T, 2, DN>();                      \
            case 3: return dw_ptr<T, 3, DN>();                      \
            case 4: return dw_ptr<T, 4, DN>();                      \
            default: return nullptr;                                \
        }                                                           \
    }
    WL_D(8, true) WL_D(8, false) WL_D(16, true) WL_D(16, false)
#undef WL_D
    return nullptr;
}

int docwarp_blocks_per_sm(int K, int stage_ck, int tpl, int M, int dense) {
    const int smem = docwarp_smem_bytes(K, stage_ck, tpl, dense);
    const void* f = docwarp_pick(tpl, M, dense != 0);
    if (!f) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_doc_warp(int tpl, bool dense, const PhaseArgs& a, const int32_t* docs, int ndocs,
                            int* counter, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (ndocs <= 0) return cudaSuccess;
    const int smem = docwarp_smem_bytes(a.K, a.stage_ck, tpl, dense ? 1 : 0);
    const void* f = docwarp_pick(tpl, a.M, dense);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    PhaseArgs args = a;
    int tab_words = docwarp_table_words(a.K, tpl, dense ? 1 : 0);
    void* params[] = {&args, (void*)&docs, &ndocs, &counter, &tab_words};
    return cudaLaunchKernel(f, dim3(grid), dim3(kThreads), params, (size_t)smem, st);
}

}  // namespace wl
