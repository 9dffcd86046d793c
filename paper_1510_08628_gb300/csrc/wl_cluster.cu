// Word phase of heavy words on a thread-block cluster (Sec. 5.4's
// intra-word parallelism, with the count row in distributed shared memory).
//
// A word with more tokens than a block batch holds, but few enough that its
// tokens fit in the shared memory of one cluster, is sampled by one cluster
// of C blocks.  Block r of the cluster holds slice r of the word's tokens
// (its z and M pending proposals) in shared memory for the whole phase:
//   1. each block counts its slice's phase-start topics into a K-wide row;
//      the rows are reduced over the cluster -- each block sums its K/C
//      shard of every block's row through distributed shared memory, then
//      gathers the other shards -- so every block holds the word's C_w;
//   2. M chained MH steps per token against that row (Eq. 7), the picks of
//      Eq. 6 (a topic, or a rank of the post-acceptance word), and the count
//      of the new topics into a second row;
//   3. the post-acceptance rows are reduced the same way; each block turns
//      the word's row into its exclusive prefix and a guide table of ranks,
//      and resolves its picks to the j-th smallest post-acceptance topic
//      (or, with storage-order positioning, reads the j-th token's new topic
//      from the block that holds it);
//   4. z and the proposals go back to HBM once, coalesced.
// Each token is read and written once, where the multi-pass tier reads the
// word's tokens four times (histogram, accept, post histogram, draw).  The
// arithmetic and the random stream are those of the other word kernels, so
// the results are bit-identical.  Every block leaves only after a cluster
// barrier that follows the last remote read.
#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

constexpr int kClThreads = 512;
constexpr int kClWarps = kClThreads / 32;

namespace {

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Address of `local` (this block's shared memory) in block `rank` of the
// cluster.
__device__ __forceinline__ uint32_t cl_map(const void* local, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ int4 cl_ld4(uint32_t addr) {
    int4 v;
    asm volatile("ld.shared::cluster.v4.s32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ int cl_ld(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];\n" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Exclusive prefix of one value per thread over the block (kClThreads).
__device__ __forceinline__ int cl_block_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int t = lane < kClWarps ? warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xFFFFFFFFu, ti, o);
            if (lane >= o) ti += n;
        }
        if (lane < kClWarps) warp_tot[lane] = ti - t;
        if (lane == kClWarps - 1) *total = ti;
    }
    __syncthreads();
    const int r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

}  // namespace

// Shared memory of a block: two K-wide rows (padded to a multiple of 4, plus
// one entry for the prefix total), with dense tables the c_k deltas, then the
// slice's z and proposals (T tokens).
__host__ __device__ inline int cluster_row_words(int K) { return ((K + 1) + 3) & ~3; }

__host__ __device__ inline int cluster_fixed_bytes(int K, int stage_ck) {
    return (2 * cluster_row_words(K) + (stage_ck ? ((K + 3) & ~3) : 0)) * 4;
}

int cluster_slice_capacity(int K, int M, int stage_ck, int smem_max) {
    const int room = smem_max - cluster_fixed_bytes(K, stage_ck);
    if (room <= 0) return 0;
    return (room / (4 * (M + 1))) & ~3;
}

template <int M>
__global__ void __launch_bounds__(kClThreads, 1) cluster_word_kernel(PhaseArgs a, const int32_t* __restrict__ words,
                                                                     int nwords, int C, int T, int gbits) {
    extern __shared__ __align__(16) int csm[];
    __shared__ int warp_tot[kClWarps];
    __shared__ int s_total;
    const int K = a.K, tid = threadIdx.x;
    const int RW = cluster_row_words(K);
    int* rowA = csm;                   // slice histogram / post partial / guide table
    int* rowB = csm + RW;              // the word's row: C_w, then post counts, then prefix
    int* dck = rowB + RW;              // c_k deltas (dense tables)
    int* zt = dck + (a.stage_ck ? ((K + 3) & ~3) : 0);
    int* pt = zt + T;
    Checks chk;

    const uint32_t rank = cl_rank();
    const int cid = blockIdx.x / C;
    int w = (cid < nwords) ? words[cid] : 0;
    if (!chk(cid < nwords && w >= 0 && (int64_t)w < a.nseg_total, 0)) w = 0;
    const int b = a.seg_off[w];
    int L = a.seg_off[w + 1] - b;
    const int S = (L + C - 1) / C;   // slice length
    int s0 = (int)rank * S;
    int n = max(0, min(L, s0 + S) - s0);
    if (!chk(L >= 0 && S <= T && (int64_t)b + L <= a.N, 1)) {
        L = 0;
        n = 0;
        s0 = 0;
    }
    const int q0 = b + s0;   // first word-major index of the slice

    // 1. the slice in shared memory and its topic histogram
    for (int k = tid; k < 2 * RW; k += kClThreads) csm[k] = 0;
    if (a.stage_ck)
        for (int k = tid; k < K; k += kClThreads) dck[k] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kClThreads) {
        const int z0 = chk.topic(a.z[q0 + i], K, 3);
        zt[i] = z0;
#pragma unroll
        for (int u = 0; u < M; ++u) pt[i * M + u] = chk.topic(a.prop[(int64_t)(q0 + i) * M + u], K, 4);
        atomicAdd(&rowA[z0], 1);
    }
    // the cluster's sum of the rows in rowA, into every block's rowB: each
    // block reduces its shard of 16-byte chunks, then gathers the others
    const int nch = RW / 4;
    const int shard = (nch + C - 1) / C;
    auto reduce_rows = [&]() {
        cl_sync();
        const int c0 = (int)rank * shard, c1 = min(nch, c0 + shard);
        for (int c = c0 + tid; c < c1; c += kClThreads) {
            int4 s = make_int4(0, 0, 0, 0);
            for (int r = 0; r < C; ++r) {
                const int4 v = cl_ld4(cl_map(rowA + 4 * c, (uint32_t)r));
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
            reinterpret_cast<int4*>(rowB)[c] = s;
        }
        cl_sync();
        for (int c = tid; c < nch; c += kClThreads) {
            const int owner = c / shard;
            if (owner == (int)rank) continue;
            reinterpret_cast<int4*>(rowB)[c] = cl_ld4(cl_map(rowB + 4 * c, (uint32_t)owner));
        }
        cl_sync();
    };
    reduce_rows();
    // rowB = C_w (phase-start); rowA becomes the post-acceptance partial row
    for (int k = tid; k < RW; k += kClThreads) rowA[k] = 0;
    __syncthreads();

    // 2. M chained MH steps per token and the picks of Eq. 6
    const uint32_t phase = kPhaseWord;
    const float Lf = __int2float_rn(L);
    const float LG = __fadd_rn(Lf, a.G);
    for (int i = tid; i < n; i += kClThreads) {
        const int q = q0 + i;
        const int z0 = zt[i];
        int s = z0;
#pragma unroll
        for (int u = 0; u < M; ++u) {
            const uint4 r = draw((uint32_t)q, a.iter, phase, (uint32_t)(u + 1), 0u, a.rk);
            const int tp = pt[i * M + u];
            if (tp != s) {
                const float cs = __ldg(a.ckb + s), ct = __ldg(a.ckb + tp);
                if (accept(r.x, rowB[s], rowB[tp], a.g, cs, ct)) s = tp;
            }
            pt[i * M + u] = coin(r.y, Lf, LG) ? -(int)(dice(r.z, (uint32_t)max(L, 1)) + 1)
                                              : (int)dice(r.z, (uint32_t)K);
        }
        zt[i] = s;
        atomicAdd(&rowA[s], 1);
        if (s != z0) {
            if (a.stage_ck) {
                atomicSub(&dck[z0], 1);
                atomicAdd(&dck[s], 1);
            } else if (a.ck_delta) {
                atomicSub(&a.ck[z0], 1);
                atomicAdd(&a.ck[s], 1);
            }
        }
    }
    __syncthreads();

    // 3. picks of ranks: the j-th smallest post-acceptance topic of the word
    //    (guide table over the prefix), or the topic of its j-th token
    if (a.word_storage) {
        cl_sync();   // every slice holds its new topics
        for (int i = tid; i < n; i += kClThreads) {
#pragma unroll
            for (int u = 0; u < M; ++u) {
                const int pk = pt[i * M + u];
                if (pk >= 0) continue;
                int j = -pk - 1;
                if (!chk.tok((uint32_t)j < (uint32_t)L, 5)) j = 0;
                const int owner = j / S;
                pt[i * M + u] = cl_ld(cl_map(zt + (j - owner * S), (uint32_t)owner));
            }
        }
        cl_sync();   // no block leaves while another reads its slice
    } else {
        reduce_rows();   // rowB = post-acceptance counts; no remote reads after this
        // exclusive prefix in place, P[K] = L
        const int per = (K + kClThreads - 1) / kClThreads;
        const int k0 = min(K, tid * per), k1 = min(K, k0 + per);
        int sum = 0;
        for (int k = k0; k < k1; ++k) sum += rowB[k];
        int run = cl_block_scan(sum, warp_tot, &s_total);
        for (int k = k0; k < k1; ++k) {
            const int c = rowB[k];
            rowB[k] = run;
            run += c;
        }
        if (tid == 0) rowB[K] = s_total;
        __syncthreads();
        // guide table in rowA: bucket B(j) = (j * floor(2^(32+gb) / L)) >> 32
        // holds the topic of the smallest rank of the bucket
        const int nb = 1 << gbits;
        const uint64_t mult = (1ull << (32 + gbits)) / (uint64_t)max(L, 1);
        auto bucket_of = [&](int j) { return j < 0 ? -1 : (int)(((uint64_t)j * mult) >> 32); };
        for (int k = k0; k < k1; ++k) {
            const int bb0 = bucket_of(rowB[k] - 1) + 1, bb1 = min(bucket_of(rowB[k + 1] - 1), nb - 1);
            for (int bb = bb0; bb <= bb1; ++bb) rowA[bb] = k;
        }
        for (int bb = max(0, bucket_of(L - 1) + 1) + tid; bb < nb; bb += kClThreads) rowA[bb] = K - 1;
        __syncthreads();
        for (int i = tid; i < n; i += kClThreads) {
#pragma unroll
            for (int u = 0; u < M; ++u) {
                const int pk = pt[i * M + u];
                if (pk >= 0) continue;
                int j = -pk - 1;
                if (!chk.tok((uint32_t)j < (uint32_t)L, 5)) j = 0;
                int k = rowA[bucket_of(j)];
                for (int steps = 0; k + 1 < K && rowB[k + 1] <= j && steps < K; ++steps) ++k;
                pt[i * M + u] = chk.tok(rowB[k + 1] > j, 6) ? k : 0;
            }
        }
    }
    __syncthreads();

    // 4. write back
    for (int i = tid; i < n; i += kClThreads) {
        a.z[q0 + i] = zt[i];
#pragma unroll
        for (int u = 0; u < M; ++u) a.prop[(int64_t)(q0 + i) * M + u] = pt[i * M + u];
    }
    if (a.stage_ck) {
        __syncthreads();
        for (int k = tid; k < K; k += kClThreads)
            if (dck[k] != 0) atomicAdd(&a.ck[k], dck[k]);
    }
    chk.publish(a.fault, kSiteWordCluster);
}

int cluster_guide_bits(int K) {
    int b = 0;
    while (b < 14 && (2 << b) <= K) ++b;   // 2^b <= K: the guide fits in a row
    return b;
}

static const void* cluster_pick(int M) {
    switch (M) {
        case 1: return (const void*)cluster_word_kernel<1>;
        case 2: return (const void*)cluster_word_kernel<2>;
        case 3: return (const void*)cluster_word_kernel<3>;
        case 4: return (const void*)cluster_word_kernel<4>;
        default: return nullptr;
    }
}

int cluster_size_supported(int K, int M, int stage_ck, int C, int smem) {
    const void* f = cluster_pick(M);
    if (!f || smem < cluster_fixed_bytes(K, stage_ck)) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (C > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_cluster_word(const PhaseArgs& a, const int32_t* words, int nwords, int C, int T, int smem,
                                cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nwords <= 0) return cudaSuccess;
    const void* f = cluster_pick(a.M);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((int64_t)nwords * C));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PhaseArgs args = a;
    int gb = cluster_guide_bits(a.K);
    void* params[] = {&args, (void*)&words, &nwords, &C, &T, &gb};
    return cudaLaunchKernelExC(&cfg, f, params);
}

}  // namespace wl
