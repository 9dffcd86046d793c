// On-chip tier of the document and word phases (Sec. 4.4): one thread block
// takes a batch of consecutive documents (or words) with at most 4095 tokens
// in all, builds every segment's count table in shared memory (Sec. 5.4),
// runs the M chained MH steps of each token against it (Alg. 1, Eq. 7), and
// draws the M new proposals of Eq. 6 from the post-acceptance assignments:
//   document phase: random positioning (Sec. 4.3) in the caller's token order;
//   word phase:     the j-th smallest post-acceptance topic of the word.
// Word-major arrays are read and written with 128-bit accesses in the word
// phase and through perm (the doc-major -> word-major pointer array of
// Sec. 5.2) in the document phase.
#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

// Shared-memory layout of a batch block (bytes), shared with the host.
struct BatchSmem {
    int ck_off, seg_off, region_off, stage_off, cnt_off, total;
};

__host__ __device__ inline BatchSmem batch_smem_layout(int K, int stage_ck, int region_words,
                                                       int tpt, int word_phase) {
    BatchSmem s;
    int o = 0;
    s.ck_off = o;
    if (stage_ck) o += 2 * K * 4;
    o = (o + 15) & ~15;
    s.seg_off = o;
    o += (3 * kSegsMax + 4) * 4;
    o = (o + 15) & ~15;
    s.region_off = o;
    o += region_words * 4;
    o = (o + 15) & ~15;
    s.stage_off = o;
    const int n = kThreads * tpt;
    o += (n + (n >> 5) + 4) * 4;
    o = (o + 15) & ~15;
    s.cnt_off = o;
    if (word_phase) o += 16 * kThreads * 2;
    s.total = (o + 15) & ~15;
    return s;
}

template <int M>
struct Props { int v[M]; };

template <bool kDoc, int TPT, int M>
__global__ void __launch_bounds__(kThreads) batch_phase_kernel(PhaseArgs a,
                                                               const int2* __restrict__ batches,
                                                               int nbatch, int* __restrict__ counter,
                                                               int region_words, int kbits) {
    static_assert(TPT % 4 == 0, "tokens per thread come in chunks of four");
    extern __shared__ __align__(16) unsigned char smem[];
    const BatchSmem L = batch_smem_layout(a.K, a.stage_ck, region_words, TPT, kDoc ? 0 : 1);
    float* ckb_s = reinterpret_cast<float*>(smem + L.ck_off);
    int* dck_s = reinterpret_cast<int*>(smem + L.ck_off) + a.K;
    int* seg_tok = reinterpret_cast<int*>(smem + L.seg_off);        // [kSegsMax + 1]
    int* seg_reg = seg_tok + kSegsMax + 1;                          // [kSegsMax]
    int* seg_cap = seg_reg + kSegsMax;                              // [kSegsMax]
    uint32_t* region = reinterpret_cast<uint32_t*>(smem + L.region_off);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + L.stage_off);
    uint16_t* cnt = reinterpret_cast<uint16_t*>(smem + L.cnt_off);
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total, s_batch;

    const int tid = threadIdx.x;
    const int K = a.K;
    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    __syncthreads();

    for (;;) {
        if (tid == 0) s_batch = atomicAdd(counter, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int2 br = batches[b];
        const int nseg = br.y - br.x;
        const int base = a.seg_off[br.x];
        const int end = a.seg_off[br.y];

        // segment table: token offsets and count-table shapes
        for (int s = tid; s < nseg; s += kThreads) {
            const int o0 = a.seg_off[br.x + s], o1 = a.seg_off[br.x + s + 1];
            uint32_t w, cap;
            table_shape((uint32_t)(o1 - o0), (uint32_t)K, &w, &cap);
            seg_tok[s] = o0 - base;
            seg_reg[s] = (int)w;
            seg_cap[s] = (int)cap;
        }
        if (tid == 0) seg_tok[nseg] = end - base;
        __syncthreads();
        block_scan_array(seg_reg, nseg, warp_tot, &s_total);
        const int region_used = s_total;
        for (int i = tid; i < region_used; i += kThreads) region[i] = 0u;
        __syncthreads();

        // load the tokens this thread owns: chunks of 4 consecutive positions
        const int abase = base & ~3;
        int tk[TPT];          // word-major token index (-1: not ours)
        int zz[TPT];          // topic: phase-start, then post-acceptance
        int sl[TPT];          // segment slot in the batch
        Props<M> pp[TPT];     // pending proposals, then picks
#pragma unroll
        for (int c = 0; c < TPT / 4; ++c) {
            const int q0 = abase + 4 * (c * kThreads + tid);
            int4 pv = make_int4(0, 0, 0, 0);
            int4 zv = make_int4(0, 0, 0, 0);
            if (q0 < end) {
                if (kDoc) pv = *reinterpret_cast<const int4*>(a.perm + q0);
                else zv = *reinterpret_cast<const int4*>(a.z + q0);
            }
            const int pa[4] = {pv.x, pv.y, pv.z, pv.w};
            const int za[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = 4 * c + v;
                const int q = q0 + v;
                const bool mine = (q >= base) && (q < end);
                tk[j] = mine ? (kDoc ? pa[v] : q) : -1;
                if (kDoc) {
                    zz[j] = mine ? a.z[tk[j]] : 0;
                } else {
                    zz[j] = za[v];
                }
                if (mine) {
                    const int64_t pb = (int64_t)tk[j] * M;
#pragma unroll
                    for (int i = 0; i < M; ++i) pp[j].v[i] = a.prop[pb + i];
                }
            }
        }
        // segment slots and count tables
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            if (tk[j] < 0) { sl[j] = 0; continue; }
            const int p = (kDoc ? (abase + 4 * ((j / 4) * kThreads + tid) + (j % 4))
                                : tk[j]) - base;
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_tok[mid] <= p) lo = mid; else hi = mid - 1;
            }
            sl[j] = lo;
            table_add(region + seg_reg[lo], (uint32_t)seg_cap[lo], (uint32_t)zz[j]);
        }
        __syncthreads();

        // M chained MH steps per token (Alg. 1, Eq. 7), then the picks of Eq. 6
        const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            if (tk[j] < 0) continue;
            const int slot = sl[j];
            const uint32_t* tab = region + seg_reg[slot];
            const uint32_t cap = (uint32_t)seg_cap[slot];
            const int Ls = seg_tok[slot + 1] - seg_tok[slot];
            const float Lf = __int2float_rn(Ls);
            const float LG = __fadd_rn(Lf, a.G);
            const int z0 = zz[j];
            int s = z0;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const uint4 r = draw((uint32_t)tk[j], a.iter, phase, (uint32_t)(i + 1), 0u, a.k0, a.k1);
                const int t = pp[j].v[i];
                if (t != s) {
                    const float cs = a.stage_ck ? ckb_s[s] : __ldg(a.ckb + s);
                    const float ct = a.stage_ck ? ckb_s[t] : __ldg(a.ckb + t);
                    if (accept(r.x, table_get(tab, cap, (uint32_t)s), table_get(tab, cap, (uint32_t)t),
                               a.g, cs, ct))
                        s = t;
                }
                pp[j].v[i] = coin(r.y, Lf, LG) ? -(int)(dice(r.z, (uint32_t)Ls) + 1)
                                               : (int)dice(r.z, (uint32_t)K);
            }
            if (s != z0) {
                if (a.stage_ck) {
                    atomicSub(&dck_s[z0], 1);
                    atomicAdd(&dck_s[s], 1);
                } else {
                    atomicSub(&a.ck[z0], 1);
                    atomicAdd(&a.ck[s], 1);
                }
            }
            zz[j] = s;
            const int p = (kDoc ? (abase + 4 * ((j / 4) * kThreads + tid) + (j % 4)) : tk[j]) - base;
            stage[pad(p)] = kDoc ? (uint32_t)s : (((uint32_t)slot << kbits) | (uint32_t)s);
        }
        const int ntok = end - base;
        if (!kDoc) {
            // padding keys sort last; then the word's post-acceptance topics
            // are contiguous and ascending at [seg_tok[slot], seg_tok[slot+1])
            for (int p = ntok + tid; p < kThreads * TPT; p += kThreads) stage[pad(p)] = 0xFFFFFFFFu;
            __syncthreads();
            int sbits = 0;
            while ((1 << sbits) < nseg) ++sbits;
            block_radix_sort<TPT>(stage, cnt, sbits + kbits, warp_tot, &s_total);
        }
        __syncthreads();

        // resolve picks and write back
        const uint32_t kmask = (1u << kbits) - 1u;
        if (kDoc) {
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                if (tk[j] < 0) continue;
                const int sb = seg_tok[sl[j]];
                const int64_t pb = (int64_t)tk[j] * M;
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    int pk = pp[j].v[i];
                    if (pk < 0) pk = (int)stage[pad(sb + (-pk - 1))];
                    a.prop[pb + i] = pk;
                }
                a.z[tk[j]] = zz[j];
            }
        } else {
#pragma unroll
            for (int c = 0; c < TPT / 4; ++c) {
                const int q0 = abase + 4 * (c * kThreads + tid);
                if (q0 >= end) continue;
                bool full = true;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = 4 * c + v;
                    if (tk[j] < 0) { full = false; continue; }
                    const int sb = seg_tok[sl[j]];
#pragma unroll
                    for (int i = 0; i < M; ++i) {
                        const int pk = pp[j].v[i];
                        if (pk < 0) pp[j].v[i] = (int)(stage[pad(sb + (-pk - 1))] & kmask);
                    }
                }
                if (full) {
                    *reinterpret_cast<int4*>(a.z + q0) =
                        make_int4(zz[4 * c], zz[4 * c + 1], zz[4 * c + 2], zz[4 * c + 3]);
                    int buf[4 * M];
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int i = 0; i < M; ++i) buf[v * M + i] = pp[4 * c + v].v[i];
#pragma unroll
                    for (int u = 0; u < M; ++u)
                        reinterpret_cast<int4*>(a.prop + (int64_t)q0 * M)[u] =
                            make_int4(buf[4 * u], buf[4 * u + 1], buf[4 * u + 2], buf[4 * u + 3]);
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int j = 4 * c + v;
                        if (tk[j] < 0) continue;
                        a.z[tk[j]] = zz[j];
#pragma unroll
                        for (int i = 0; i < M; ++i) a.prop[(int64_t)tk[j] * M + i] = pp[j].v[i];
                    }
                }
            }
        }
        __syncthreads();
    }

    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads) {
            const int d = dck_s[k];
            if (d != 0) atomicAdd(&a.ck[k], d);
        }
    }
}

int batch_smem_bytes(int K, int stage_ck, int region_words, int tpt, int word_phase) {
    return batch_smem_layout(K, stage_ck, region_words, tpt, word_phase).total;
}

template <bool kDoc, int TPT>
static cudaError_t launch_t(const PhaseArgs& a, const int2* batches, int nbatch, int* counter,
                            int region_words, int kbits, int grid, cudaStream_t st) {
    const int smem = batch_smem_bytes(a.K, a.stage_ck, region_words, TPT, kDoc ? 0 : 1);
    cudaError_t e = cudaSuccess;
    switch (a.M) {
#define WL_CASE(MM)                                                                            \
    case MM: {                                                                                 \
        auto kern = batch_phase_kernel<kDoc, TPT, MM>;                                         \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);     \
        if (e != cudaSuccess) return e;                                                        \
        kern<<<grid, kThreads, smem, st>>>(a, batches, nbatch, counter, region_words, kbits);  \
        return cudaGetLastError();                                                             \
    }
        WL_CASE(1)
        WL_CASE(2)
        WL_CASE(3)
        WL_CASE(4)
#undef WL_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return e;
}

int batch_blocks_per_sm(int K, int stage_ck, int region_words, int tpt, int word_phase, int M) {
    const int smem = batch_smem_bytes(K, stage_ck, region_words, tpt, word_phase);
    int n = 0;
    const void* f = nullptr;
#define WL_PICK(D, T, MM) \
    if (word_phase == !D && tpt == T && M == MM) f = (const void*)batch_phase_kernel<D, T, MM>;
    WL_PICK(true, 16, 1) WL_PICK(true, 16, 2) WL_PICK(true, 16, 3) WL_PICK(true, 16, 4)
    WL_PICK(false, 16, 1) WL_PICK(false, 16, 2) WL_PICK(false, 16, 3) WL_PICK(false, 16, 4)
    WL_PICK(true, 8, 1) WL_PICK(true, 8, 2) WL_PICK(true, 8, 3) WL_PICK(true, 8, 4)
    WL_PICK(false, 8, 1) WL_PICK(false, 8, 2) WL_PICK(false, 8, 3) WL_PICK(false, 8, 4)
#undef WL_PICK
    if (!f) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_batch_phase(bool doc, int tpt, const PhaseArgs& a, const int2* batches,
                               int nbatch, int* counter, int region_words, int kbits, int grid,
                               cudaStream_t st) {
    if (nbatch <= 0) return cudaSuccess;
    if (tpt == 16)
        return doc ? launch_t<true, 16>(a, batches, nbatch, counter, region_words, kbits, grid, st)
                   : launch_t<false, 16>(a, batches, nbatch, counter, region_words, kbits, grid, st);
    if (tpt == 8)
        return doc ? launch_t<true, 8>(a, batches, nbatch, counter, region_words, kbits, grid, st)
                   : launch_t<false, 8>(a, batches, nbatch, counter, region_words, kbits, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace wl
