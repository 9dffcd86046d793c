// Fold-in of new documents against a frozen model: the document phase and
// word phase of Sec. 4.4 with the word side frozen (the paper trains only;
// the readings are those of the oracle's fold-in):
//   model   : the trained C_w as a dense [V, K] table, each word's trained
//             topics sorted ascending (word-major, [N]), frozen c_k;
//   document: pi^word (Eq. 7) against the document's phase-start c_d and the
//             frozen c_k, then positioning over the post-acceptance z_d
//             (Sec. 4.3);
//   word    : pi^doc against the frozen C_w row of the token's word and the
//             frozen c_k, then a word proposal from the frozen row (Eq. 6):
//             with probability L_w / (L_w + K beta) the j-th smallest topic
//             of the word (one load from its sorted topics), else uniform.
// Random numbers: Philox keyed by the fold-in seed, counter = (position in
// the document, iteration, phase << 8 | i, document id), phases 3/4/5, so a
// document's result does not depend on the other documents of the call.
// Two schedules with the same results.  One warp per document, all sweeps
// in one launch (the learned proposal, serving, and tuning foldin_kernel =
// 1): the document's count table lives in the warp's slice of shared
// memory, its z and proposals in global memory (document order, coalesced),
// the frozen rows read where the tokens need them.  Word-major phases (the
// plain proposal's default, below): per sweep a document-phase launch and a
// word-phase launch over the tokens grouped by word.
#include <algorithm>

#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

enum : uint32_t { kPhaseFoldInit = 3, kPhaseFoldDoc = 4, kPhaseFoldWord = 5 };

// ---------------------------------------------------------------------------
// Frozen model: per-word topic counts of the trained state (dense [V, K]),
// then each word's topics in ascending order (a counting sort through its
// row: topic k fills C_wk consecutive slots).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) model_counts_kernel(const int32_t* __restrict__ z,
                                                                const int32_t* __restrict__ word_off,
                                                                int64_t V, int K, int32_t* __restrict__ Cw,
                                                                int32_t* fault) {
    Checks chk;
    for (int64_t w = blockIdx.x; w < V; w += gridDim.x) {
        int32_t* row = Cw + w * (int64_t)K;
        for (int t = word_off[w] + threadIdx.x; t < word_off[w + 1]; t += kThreads)
            atomicAdd(&row[chk.topic(z[t], K, 0)], 1);
    }
    chk.publish(fault, kSiteFoldin);
}

__global__ void __launch_bounds__(kThreads) model_sort_kernel(const int32_t* __restrict__ word_off,
                                                              int64_t V, int K, const int32_t* __restrict__ Cw,
                                                              int32_t* __restrict__ Zs) {
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total;
    const int per = (K + kThreads - 1) / kThreads;
    for (int64_t w = blockIdx.x; w < V; w += gridDim.x) {
        const int32_t* row = Cw + w * (int64_t)K;
        const int base = word_off[w], Lw = word_off[w + 1] - base;
        const int k0 = min(K, (int)threadIdx.x * per), k1 = min(K, k0 + per);
        int sum = 0;
        for (int k = k0; k < k1; ++k) sum += row[k];
        int run = block_excl_scan(sum, warp_tot, &s_total);
        for (int k = k0; k < k1; ++k)
            for (int c = row[k]; c > 0 && run < Lw; --c) Zs[base + run++] = k;
        __syncthreads();
    }
}

cudaError_t launch_model_build(const int32_t* z, const int32_t* word_off, int64_t V, int K,
                               int32_t* Cw, int32_t* Zs, int32_t* fault, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    cudaError_t e = cudaMemsetAsync(Cw, 0, (size_t)V * K * sizeof(int32_t), st);
    if (e != cudaSuccess || V <= 0) return e;
    model_counts_kernel<<<grid, kThreads, 0, st>>>(z, word_off, V, K, Cw, fault);
    model_sort_kernel<<<grid, kThreads, 0, st>>>(word_off, V, K, Cw, Zs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The fold-in sweep of one document by one warp (shared by the batch fold-in
// kernel and the serving kernel).
// ---------------------------------------------------------------------------
int foldin_table_words(int K, int Lmax) {
    if (K <= kDenseMaxK) return ((K + 1) / 2 + 3) & ~3;
    return (int)pow2_above((uint32_t)min(2 * max(Lmax, 1), K));
}

__device__ __forceinline__ int fold_count(const uint32_t* tab, uint32_t cap, bool dense, int k) {
    return dense ? (int)((tab[(uint32_t)k >> 1] >> (((uint32_t)k & 1) * 16)) & 0xFFFFu)
                 : table_get(tab, cap, (uint32_t)k);
}

// The threads that sweep one document together: one warp, or (long
// documents in serving) the whole block.
struct WarpGroup {
    int lane;
    __device__ __forceinline__ int rank() const { return lane; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ int bcast(int v) const { return __shfl_sync(0xFFFFFFFFu, v, 0); }
};
struct BlockGroup {
    __device__ __forceinline__ int rank() const { return (int)threadIdx.x; }
    __device__ __forceinline__ int size() const { return (int)blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int bcast(int v) const {
        __shared__ int s_v;
        if (threadIdx.x == 0) s_v = v;
        __syncthreads();
        const int r = s_v;
        __syncthreads();
        return r;
    }
};

// One document's state: its tokens' word ids, z and proposals (document
// order), its stream id, and (learned proposal) its proposal row and alias
// table.
struct FoldDoc {
    int32_t* z;
    int32_t* prop;
    const int32_t* words;
    int L;
    uint32_t id;
    const float* q;
    const int2* atab;
};

// The group's count table of the document's current z (dense, or a hash of
// capacity cap).
template <bool kDense, class G>
__device__ __forceinline__ void fold_table(uint32_t* tab, int words, uint32_t cap, const FoldDoc& doc,
                                           uint32_t km, const G& g) {
    for (int i = g.rank(); i < words; i += g.size()) tab[i] = 0u;
    g.sync();
    for (int j = g.rank(); j < doc.L; j += g.size()) {
        const uint32_t k = min((uint32_t)doc.z[j], km);
        if (kDense) atomicAdd(&tab[k >> 1], (k & 1) ? 65536u : 1u);
        else table_add(tab, cap, k);
    }
    g.sync();
}

// Initialisation: z = Dice(K), proposals = z.
template <int M, class G>
__device__ __forceinline__ void fold_init(const FoldArgs& f, const FoldDoc& doc, const G& g) {
    for (int j = g.rank(); j < doc.L; j += g.size()) {
        const uint4 r = draw((uint32_t)j, 0u, kPhaseFoldInit, 0u, doc.id, f.rk);
        const int z0 = (int)dice(r.x, (uint32_t)f.K);
#pragma unroll
        for (int i = 0; i < M; ++i) doc.prop[j * M + i] = z0;
        doc.z[j] = z0;
    }
    g.sync();
}

// The document phase of sweep `it` of one document.  kLearned: the learned
// document proposal (the encoder's q through its alias table) replaces
// positioning.
template <int M, bool kDense, bool kLearned, class G>
__device__ void fold_doc_phase(const FoldArgs& f, const FoldDoc& doc, int it, uint32_t* tab, int words,
                               uint32_t cap, const G& g) {
    const int K = f.K, L = doc.L;
    const uint32_t km = (uint32_t)K - 1u;
    int32_t* z = doc.z;
    int32_t* prop = doc.prop;
    const float Lf = __int2float_rn(L);
    const float LG = __fadd_rn(Lf, f.abar);
    // document phase: accept with the phase-start c_d ...
    fold_table<kDense>(tab, words, cap, doc, km, g);
    for (int j = g.rank(); j < L; j += g.size()) {
        // operands first, then the Philox blocks, then the chain
        int s = min((uint32_t)z[j], km);
        int cs = fold_count(tab, cap, kDense, s);
        float ks = __ldg(f.ckb + s);
        int tv[M], ctv[M];
        float ktv[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            tv[i] = (int)min((uint32_t)prop[j * M + i], km);
            ctv[i] = fold_count(tab, cap, kDense, tv[i]);
            ktv[i] = __ldg(f.ckb + tv[i]);
        }
        uint32_t r0[M];
#pragma unroll
        for (int i = 0; i < M; ++i)
            r0[i] = draw((uint32_t)j, (uint32_t)it, kPhaseFoldDoc, (uint32_t)(i + 1), doc.id, f.rk).x;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (tv[i] != s && accept(r0[i], cs, ctv[i], f.alpha, ks, ktv[i])) {
                s = tv[i];
                cs = ctv[i];
                ks = ktv[i];
            }
        }
        z[j] = s;
    }
    g.sync();
    // ... then positioning over the post-acceptance z_d (or draws from the
    // learned proposal's alias table)
    for (int j = g.rank(); j < L; j += g.size()) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const uint4 r = draw((uint32_t)j, (uint32_t)it, kPhaseFoldDoc, (uint32_t)(i + 1), doc.id, f.rk);
            if (kLearned) {
                const int k = (int)dice(r.z, (uint32_t)K);
                const int2 e = __ldg(doc.atab + k);
                prop[j * M + i] = u24(r.y) < __int_as_float(e.x) ? k : (int)min((uint32_t)e.y, km);
            } else {
                prop[j * M + i] = coin(r.y, Lf, LG) ? z[dice(r.z, (uint32_t)L)] : (int)dice(r.z, (uint32_t)K);
            }
        }
    }
    g.sync();
}

// Sweep `it` of one document: the document phase, then the word phase
// against the frozen rows.  kLearned: the word phase accepts the learned
// proposal with the independence-sampler rate min{1, p(t) q(s) / (p(s) q(t))}
// of Alg. 1, p(k) = (C_dk + alpha)(C_wk + beta)/(c_k + beta_bar) with the word
// phase's phase-start c_d (the oracle's readings L6-L7).
template <int M, bool kDense, bool kLearned, class G>
__device__ void fold_sweep(const FoldArgs& f, const FoldDoc& doc, int it, uint32_t* tab, int words,
                           uint32_t cap, Checks& chk, const G& g) {
    const int K = f.K, L = doc.L;
    const uint32_t km = (uint32_t)K - 1u;
    int32_t* z = doc.z;
    int32_t* prop = doc.prop;
    fold_doc_phase<M, kDense, kLearned>(f, doc, it, tab, words, cap, g);
    if (kLearned) fold_table<kDense>(tab, words, cap, doc, km, g);   // the word phase's phase-start c_d
    // word phase against the frozen rows: accept, then a proposal from the
    // token's frozen row (one Philox block per step)
    for (int j = g.rank(); j < L; j += g.size()) {
        int w = doc.words[j];
        if (!chk((uint32_t)w < (uint32_t)f.V, 1)) w = 0;
        const int32_t* row = f.Cw + (int64_t)w * K;
        const int wb = __ldg(f.word_off + w);
        const int Lw = __ldg(f.word_off + w + 1) - wb;
        const float Lwf = __int2float_rn(Lw);
        const float LwG = __fadd_rn(Lwf, f.kbeta);
        int s = min((uint32_t)z[j], km);
        int cs = __ldg(row + s);
        float ks = __ldg(f.ckb + s);
        float qs = kLearned ? __ldg(doc.q + s) : 0.0f;
        uint32_t r1[M], r2[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const uint4 r = draw((uint32_t)j, (uint32_t)it, kPhaseFoldWord, (uint32_t)(i + 1), doc.id, f.rk);
            r1[i] = r.y;
            r2[i] = r.z;
            const int t = (int)min((uint32_t)prop[j * M + i], km);
            if (t != s) {
                const int ct = __ldg(row + t);
                const float kt = __ldg(f.ckb + t);
                const float qt = kLearned ? __ldg(doc.q + t) : 0.0f;
                bool acc;
                if (kLearned) {
                    const float cds = __int2float_rn(fold_count(tab, cap, kDense, s));
                    const float cdt = __int2float_rn(fold_count(tab, cap, kDense, t));
                    const float num = __fmul_rn(__fmul_rn(__fmul_rn(__fadd_rn(cdt, f.alpha),
                                                                    __fadd_rn(__int2float_rn(ct), f.beta)),
                                                          ks), qs);
                    const float den = __fmul_rn(__fmul_rn(__fmul_rn(__fadd_rn(cds, f.alpha),
                                                                    __fadd_rn(__int2float_rn(cs), f.beta)),
                                                          kt), qt);
                    acc = __fmul_rn(u24(r.x), den) < num;
                } else {
                    acc = accept(r.x, cs, ct, f.beta, ks, kt);
                }
                if (acc) {
                    s = t;
                    cs = ct;
                    ks = kt;
                    qs = qt;
                }
            }
        }
        z[j] = s;
#pragma unroll
        for (int i = 0; i < M; ++i)
            prop[j * M + i] = (Lw > 0 && coin(r1[i], Lwf, LwG))
                                  ? __ldg(f.Zs + wb + (int)dice(r2[i], (uint32_t)Lw))
                                  : (int)dice(r2[i], (uint32_t)K);
    }
    g.sync();
}

// theta (Eq. 4) of the document's current z.
template <bool kDense, class G>
__device__ __forceinline__ void fold_theta(const FoldArgs& f, const FoldDoc& doc, float* th, uint32_t* tab,
                                           int words, uint32_t cap, const G& g) {
    fold_table<kDense>(tab, words, cap, doc, (uint32_t)f.K - 1u, g);
    const float den = __fadd_rn(__int2float_rn(doc.L), f.abar);
    for (int k = g.rank(); k < f.K; k += g.size())
        th[k] = __fdiv_rn(__fadd_rn(__int2float_rn(fold_count(tab, cap, kDense, k)), f.alpha), den);
    g.sync();
}

template <int M, bool kDense, bool kLearned>
__global__ void __launch_bounds__(kThreads) foldin_kernel(FoldArgs f, int tab_words) {
    extern __shared__ __align__(16) uint32_t fsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tab = fsm + warp * tab_words;
    const int K = f.K;
    Checks chk;
    for (;;) {
        int di = 0;
        if (lane == 0) di = atomicAdd(f.counter, 1);
        di = __shfl_sync(0xFFFFFFFFu, di, 0);
        if (di >= f.Dn) break;
        int d = f.order[di];
        if (!chk(d >= 0 && d < f.Dn, 0)) d = 0;
        const int b = f.doc_off[d];
        int L = f.doc_off[d + 1] - b;
        if (!chk(L >= 0 && L <= f.Lmax, 0)) L = 0;
        FoldDoc doc;
        doc.z = f.z + b;
        doc.prop = f.prop + (int64_t)b * M;
        doc.words = f.words + b;
        doc.L = L;
        doc.id = (uint32_t)f.ids[d];
        doc.q = kLearned ? f.q + (int64_t)d * K : nullptr;
        doc.atab = kLearned ? f.atab + (int64_t)d * K : nullptr;
        const uint32_t cap = kDense ? 0u : pow2_above((uint32_t)min(2 * max(L, 1), K));
        const int words = kDense ? tab_words : (int)cap;
        const WarpGroup wg{lane};
        fold_init<M>(f, doc, wg);
        for (int it = 1; it <= f.sweeps; ++it) fold_sweep<M, kDense, kLearned>(f, doc, it, tab, words, cap, chk, wg);
        if (f.theta) fold_theta<kDense>(f, doc, f.theta + (int64_t)d * K, tab, words, cap, wg);
    }
    chk.publish(f.fault, kSiteFoldin);
}

// Serving: one launch advances every active slot by one sweep (a slot's
// first launch initialises it; its last writes theta).  The step lasts as
// long as its longest document takes, so long documents (sl.long_active)
// are swept by a whole block each, from the first sl.long_blocks blocks;
// the other blocks' warps take one short document each.  Slots are handed
// out by work counters.
template <int M, bool kDense, bool kLearned, class G>
__device__ __forceinline__ void serve_slot(const FoldArgs& f, const ServeSlots& sl, int s, uint32_t* tab,
                                           int tab_words, Checks& chk, const G& g) {
    const int K = f.K;
    if (!chk(s >= 0 && s < sl.nslots, 0)) return;
    const int4 info = sl.info[s];   // {token offset, L, sweeps done, stream id}
    const int L = info.y;
    if (!chk(info.x >= 0 && L >= 0 && L <= f.Lmax && (int64_t)info.x + L <= sl.pool_tokens, 0)) return;
    FoldDoc doc;
    doc.z = sl.z + info.x;
    doc.prop = sl.prop + (int64_t)info.x * M;
    doc.words = sl.words + info.x;
    doc.L = L;
    doc.id = (uint32_t)info.w;
    doc.q = kLearned ? sl.q + (int64_t)s * K : nullptr;
    doc.atab = kLearned ? sl.atab + (int64_t)s * K : nullptr;
    const uint32_t cap = kDense ? 0u : pow2_above((uint32_t)min(2 * max(L, 1), K));
    const int words = kDense ? tab_words : (int)cap;
    const int done = info.z;
    if (done == 0) fold_init<M>(f, doc, g);
    fold_sweep<M, kDense, kLearned>(f, doc, done + 1, tab, words, cap, chk, g);
    if (done + 1 >= f.sweeps) {
        // finished: theta into the next row of the step's output
        int oi = 0;
        if (g.rank() == 0) oi = atomicAdd(sl.fin_count, 1);
        oi = g.bcast(oi);
        if (chk(oi < sl.nslots, 0)) {
            fold_theta<kDense>(f, doc, sl.fin_theta + (int64_t)oi * K, tab, words, cap, g);
            if (g.rank() == 0) sl.fin_slot[oi] = s;
        }
    }
    if (g.rank() == 0) sl.info[s].z = done + 1;
}

template <int M, bool kDense, bool kLearned>
__global__ void __launch_bounds__(kThreads) serve_kernel(FoldArgs f, ServeSlots sl, int tab_words) {
    extern __shared__ __align__(16) uint32_t fsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Checks chk;
    if ((int)blockIdx.x < sl.long_blocks) {
        const BlockGroup bg;
        for (;;) {
            int si = 0;
            if (threadIdx.x == 0) si = atomicAdd(sl.long_counter, 1);
            si = bg.bcast(si);
            if (si >= sl.nlong) break;
            serve_slot<M, kDense, kLearned>(f, sl, sl.long_active[si], fsm, tab_words, chk, bg);
            __syncthreads();   // the table is the next document's
        }
    } else {
        const WarpGroup wg{lane};
        uint32_t* tab = fsm + warp * tab_words;
        for (;;) {
            int si = 0;
            if (lane == 0) si = atomicAdd(f.counter, 1);
            si = __shfl_sync(0xFFFFFFFFu, si, 0);
            if (si >= sl.nactive) break;
            serve_slot<M, kDense, kLearned>(f, sl, sl.active[si], tab, tab_words, chk, wg);
        }
    }
    chk.publish(f.fault, kSiteFoldin);
}

// ---------------------------------------------------------------------------
// Word-major fold-in (plain proposal).  In the kernel above a token's word
// phase reads its word's frozen row at random: C_wz and C_wt of M proposals
// and M entries of the word's sorted topics, one 32-byte sector each, out of
// a model several times the size of L2.  Here each sweep is two launches:
// the document phase, one warp per document as above (the requests' z and
// proposals stay in document order), then the word phase over the requests'
// tokens regrouped by word.  A warp takes pieces of up to kFoldPiece
// tokens of one word; for a word with at least `stage_min` tokens in the
// request set it loads the word's frozen row once into shared memory as
// prefix sums P (C_wk = P[k+1] - P[k], and the j-th smallest trained topic
// is the k with P[k] <= j < P[k+1], the value the sorted topics hold at j),
// so its tokens touch the model only there.  The other words keep the direct
// loads.  Every token draws the same Philox blocks and takes the same FP32
// decisions as in the per-document kernel: theta and z are identical.
// ---------------------------------------------------------------------------
constexpr int kFoldPiece = 256;

// Request tokens per word (warp-aggregated atomics: a warp's tokens of one
// word add once).
__global__ void fw_count_kernel(const int32_t* __restrict__ words, int64_t Nn, int32_t* __restrict__ cnt) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < Nn; b += step) {
        const int64_t g = b + threadIdx.x;
        const int w = g < Nn ? words[g] : -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, w);
        if (w >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[w], __popc(peers));
    }
}

// Per word (and one zero entry at V, which the exclusive scans turn into
// totals): records in the staged region, records in the direct region,
// staged pieces.
__global__ void fw_class_kernel(const int32_t* __restrict__ cnt, int64_t V, int stage_min,
                                int32_t* __restrict__ hc, int32_t* __restrict__ lc, int32_t* __restrict__ pc) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w <= V; w += step) {
        const int n = w < V ? cnt[w] : 0;
        const bool st = n >= stage_min;
        hc[w] = st ? n : 0;
        lc[w] = st ? 0 : n;
        pc[w] = st ? (n + kFoldPiece - 1) / kFoldPiece : 0;
    }
}

// Write cursor of each word's records: the staged region first, then the
// direct region.
__global__ void fw_cursor_kernel(const int32_t* __restrict__ cnt, const int32_t* __restrict__ hc,
                                 const int32_t* __restrict__ lc, int64_t V, int stage_min,
                                 int32_t* __restrict__ cur) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int htot = hc[V];
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < V; w += step)
        cur[w] = cnt[w] >= stage_min ? hc[w] : htot + lc[w];
}

// One warp per document: each token's record {token index, position in the
// document, stream id, word} at its word's cursor.
__global__ void fw_scatter_kernel(const int32_t* __restrict__ doc_off, const int64_t* __restrict__ ids,
                                  const int32_t* __restrict__ words, int Dn, int64_t Nn, int V,
                                  int32_t* __restrict__ cur, int4* __restrict__ rec, int32_t* fault) {
    Checks chk;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int d = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); d < Dn; d += nw) {
        const int b = doc_off[d], L = doc_off[d + 1] - b;
        const int id = (int)(uint32_t)ids[d];
        for (int jb = 0; jb < L; jb += 32) {
            const int j = jb + lane;
            int w = j < L ? words[b + j] : -1;
            if (w >= V) w = -1;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, w);
            const int leader = __ffs(peers) - 1;
            int pos = 0;
            if (lane == leader && w >= 0) pos = atomicAdd(&cur[w], __popc(peers));
            pos = __shfl_sync(0xFFFFFFFFu, pos, leader) + __popc(peers & ((1u << lane) - 1u));
            if (w >= 0 && chk(pos >= 0 && (int64_t)pos < Nn, 2)) rec[pos] = make_int4(b + j, j, id, w);
        }
    }
    chk.publish(fault, kSiteFoldin);
}

// The pieces: staged words' records in pieces of up to kFoldPiece, then the
// direct region cut the same way.
__global__ void fw_pieces_kernel(const int32_t* __restrict__ cnt, const int32_t* __restrict__ hc,
                                 const int32_t* __restrict__ lc, const int32_t* __restrict__ pc, int64_t V,
                                 int stage_min, int4* __restrict__ pieces, int32_t* __restrict__ npieces) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ptot = pc[V], htot = hc[V], ltot = lc[V];
    const int nlight = (ltot + kFoldPiece - 1) / kFoldPiece;
    for (int64_t w = tid; w < V; w += step) {
        const int n = cnt[w];
        if (n < stage_min) continue;
        int p = pc[w];
        for (int q = 0; q < n; q += kFoldPiece) pieces[p++] = make_int4((int)w, hc[w] + q, min(kFoldPiece, n - q), 1);
    }
    for (int64_t q = tid; q < nlight; q += step) {
        const int first = (int)q * kFoldPiece;
        pieces[ptot + q] = make_int4(-1, htot + first, min(kFoldPiece, ltot - first), 0);
    }
    if (tid == 0) *npieces = ptot + nlight;
}

// The j-th smallest trained topic of a staged word: the k with
// P[k] <= j < P[k+1] (P[0] = 0 <= j < P[K] = L_w).
__device__ __forceinline__ int fold_rank(const int32_t* P, int K, int j) {
    int lo = 0, hi = K;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// A token of the word phase with its state loaded: record {token index,
// position in its document, stream id, word}, z and proposals.
template <int M>
struct WordTok {
    int4 rc;
    int z;
    int p[M];
    bool ok;
};

template <int M>
__device__ __forceinline__ WordTok<M> fold_word_load(const FoldArgs& f, const FoldWords& fw, const int4 rc,
                                                     Checks& chk) {
    WordTok<M> t;
    t.rc = rc;
    t.ok = chk((int64_t)(uint32_t)rc.x < fw.Nn && (uint32_t)rc.w < (uint32_t)f.V, 1);
    const int64_t g = t.ok ? rc.x : 0;
    t.z = f.z[g];
    if (M == 2) {
        const int2 v = *reinterpret_cast<const int2*>(f.prop + g * 2);
        t.p[0] = v.x;
        t.p[M - 1] = v.y;
    } else if (M == 4) {
        const int4 v = *reinterpret_cast<const int4*>(f.prop + g * 4);
        t.p[0] = v.x;
        t.p[1 % M] = v.y;
        t.p[2 % M] = v.z;
        t.p[M - 1] = v.w;
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) t.p[i] = f.prop[g * M + i];
    }
    return t;
}

// The word phase of one token (the plain-proposal branch of fold_sweep):
// accept against the frozen row, then M proposals from it.  kStaged: the row
// is the warp's prefix array P; else direct loads of C_w and the sorted
// topics.
template <int M, bool kStaged>
__device__ __forceinline__ void fold_word_apply(const FoldArgs& f, const WordTok<M>& tk, int it,
                                                const int32_t* P) {
    if (!tk.ok) return;
    const int K = f.K;
    const uint32_t km = (uint32_t)K - 1u;
    const int g = tk.rc.x, j = tk.rc.y, w = tk.rc.w;
    const uint32_t id = (uint32_t)tk.rc.z;
    const int32_t* row = f.Cw + (int64_t)w * K;
    int wb = 0, Lw;
    if (kStaged) {
        Lw = P[K];
    } else {
        wb = __ldg(f.word_off + w);
        Lw = __ldg(f.word_off + w + 1) - wb;
    }
    auto cw = [&](int k) { return kStaged ? P[k + 1] - P[k] : __ldg(row + k); };
    const float Lwf = __int2float_rn(Lw);
    const float LwG = __fadd_rn(Lwf, f.kbeta);
    // the counts and c_k of z and of every proposal first, then the Philox
    // blocks while those loads are in flight, then the chain
    int s = min((uint32_t)tk.z, km);
    int cs = cw(s);
    float ks = __ldg(f.ckb + s);
    int tv[M], ctv[M];
    float ktv[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        tv[i] = (int)min((uint32_t)tk.p[i], km);
        ctv[i] = cw(tv[i]);
        ktv[i] = __ldg(f.ckb + tv[i]);
    }
    uint32_t r0[M], r1[M], r2[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const uint4 r = draw((uint32_t)j, (uint32_t)it, kPhaseFoldWord, (uint32_t)(i + 1), id, f.rk);
        r0[i] = r.x;
        r1[i] = r.y;
        r2[i] = r.z;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (tv[i] != s && accept(r0[i], cs, ctv[i], f.beta, ks, ktv[i])) {
            s = tv[i];
            cs = ctv[i];
            ks = ktv[i];
        }
    }
    f.z[g] = s;
    int out[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (Lw > 0 && coin(r1[i], Lwf, LwG)) {
            const int jj = (int)dice(r2[i], (uint32_t)Lw);
            out[i] = kStaged ? fold_rank(P, K, jj) : __ldg(f.Zs + wb + jj);
        } else {
            out[i] = (int)dice(r2[i], (uint32_t)K);
        }
    }
    int32_t* prop = f.prop + (int64_t)g * M;
    if (M == 2) {
        *reinterpret_cast<int2*>(prop) = make_int2(out[0], out[M - 1]);
    } else if (M == 4) {
        *reinterpret_cast<int4*>(prop) = make_int4(out[0], out[1 % M], out[2 % M], out[M - 1]);
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) prop[i] = out[i];
    }
}

// The tokens of one piece, lane-strided, software-pipelined: the record two
// tokens ahead and the z and proposals of the next token are in flight
// while a token is sampled.
template <int M, bool kStaged>
__device__ __forceinline__ void fold_word_piece(const FoldArgs& f, const FoldWords& fw, const int4 pc, int it,
                                                const int32_t* P, Checks& chk, int lane) {
    const int n = pc.z;
    const int4* rp = fw.rec + pc.y;
    if (lane >= n) return;
    int4 rn = __ldcs(rp + lane);
    WordTok<M> cur = fold_word_load<M>(f, fw, rn, chk);
    if (lane + 32 < n) rn = __ldcs(rp + lane + 32);
    for (int i = lane; i < n; i += 32) {
        const bool more = i + 32 < n;
        WordTok<M> nxt = cur;
        if (more) {
            nxt = fold_word_load<M>(f, fw, rn, chk);
            if (i + 64 < n) rn = __ldcs(rp + i + 64);
        }
        fold_word_apply<M, kStaged>(f, cur, it, P);
        cur = nxt;
    }
}

// The word phase of sweep `it`: warp w takes a contiguous range of the
// pieces (so consecutive pieces of one word are staged once).  The records
// are streamed with the evict-first hint, so that L2 keeps the requests' z
// and proposals, which the word order reads and writes at random.
template <int M>
__global__ void __launch_bounds__(kThreads) fold_word_kernel(FoldArgs f, FoldWords fw, int it) {
    extern __shared__ __align__(16) int32_t wsm[];
    const int lane = threadIdx.x & 31;
    const int K = f.K;
    int32_t* P = wsm + (threadIdx.x >> 5) * fw.pstride;
    Checks chk;
    const int np = *fw.npieces;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int p0 = (int)(np * gw / nw), p1 = (int)(np * (gw + 1) / nw);
    int staged = -1;
    for (int p = p0; p < p1; ++p) {
        const int4 pc = fw.pieces[p];   // {word, first record, records, staged}
        if (!chk(pc.y >= 0 && pc.z >= 0 && (int64_t)pc.y + pc.z <= fw.Nn, 2)) continue;
        if (pc.w != 0 && fw.pstride > 0 && (uint32_t)pc.x < (uint32_t)f.V) {
            if (pc.x != staged) {
                // P[k + 1] = C_wk, then prefix sums: lane l sums its chunk of
                // `per` entries (odd, so the lanes' chunks fall in distinct
                // banks), a warp scan of the chunk sums, then the chunk.
                const int32_t* row = f.Cw + (int64_t)pc.x * K;
                __syncwarp();
                for (int k = lane; k < K; k += 32) P[k + 1] = __ldg(row + k);
                __syncwarp();
                const int k0 = min(K, lane * fw.per), k1 = min(K, k0 + fw.per);
                int sum = 0;
                for (int k = k0; k < k1; ++k) sum += P[k + 1];
                int x = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if (lane >= o) x += y;
                }
                int run = x - sum;
                for (int k = k0; k < k1; ++k) {
                    run += P[k + 1];
                    P[k + 1] = run;
                }
                if (lane == 0) P[0] = 0;
                __syncwarp();
                staged = pc.x;
            }
            fold_word_piece<M, true>(f, fw, pc, it, P, chk, lane);
        } else {
            fold_word_piece<M, false>(f, fw, pc, it, P, chk, lane);
        }
    }
    chk.publish(f.fault, kSiteFoldin);
}

// One launch per phase of the document side: mode bit 1 initialises z and
// the proposals, bit 2 runs the document phase of sweep `it`, bit 4 writes
// theta.  `counter` is this launch's own work counter (zero on entry).
template <int M, bool kDense>
__global__ void __launch_bounds__(kThreads) fold_doc_kernel(FoldArgs f, int tab_words, int it, int mode,
                                                            int32_t* counter) {
    extern __shared__ __align__(16) uint32_t fsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tab = fsm + warp * tab_words;
    Checks chk;
    for (;;) {
        int di = 0;
        if (lane == 0) di = atomicAdd(counter, 1);
        di = __shfl_sync(0xFFFFFFFFu, di, 0);
        if (di >= f.Dn) break;
        int d = f.order[di];
        if (!chk(d >= 0 && d < f.Dn, 0)) d = 0;
        const int b = f.doc_off[d];
        int L = f.doc_off[d + 1] - b;
        if (!chk(L >= 0 && L <= f.Lmax, 0)) L = 0;
        FoldDoc doc;
        doc.z = f.z + b;
        doc.prop = f.prop + (int64_t)b * M;
        doc.words = f.words + b;
        doc.L = L;
        doc.id = (uint32_t)f.ids[d];
        doc.q = nullptr;
        doc.atab = nullptr;
        const uint32_t cap = kDense ? 0u : pow2_above((uint32_t)min(2 * max(L, 1), f.K));
        const int words = kDense ? tab_words : (int)cap;
        const WarpGroup wg{lane};
        if (mode & 1) fold_init<M>(f, doc, wg);
        if (mode & 2) fold_doc_phase<M, kDense, false>(f, doc, it, tab, words, cap, wg);
        if ((mode & 4) && f.theta) fold_theta<kDense>(f, doc, f.theta + (int64_t)d * f.K, tab, words, cap, wg);
    }
    chk.publish(f.fault, kSiteFoldin);
}

int64_t fold_pieces_bound(int64_t Nn, int stage_min) {
    return 2 * (Nn / kFoldPiece + 1) + Nn / std::max(stage_min, 1) + 2;
}

cudaError_t launch_fold_words_build(const FoldArgs& f, int64_t Nn, int stage_min, int32_t* cnt, int32_t* hc,
                                    int32_t* lc, int32_t* pc, int32_t* cur, int32_t* scan_tmp, int4* rec,
                                    int4* pieces, int32_t* npieces, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    const int64_t V = f.V;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)(V + 1) * 4, st);
    if (e != cudaSuccess) return e;
    if (Nn > 0) fw_count_kernel<<<grid, kThreads, 0, st>>>(f.words, Nn, cnt);
    fw_class_kernel<<<grid, kThreads, 0, st>>>(cnt, V, stage_min, hc, lc, pc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_scan_exclusive(hc, V + 1, scan_tmp, st)) != cudaSuccess) return e;
    if ((e = launch_scan_exclusive(lc, V + 1, scan_tmp, st)) != cudaSuccess) return e;
    if ((e = launch_scan_exclusive(pc, V + 1, scan_tmp, st)) != cudaSuccess) return e;
    fw_cursor_kernel<<<grid, kThreads, 0, st>>>(cnt, hc, lc, V, stage_min, cur);
    if (f.Dn > 0) fw_scatter_kernel<<<grid, kThreads, 0, st>>>(f.doc_off, f.ids, f.words, f.Dn, Nn, f.V, cur, rec, f.fault);
    fw_pieces_kernel<<<grid, kThreads, 0, st>>>(cnt, hc, lc, pc, V, stage_min, pieces, npieces);
    return cudaGetLastError();
}

template <int M>
static const void* fold_doc_ptr(bool dense) {
    return dense ? (const void*)fold_doc_kernel<M, true> : (const void*)fold_doc_kernel<M, false>;
}

static const void* fold_doc_pick(int M, bool dense) {
    switch (M) {
        case 1: return fold_doc_ptr<1>(dense);
        case 2: return fold_doc_ptr<2>(dense);
        case 3: return fold_doc_ptr<3>(dense);
        case 4: return fold_doc_ptr<4>(dense);
        default: return nullptr;
    }
}

static const void* fold_word_pick(int M) {
    switch (M) {
        case 1: return (const void*)fold_word_kernel<1>;
        case 2: return (const void*)fold_word_kernel<2>;
        case 3: return (const void*)fold_word_kernel<3>;
        case 4: return (const void*)fold_word_kernel<4>;
        default: return nullptr;
    }
}

cudaError_t launch_fold_doc(const FoldArgs& f, int tab_words, int it, int mode, int32_t* counter, int grid,
                            cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (f.Dn <= 0) return cudaSuccess;
    const void* fn = fold_doc_pick(f.M, f.K <= kDenseMaxK);
    const int warps = foldin_warps(tab_words);
    if (!fn || warps < 1) return cudaErrorInvalidValue;
    const int smem = warps * tab_words * 4;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FoldArgs args = f;
    int tw = tab_words, i = it, m = mode;
    int32_t* cnt = counter;
    void* params[] = {&args, &tw, &i, &m, &cnt};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * warps), params, (size_t)smem, st);
}

int fold_word_smem(const FoldWords& fw) { return kWarps * fw.pstride * 4; }

cudaError_t launch_fold_word(const FoldArgs& f, const FoldWords& fw, int it, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (fw.Nn <= 0) return cudaSuccess;
    const void* fn = fold_word_pick(f.M);
    if (!fn) return cudaErrorInvalidValue;
    const int smem = fold_word_smem(fw);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FoldArgs args = f;
    FoldWords w = fw;
    int i = it;
    void* params[] = {&args, &w, &i};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), params, (size_t)smem, st);
}

int fold_doc_blocks_per_sm(int K, int M, int tab_words) {
    const void* fn = fold_doc_pick(M, K <= kDenseMaxK);
    const int warps = foldin_warps(tab_words);
    if (!fn || warps < 1) return 0;
    const int smem = warps * tab_words * 4;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * warps, smem) != cudaSuccess) return 0;
    return n;
}

int fold_word_blocks_per_sm(int M, const FoldWords& fw) {
    const void* fn = fold_word_pick(M);
    if (!fn) return 0;
    const int smem = fold_word_smem(fw);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

template <int M, bool kDense>
static const void* fold_ptr(bool learned, bool serve) {
    if (serve)
        return learned ? (const void*)serve_kernel<M, kDense, true> : (const void*)serve_kernel<M, kDense, false>;
    return learned ? (const void*)foldin_kernel<M, kDense, true> : (const void*)foldin_kernel<M, kDense, false>;
}

static const void* fold_pick(int M, bool dense, bool learned, bool serve = false) {
    switch (M) {
        case 1: return dense ? fold_ptr<1, true>(learned, serve) : fold_ptr<1, false>(learned, serve);
        case 2: return dense ? fold_ptr<2, true>(learned, serve) : fold_ptr<2, false>(learned, serve);
        case 3: return dense ? fold_ptr<3, true>(learned, serve) : fold_ptr<3, false>(learned, serve);
        case 4: return dense ? fold_ptr<4, true>(learned, serve) : fold_ptr<4, false>(learned, serve);
        default: return nullptr;
    }
}

// Warps per block: as many as 8 whose count tables fit in 192 KB.
int foldin_warps(int tab_words) {
    const int w = (192 * 1024) / (tab_words * 4);
    return w < 1 ? 0 : (w > kWarps ? kWarps : w);
}

cudaError_t launch_foldin(const FoldArgs& f, int tab_words, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (f.Dn <= 0) return cudaSuccess;
    const bool dense = f.K <= kDenseMaxK;
    const void* fn = fold_pick(f.M, dense, f.q != nullptr);
    const int warps = foldin_warps(tab_words);
    if (!fn || warps < 1) return cudaErrorInvalidValue;
    const int smem = warps * tab_words * 4;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FoldArgs args = f;
    int tw = tab_words;
    void* params[] = {&args, &tw};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * warps), params, (size_t)smem, st);
}

// Admission of staged requests: request i (slot, pool offset, L, id) copies
// its words from the staging buffer into the pool and sets its slot.
__global__ void serve_admit_kernel(const int32_t* __restrict__ staged, const int4* __restrict__ req,
                                   const int32_t* __restrict__ src, int n, int nslots, int64_t pool_tokens,
                                   int32_t* __restrict__ pool_words, int4* __restrict__ info) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int4 r = req[i];   // {slot, pool offset, L, id}
        if (r.x < 0 || r.x >= nslots || r.y < 0 || r.z < 0 || (int64_t)r.y + r.z > pool_tokens) continue;
        for (int j = threadIdx.x; j < r.z; j += blockDim.x) pool_words[r.y + j] = staged[src[i] + j];
        if (threadIdx.x == 0) info[r.x] = make_int4(r.y, r.z, 0, r.w);
    }
}

// Rows i of src (n rows of K words) to rows slots[i] of dst.
__global__ void serve_rows_kernel(const uint32_t* __restrict__ src, const int32_t* __restrict__ slots, int n,
                                  int K, int nslots, uint32_t* __restrict__ dst) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int s = slots[i];
        if (s < 0 || s >= nslots) continue;
        for (int k = threadIdx.x; k < K; k += blockDim.x) dst[(int64_t)s * K + k] = src[(int64_t)i * K + k];
    }
}

cudaError_t launch_serve_admit(const int32_t* staged, const int4* req, const int32_t* src, int n, int nslots,
                               int64_t pool_tokens, int32_t* pool_words, int4* info, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (n <= 0) return cudaSuccess;
    serve_admit_kernel<<<std::min(n, 4096), 256, 0, st>>>(staged, req, src, n, nslots, pool_tokens, pool_words, info);
    return cudaGetLastError();
}

cudaError_t launch_serve_rows(const void* src, const int32_t* slots, int n, int K, int nslots, void* dst,
                              cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (n <= 0) return cudaSuccess;
    serve_rows_kernel<<<std::min(n, 4096), 256, 0, st>>>((const uint32_t*)src, slots, n, K, nslots, (uint32_t*)dst);
    return cudaGetLastError();
}

cudaError_t launch_serve(const FoldArgs& f, const ServeSlots& sl, int tab_words, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (sl.nactive <= 0 && sl.nlong <= 0) return cudaSuccess;
    const bool dense = f.K <= kDenseMaxK;
    const void* fn = fold_pick(f.M, dense, sl.q != nullptr, true);
    const int warps = foldin_warps(tab_words);
    if (!fn || warps < 1) return cudaErrorInvalidValue;
    const int smem = warps * tab_words * 4;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FoldArgs args = f;
    ServeSlots slots = sl;
    int tw = tab_words;
    void* params[] = {&args, &slots, &tw};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * warps), params, (size_t)smem, st);
}

int foldin_blocks_per_sm(int K, int M, int tab_words) {
    const void* fn = fold_pick(M, K <= kDenseMaxK, false);
    const int warps = foldin_warps(tab_words);
    if (!fn || warps < 1) return 0;
    const int smem = warps * tab_words * 4;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * warps, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace wl
