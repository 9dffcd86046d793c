// On-chip tier of the document and word phases (Sec. 4.4): one thread block
// takes a batch of consecutive documents (or words) with at most 4093 tokens
// in all, builds every segment's count table in shared memory (Sec. 5.4),
// runs the M chained MH steps of each token against it (Alg. 1, Eq. 7), and
// draws the M new proposals of Eq. 6 from the post-acceptance assignments:
//   document phase: random positioning (Sec. 4.3) in the caller's token order;
//   word phase:     the j-th smallest post-acceptance topic of the word.
// Count tables are dense (two 16-bit counts per word) when K <= 2048, else
// the paper's open-addressing hash; the choice is uniform per context.  The
// word phase orders each word's post-acceptance topics by a counting sort
// through its dense table, or by a block radix sort with hash tables.
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
                                                       int tpt, int radix) {
    BatchSmem s;
    int o = 0;
    s.ck_off = o;
    if (stage_ck) o += 2 * K * 4;
    o = (o + 15) & ~15;
    s.seg_off = o;
    o += (3 * kSegsMax + 4) * 4;
    o = (o + 15) & ~15;
    s.region_off = o;
    o += ((region_words + 3) & ~3) * 4;
    s.stage_off = o;
    const int n = kThreads * tpt;
    o += (n + (n >> 5) + 4) * 4;
    o = (o + 15) & ~15;
    s.cnt_off = o;
    if (radix) o += 16 * kThreads * 2;
    s.total = (o + 15) & ~15;
    return s;
}

template <int M>
struct Props { int v[M]; };

// The M proposals of token t: one 8- or 16-byte load when M is 2 or 4.
template <int M>
__device__ __forceinline__ void load_props(const int32_t* prop, int t, int* v) {
    if (M == 2) {
        const int2 x = *reinterpret_cast<const int2*>(prop + (int64_t)t * 2);
        v[0] = x.x;
        v[1 % M] = x.y;
    } else if (M == 4) {
        const int4 x = *reinterpret_cast<const int4*>(prop + (int64_t)t * 4);
        v[0] = x.x;
        v[1 % M] = x.y;
        v[2 % M] = x.z;
        v[3 % M] = x.w;
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = prop[(int64_t)t * M + i];
    }
}

template <int M>
__device__ __forceinline__ void store_props(int32_t* prop, int t, const int* v) {
    if (M == 2) {
        *reinterpret_cast<int2*>(prop + (int64_t)t * 2) = make_int2(v[0], v[1 % M]);
    } else if (M == 4) {
        *reinterpret_cast<int4*>(prop + (int64_t)t * 4) = make_int4(v[0], v[1 % M], v[2 % M], v[3 % M]);
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) prop[(int64_t)t * M + i] = v[i];
    }
}

// Dense table: topic k's 16-bit count lives in word k >> 1.
__device__ __forceinline__ uint32_t dense_unit(uint32_t k) { return (k & 1) ? 65536u : 1u; }
__device__ __forceinline__ int dense_get(const uint32_t* tab, uint32_t k) {
    return (int)((tab[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu);
}

template <bool kDense>
__device__ __forceinline__ void tab_add(uint32_t* tab, uint32_t cap, uint32_t k) {
    if (kDense) atomicAdd(&tab[k >> 1], dense_unit(k));
    else table_add(tab, cap, k);
}

template <bool kDense>
__device__ __forceinline__ int tab_get(const uint32_t* tab, uint32_t cap, uint32_t k) {
    return kDense ? dense_get(tab, k) : table_get(tab, cap, k);
}

// Resident blocks per SM the register allocation is held to.  Word batches
// of 8 tokens per thread: three (80 registers, a few spilled) measured
// faster than two (126 registers): PubMed-shaped 3.99 -> 3.78 ms, NYTimes-
// shaped 0.71 -> 0.69 ms per sweep; batches of 16 tokens per thread: two
// (128 registers) rather than one (159): PubMed-shaped word batches 3.78 ->
// 3.49 ms, its long documents 0.41 -> 0.32 ms.
template <bool kDoc, int TPT>
constexpr int batch_min_blocks() { return TPT == 4 ? 3 : (TPT == 8 ? (kDoc ? 2 : 3) : 2); }

template <bool kDoc, bool kDense, int TPT, int M>
__global__ void __launch_bounds__(kThreads, (batch_min_blocks<kDoc, TPT>())) batch_phase_kernel(
    PhaseArgs a, const int4* __restrict__ batches, int nbatch, int* __restrict__ counter,
    const int32_t* __restrict__ seg_region, int region_words, int kbits) {
    static_assert(TPT % 4 == 0, "tokens per thread come in chunks of four");
    constexpr bool kRadix = !kDoc && !kDense;
    extern __shared__ __align__(16) unsigned char smem[];
    const BatchSmem L = batch_smem_layout(a.K, kDense ? 1 : 0, region_words, TPT, kRadix ? 1 : 0);
    float* ckb_s = reinterpret_cast<float*>(smem + L.ck_off);
    int* dck_s = reinterpret_cast<int*>(smem + L.ck_off) + a.K;   // c_k deltas (dense tables)
    int* seg_tok = reinterpret_cast<int*>(smem + L.seg_off);   // [kSegsMax + 1] token offsets
    int* seg_reg = seg_tok + kSegsMax + 1;                     // [kSegsMax + 1] table offsets
    int* seg_aux = seg_reg + kSegsMax + 1;                     // [kSegsMax] hash cap / prefix base
    uint32_t* region = reinterpret_cast<uint32_t*>(smem + L.region_off);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + L.stage_off);
    uint16_t* cnt = reinterpret_cast<uint16_t*>(smem + L.cnt_off);
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total, s_batch;

    const int tid = threadIdx.x;
    const int K = a.K;
    Checks chk;
    if (tid == 0) s_batch = atomicAdd(counter, 1);
    if (kDense) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    __syncthreads();

    for (;;) {
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 br = batches[b];      // {first segment, end segment, table words, 0}
        int nseg = br.y - br.x;
        int used = br.z;
        const int base = a.seg_off[br.x];
        int end = a.seg_off[br.y];
        if (!(chk(br.x >= 0 && nseg >= 1 && nseg <= kSegsMax && br.y <= a.nseg_total, 0) &
              chk(used >= 0 && used <= region_words, 1) &
              chk(end >= base && end - (base & ~3) <= kThreads * TPT && end <= a.N, 2))) {
            nseg = 1;            // a malformed batch is skipped
            used = 0;
            end = base;
        }

        // segment table (layout precomputed at init) and cleared count tables;
        // a segment whose table would leave the region gets a one-entry hash
        // at offset 0 (wrong counts, reported, but no access out of bounds)
        for (int s = tid; s < nseg; s += kThreads) {
            const int o0 = a.seg_off[br.x + s];
            const uint32_t Ls = (uint32_t)(a.seg_off[br.x + s + 1] - o0);
            uint32_t w, cap;
            if (kDense) {
                w = Ls ? (uint32_t)(K + 1) / 2 : 0u;
                cap = 0u;
            } else {
                table_shape(Ls, (uint32_t)K, &w, &cap);
            }
            int off = seg_region[br.x + s];
            if (!chk(off >= 0 && (int64_t)off + w <= used, 3)) {
                off = 0;
                cap = 1u;
            }
            seg_tok[s] = o0 - base;
            seg_reg[s] = off;
            if (!kDense) seg_aux[s] = (int)cap;
        }
        if (tid == 0) {
            seg_tok[nseg] = end - base;
            seg_reg[nseg] = used;
        }
        for (int i = tid; i < ((used + 3) >> 2); i += kThreads)
            reinterpret_cast<uint4*>(region)[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (tid == 0) s_batch = atomicAdd(counter, 1);   // every thread has read b

        // load the tokens this thread owns: chunks of 4 consecutive positions
        const int abase = base & ~3;
        int tk[TPT];          // word-major token index (-1: not ours)
        int zz[TPT];          // topic: phase-start, then post-acceptance
        int zo[TPT];          // phase-start topic (word phase with dense tables)
        int sl[TPT];          // segment slot in the batch
        Props<M> pp[TPT];     // pending proposals, then picks
#pragma unroll
        for (int c = 0; c < TPT / 4; ++c) {
            const int q0 = abase + 4 * (c * kThreads + tid);
            int4 pv = make_int4(0, 0, 0, 0);
            int4 zv = make_int4(0, 0, 0, 0);
            int pw[4 * M];
#pragma unroll
            for (int i = 0; i < 4 * M; ++i) pw[i] = 0;
            uint4 iv = make_uint4(0u, 0u, 0u, 0u);
            if (q0 < end) {
                if (kDoc) {
                    // a document batch's tokens in word-major order: lanes
                    // reading neighbouring tokens of one word share sectors
                    pv = *reinterpret_cast<const int4*>(a.sperm + q0);
                    iv = *reinterpret_cast<const uint4*>(a.sinfo + q0);
                } else {
                    zv = *reinterpret_cast<const int4*>(a.z + q0);
                    // the chunk's 4M proposals are M aligned 16-byte words
#pragma unroll
                    for (int u = 0; u < M; ++u) {
                        const int4 x = reinterpret_cast<const int4*>(a.prop + (int64_t)q0 * M)[u];
                        pw[4 * u] = x.x;
                        pw[4 * u + 1] = x.y;
                        pw[4 * u + 2] = x.z;
                        pw[4 * u + 3] = x.w;
                    }
                }
            }
            const int pa[4] = {pv.x, pv.y, pv.z, pv.w};
            const int za[4] = {zv.x, zv.y, zv.z, zv.w};
            const uint32_t ia[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = 4 * c + v;
                const int q = q0 + v;
                const bool mine = (q >= base) && (q < end);
                bool ok = mine;
                if (kDoc && mine)
                    ok = chk.tok((uint32_t)pa[v] < (uint32_t)a.N, 4) &
                         chk.tok((int)(ia[v] >> 16) < nseg && (int)(ia[v] & 0xFFFFu) < end - base, 5);
                tk[j] = ok ? (kDoc ? pa[v] : q) : -1;
                if (kDoc) {
                    sl[j] = ok ? (int)ia[v] : 0;     // slot << 16 | position, split below
                    zz[j] = ok ? a.z[tk[j]] : 0;
                    if (ok) load_props<M>(a.prop, tk[j], pp[j].v);
                } else {
                    zz[j] = za[v];
#pragma unroll
                    for (int i = 0; i < M; ++i) pp[j].v[i] = pw[v * M + i];
                }
                if (ok) {
                    zz[j] = chk.topic(zz[j], K, 6);
#pragma unroll
                    for (int i = 0; i < M; ++i) pp[j].v[i] = chk.topic(pp[j].v[i], K, 7);
                }
            }
        }
        // segment slots and count tables: documents carry their slot and
        // position; words find the slot by one binary search per chunk of four
        int lp[TPT];          // document phase: position within the batch (document order)
#pragma unroll
        for (int c = 0; c < TPT / 4; ++c) {
            const int q0 = abase + 4 * (c * kThreads + tid);
            int slot = 0;
            if (!kDoc && q0 < end) {
                const int pf = (q0 > base ? q0 : base) - base;
                int lo = 0, hi = nseg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (seg_tok[mid] <= pf) lo = mid; else hi = mid - 1;
                }
                slot = lo;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = 4 * c + v;
                if (kDoc) {
                    lp[j] = sl[j] & 0xFFFF;
                    sl[j] = sl[j] >> 16;
                } else {
                    lp[j] = 0;
                    sl[j] = 0;
                    if (tk[j] < 0) continue;
                    const int p = q0 + v - base;
                    while (slot + 1 < nseg && seg_tok[slot + 1] <= p) ++slot;
                    sl[j] = slot;
                }
                if (tk[j] < 0) continue;
                tab_add<kDense>(region + seg_reg[sl[j]], kDense ? 0u : (uint32_t)seg_aux[sl[j]],
                                (uint32_t)zz[j]);
            }
        }
        __syncthreads();

        // M chained MH steps per token (Alg. 1, Eq. 7), then the picks of Eq. 6:
        // a topic, or -(index + 1) into the post-acceptance segment.  Every
        // operand a token's chain can need -- the counts and c_k entries of
        // its phase-start topic and of each proposal -- is loaded up front
        // for a group of tokens, so the group waits on shared memory twice;
        // the chain itself is branch-free (a token that is not ours runs on
        // topic 0 of slot 0 and has its side effects masked).
        const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
        constexpr int kGroup = 4;
#pragma unroll
        for (int g0 = 0; g0 < TPT; g0 += kGroup) {
            int toff[kGroup], tlen[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int slot = sl[g0 + u];
                toff[u] = tk[g0 + u] >= 0 ? seg_reg[slot] : 0;
                tlen[u] = max(seg_tok[slot + 1] - seg_tok[slot], 1);
            }
            int cnt_v[kGroup][M + 1];
            float ck_v[kGroup][M + 1];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int j = g0 + u;
                const bool mine = tk[j] >= 0;
                const uint32_t* tab = region + toff[u];
                const uint32_t cap = (kDense || !mine) ? 0u : (uint32_t)seg_aux[sl[j]];
#pragma unroll
                for (int i = 0; i <= M; ++i) {
                    const int k = mine ? (i == 0 ? zz[j] : pp[j].v[i - 1]) : 0;
                    cnt_v[u][i] = tab_get<kDense>(tab, cap, (uint32_t)k);
                    ck_v[u][i] = kDense ? ckb_s[k] : __ldg(a.ckb + k);
                }
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int j = g0 + u;
                const bool mine = tk[j] >= 0;
                zo[j] = zz[j];
                const int Ls = tlen[u];
                const float Lf = __int2float_rn(Ls);
                const float LG = __fadd_rn(Lf, a.G);
                const int z0 = mine ? zz[j] : 0;
                int s = z0;
                int cs = cnt_v[u][0];
                float ks = ck_v[u][0];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const uint4 r = draw((uint32_t)(mine ? tk[j] : 0), a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
                    const int t = mine ? pp[j].v[i] : s;
                    const int ct = cnt_v[u][i + 1];
                    const float kt = ck_v[u][i + 1];
                    const bool acc = (t != s) && accept(r.x, cs, ct, a.g, ks, kt);
                    s = acc ? t : s;
                    cs = acc ? ct : cs;
                    ks = acc ? kt : ks;
                    const int head = -(int)(dice(r.z, (uint32_t)Ls) + 1);
                    const int tail = (int)dice(r.z, (uint32_t)K);
                    pp[j].v[i] = coin(r.y, Lf, LG) ? head : tail;
                }
                if (kDense && mine && s != z0) {
                    atomicSub(&dck_s[z0], 1);
                    atomicAdd(&dck_s[s], 1);
                } else if (!kDense && a.ck_delta && mine && s != z0) {
                    atomicSub(&a.ck[z0], 1);
                    atomicAdd(&a.ck[s], 1);
                }
                zz[j] = mine ? s : zz[j];
                if ((kDoc || kRadix || a.word_storage) && mine) {
                    // document phase and storage-order word positioning: the
                    // new topic at its position; radix sort: the sort key
                    const int p = kDoc ? lp[j] : tk[j] - base;
                    stage[pad(p)] = (kDoc || a.word_storage) ? (uint32_t)s
                                                             : (((uint32_t)sl[j] << kbits) | (uint32_t)s);
                }
            }
        }
        __syncthreads();

        if (!kDoc && kDense && !a.word_storage) {
            // counting sort of each word's post-acceptance topics through its
            // dense table: post-acceptance counts, a block-wide exclusive scan
            // of the tables in place (16-bit prefixes), then each token takes
            // the next slot of its topic's range
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                if (tk[j] < 0 || zz[j] == zo[j]) continue;
                uint32_t* tab = region + seg_reg[sl[j]];
                atomicSub(&tab[(uint32_t)zo[j] >> 1], dense_unit((uint32_t)zo[j]));
                atomicAdd(&tab[(uint32_t)zz[j] >> 1], dense_unit((uint32_t)zz[j]));
            }
            __syncthreads();
            const int per = (used + kThreads - 1) / kThreads;
            const int w0 = tid * per, w1 = min(used, w0 + per);
            int sum = 0;
            for (int w = w0; w < w1; ++w) {
                const uint32_t x = region[w];
                sum += (int)(x & 0xFFFFu) + (int)(x >> 16);
            }
            int run = block_excl_scan(sum, warp_tot, &s_total);
            for (int w = w0; w < w1; ++w) {
                const uint32_t x = region[w];
                const int lo = (int)(x & 0xFFFFu);
                region[w] = (uint32_t)run | ((uint32_t)(run + lo) << 16);
                run += lo + (int)(x >> 16);
            }
            __syncthreads();
            for (int s = tid; s < nseg; s += kThreads)
                if (seg_tok[s + 1] > seg_tok[s]) seg_aux[s] = (int)(region[seg_reg[s]] & 0xFFFFu);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                if (tk[j] < 0) continue;
                const int slot = sl[j];
                const uint32_t k = (uint32_t)zz[j];
                const uint32_t old = atomicAdd(&region[seg_reg[slot] + (k >> 1)], dense_unit(k));
                const int g = (int)((old >> ((k & 1) * 16)) & 0xFFFFu);
                const int pos = seg_tok[slot] + g - seg_aux[slot];
                if (chk.tok(pos >= seg_tok[slot] && pos < seg_tok[slot + 1], 8)) stage[pad(pos)] = k;
            }
            __syncthreads();
        }
        const int ntok = end - base;
        if (kRadix && !a.word_storage) {
            // padding keys sort last; then the word's post-acceptance topics
            // are contiguous and ascending at [seg_tok[slot], seg_tok[slot+1])
            for (int p = ntok + tid; p < kThreads * TPT; p += kThreads) stage[pad(p)] = 0xFFFFFFFFu;
            __syncthreads();
            int sbits = 0;
            while ((1 << sbits) < nseg) ++sbits;
            block_radix_sort<TPT>(stage, cnt, sbits + kbits, warp_tot, &s_total);
            __syncthreads();
        }

        // resolve picks and write back
        const uint32_t kmask = (kRadix && !a.word_storage) ? ((1u << kbits) - 1u) : 0xFFFFFFFFu;
        if (kDoc) {
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int sb = seg_tok[sl[j]];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const int pk = pp[j].v[i];
                    const int v = (int)stage[pad(sb + (pk < 0 ? -pk - 1 : 0))];
                    pp[j].v[i] = pk < 0 ? v : pk;
                }
                if (tk[j] >= 0) {
                    store_props<M>(a.prop, tk[j], pp[j].v);
                    if (zz[j] != zo[j]) a.z[tk[j]] = zz[j];   // rejected chains leave z as it was
                }
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
                        if (pk < 0) pp[j].v[i] = (int)(stage[pad(sb - pk - 1)] & kmask);
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

    if (kDense) {
        for (int k = tid; k < K; k += kThreads) {
            const int d = dck_s[k];
            if (d != 0) atomicAdd(&a.ck[k], d);
        }
    }
    chk.publish(a.fault, kDoc ? kSiteDocBatch : kSiteWordBatch);
}

int batch_smem_bytes(int K, int stage_ck, int region_words, int tpt, int word_phase, int dense) {
    (void)stage_ck;   // c_k is staged in shared memory exactly with dense tables
    return batch_smem_layout(K, dense, region_words, tpt, (word_phase && !dense) ? 1 : 0).total;
}

template <bool kDoc, bool kDense, int TPT, int M>
static const void* kernel_ptr() {
    return (const void*)batch_phase_kernel<kDoc, kDense, TPT, M>;
}

static const void* pick_kernel(bool doc, bool dense, int tpt, int M) {
#define WL_K(D, DN, T)                                                     \
    if (doc == D && dense == DN && tpt == T) {                             \
        switch (M) {                                                       \
            case 1: return kernel_ptr<D, DN, T, 1>();                      \
            case 2: return kernel_ptr<D, DN, T, 2>();                      \
            case 3: return kernel_ptr<D, DN, T, 3>();                      \
            case 4: return kernel_ptr<D, DN, T, 4>();                      \
            default: return nullptr;                                       \
        }                                                                  \
    }
    WL_K(true, true, 8) WL_K(true, true, 16) WL_K(true, false, 4) WL_K(true, false, 8) WL_K(true, false, 16)
    WL_K(false, true, 8) WL_K(false, true, 16) WL_K(false, false, 8) WL_K(false, false, 16)
#undef WL_K
    return nullptr;
}

int batch_blocks_per_sm(int K, int stage_ck, int region_words, int tpt, int word_phase, int M,
                        int dense) {
    const int smem = batch_smem_bytes(K, stage_ck, region_words, tpt, word_phase, dense);
    const void* f = pick_kernel(!word_phase, dense != 0, tpt, M);
    if (!f) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_batch_phase(bool doc, bool dense, int tpt, const PhaseArgs& a,
                               const int4* batches, int nbatch, int* counter,
                               const int32_t* seg_region, int region_words, int kbits, int grid,
                               cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nbatch <= 0) return cudaSuccess;
    const int smem = batch_smem_bytes(a.K, a.stage_ck, region_words, tpt, doc ? 0 : 1, dense ? 1 : 0);
    const void* f = pick_kernel(doc, dense, tpt, a.M);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    PhaseArgs args = a;
    void* params[] = {&args, (void*)&batches, &nbatch, &counter, (void*)&seg_region, &region_words,
                      &kbits};
    return cudaLaunchKernel(f, dim3(grid), dim3(kThreads), params, (size_t)smem, st);
}

}  // namespace wl
