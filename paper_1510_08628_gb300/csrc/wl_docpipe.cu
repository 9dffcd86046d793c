// Pipelined document phase (Sec. 4.4, Alg. 2 document loop) for batches of
// consecutive short documents.  The work per token is that of the block
// batch tier (wl_batch.cu): the document's count table C_d of its
// phase-start topics (Sec. 5.4), M chained MH steps against it with the
// acceptance rate pi^word of Eq. 7, and M new document proposals drawn from
// the mixture of Eq. 6 by random positioning over the post-acceptance
// document (Sec. 4.3).  What differs is how the batch reaches the block:
//
//  * Each block keeps a two-slot ring in shared memory.  While it samples the
//    batch in one slot, the tokens of its next batch are already being
//    gathered into the other: the batch's word-major token list and its
//    (slot, position) tags arrive as 16-byte cp.async copies, then every
//    token's z and proposals as 4/8/16-byte cp.async gathers through that
//    list.  The gathers therefore overlap the sampling instead of stalling
//    it, and hold no registers while in flight.
//  * Tokens are dealt to threads with a stride of the block size, so every
//    warp has work in every stage and the stages' barriers stay short.
//  * Count tables with more than 2,048 topics are the paper's open-addressing
//    hash with the capacity of Sec. 5.4 (the power of two above min(2L, K)),
//    grouped into buckets of four entries: a lookup reads one bucket with a
//    single 128-bit shared-memory load, and probes on to the next bucket
//    only when the bucket is full.
#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint4 lds128_volatile(const uint32_t* p) {
    uint4 v;
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p))
                 : "memory");
    return v;
}

constexpr uint32_t kTagMask = ~((1u << kHashCountBits) - 1u);
constexpr uint32_t kCountMask = (1u << kHashCountBits) - 1u;

// Bucketed hash: topic k hashes to bucket k & nbmask; a bucket's four
// entries fill in order, so an entry that is still empty ends the search.
// Entries are (topic + 1) << 12 | count, as in the block batch tier.
__device__ __forceinline__ uint32_t bucket_match(const uint4& e, uint32_t tag) {
    return ((e.x & kTagMask) == tag) ? e.x
         : ((e.y & kTagMask) == tag) ? e.y
         : ((e.z & kTagMask) == tag) ? e.z
         : ((e.w & kTagMask) == tag) ? e.w : 0u;
}

// The count of topic k given its first bucket e (already loaded).
__device__ __forceinline__ int bucket_resolve(const uint32_t* tab, uint32_t nbmask, uint32_t k, uint4 e) {
    const uint32_t tag = (k + 1u) << kHashCountBits;
    uint32_t b = k & nbmask;
    uint32_t c = bucket_match(e, tag);
    if (c == 0u && e.w != 0u) {
        for (uint32_t n = 1; n <= nbmask; ++n) {
            b = (b + 1u) & nbmask;
            e = reinterpret_cast<const uint4*>(tab)[b];
            c = bucket_match(e, tag);
            if (c != 0u || e.w == 0u) break;
        }
    }
    return (int)(c & kCountMask);
}

__device__ __forceinline__ int bucket_get(const uint32_t* tab, uint32_t nbmask, uint32_t k) {
    const uint32_t tag = (k + 1u) << kHashCountBits;
    uint32_t b = k & nbmask;
    uint4 e = reinterpret_cast<const uint4*>(tab)[b];
    uint32_t c = bucket_match(e, tag);
    if (c == 0u && e.w != 0u) {
        // the first bucket is full and lacks the key: probe on
        for (uint32_t n = 1; n <= nbmask; ++n) {
            b = (b + 1u) & nbmask;
            e = reinterpret_cast<const uint4*>(tab)[b];
            c = bucket_match(e, tag);
            if (c != 0u || e.w == 0u) break;
        }
    }
    return (int)(c & kCountMask);
}

// Adds one occurrence of topic k; safe against concurrent adds of the block.
// An entry only ever goes from empty to its final tag, so a thread that has
// seen an entry filled knows its tag, and the first empty entry of a key's
// probe sequence is where the key belongs: a failed CAS re-reads the bucket.
__device__ __forceinline__ uint32_t bucket_add(uint32_t* tab, uint32_t nbmask, uint32_t k) {
    const uint32_t tag = (k + 1u) << kHashCountBits;
    uint32_t b = k & nbmask;
    const uint32_t limit = 8u * (nbmask + 1u) + 8u;   // each retry follows a fill or a step
    for (uint32_t n = 0; n < limit; ++n) {
        const uint4 e = lds128_volatile(tab + 4u * b);
        const uint32_t ev[4] = {e.x, e.y, e.z, e.w};
        int hit = -1, empty = -1;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            if ((ev[j] & kTagMask) == tag) hit = j;
            if (ev[j] == 0u) empty = j;
        }
        if (hit >= 0 && (empty < 0 || hit < empty)) {
            atomicAdd(&tab[4u * b + (uint32_t)hit], 1u);
            return 4u * b + (uint32_t)hit;
        }
        if (empty < 0) {
            b = (b + 1u) & nbmask;
            continue;
        }
        const uint32_t old = atomicCAS(&tab[4u * b + (uint32_t)empty], 0u, tag | 1u);
        if (old == 0u) return 4u * b + (uint32_t)empty;
        if ((old & kTagMask) == tag) {
            atomicAdd(&tab[4u * b + (uint32_t)empty], 1u);
            return 4u * b + (uint32_t)empty;
        }
        // another topic took the entry: read the bucket again
    }
    return 0u;   // not reached: the table has an empty entry for every key
}

__device__ __forceinline__ uint32_t dense_unit2(uint32_t k) { return (k & 1u) ? 65536u : 1u; }

template <int M>
__device__ __forceinline__ void cp_async_props(int32_t* dst, const int32_t* src) {
    if (M == 1) cp_async4(dst, src);
    else if (M == 2) cp_async8(dst, src);
    else if (M == 4) cp_async16(dst, src);
    else {
#pragma unroll
        for (int i = 0; i < M; ++i) cp_async4(dst + i, src + i);
    }
}

template <int M>
__device__ __forceinline__ void store_picks(int32_t* prop, int t, const int* v) {
    if (M == 2) {
        *reinterpret_cast<int2*>(prop + (int64_t)t * 2) = make_int2(v[0], v[1 % M]);
    } else if (M == 4) {
        *reinterpret_cast<int4*>(prop + (int64_t)t * 4) = make_int4(v[0], v[1 % M], v[2 % M], v[3 % M]);
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) prop[(int64_t)t * M + i] = v[i];
    }
}

// The first copies of a batch (A slot): its descriptor, word-major token
// list and tags (from a 4-aligned start), document offsets and table
// offsets.
struct SlotA {
    int4* d;          // d[0] = {first, nseg, base, ntok}, d[1] = {table words, 0, 0, 0}
    int32_t* tk;      // [T] word-major indices, from base & ~3
    uint32_t* info;   // [T] (slot << 16) | position in the batch
    int32_t* so;      // [kDocSegs + 4] document offsets
    int32_t* sr;      // [kDocSegs + 4] table offsets
};
// The gathered tokens of a batch (B slot): phase-start z and pending
// proposals by position in the sorted list.  Once the count tables are
// built, z is no longer read and holds the post-acceptance topics by
// position in the batch (document order) instead.
struct SlotB {
    int32_t* z;       // [T]
    int32_t* prop;    // [T * M]
};

__host__ __device__ inline int docpipe_slota_bytes(int T) { return 32 + T * 8 + (kDocSegs + 4) * 8; }
__host__ __device__ inline int docpipe_slotb_bytes(int T, int M) { return T * 4 * (M + 1); }

__device__ __forceinline__ SlotA slota_at(unsigned char* p, int T) {
    SlotA s;
    s.d = reinterpret_cast<int4*>(p);
    s.tk = reinterpret_cast<int32_t*>(p + 32);
    s.info = reinterpret_cast<uint32_t*>(s.tk + T);
    s.so = reinterpret_cast<int32_t*>(s.info + T);
    s.sr = s.so + kDocSegs + 4;
    return s;
}
__device__ __forceinline__ SlotB slotb_at(unsigned char* p, int T) {
    SlotB s;
    s.z = reinterpret_cast<int32_t*>(p);
    s.prop = s.z + T;
    return s;
}

}  // namespace

struct DocPipeSmem {
    int ck_off, a_off, a_bytes, b_off, b_bytes, seg_off, region_off, total;
};

// Two A slots and two B slots (a batch's first copies and its gathers go out
// one batch ahead), the segment table and the count tables; with dense
// tables also (float)c_k + beta_bar and the c_k deltas.  (A third A slot,
// to issue the first copies two batches ahead, measured 26% slower on the
// PubMed-shaped workload: the extra 9 KB per block cost a resident block
// per SM.)
__host__ __device__ inline DocPipeSmem docpipe_layout(int K, int dense, int region_words, int T, int M) {
    DocPipeSmem s;
    int o = 0;
    s.ck_off = o;
    if (dense) o += 2 * K * 4;
    o = (o + 15) & ~15;
    s.a_off = o;
    s.a_bytes = (docpipe_slota_bytes(T) + 15) & ~15;
    o += 2 * s.a_bytes;
    s.b_off = o;
    s.b_bytes = (docpipe_slotb_bytes(T, M) + 15) & ~15;
    o += 2 * s.b_bytes;
    s.seg_off = o;
    o += kDocSegs * 16;
    s.region_off = o;
    o += ((region_words + 3) & ~3) * 4;
    s.total = (o + 15) & ~15;
    return s;
}

template <bool kDense, int M, int TPT>
__global__ void __launch_bounds__(kThreads, (TPT <= 2 ? 4 : 3)) doc_pipe_kernel(
    PhaseArgs a, const int4* __restrict__ desc, int nbatch, int* __restrict__ counter,
    const int32_t* __restrict__ seg_region, int region_words) {
    constexpr int T = kThreads * TPT;
    extern __shared__ __align__(16) unsigned char smem[];
    const DocPipeSmem L = docpipe_layout(a.K, kDense ? 1 : 0, region_words, T, M);
    float* ckb_s = reinterpret_cast<float*>(smem + L.ck_off);
    int* dck_s = reinterpret_cast<int*>(smem + L.ck_off) + a.K;
    auto slot_a = [&](int i) { return slota_at(smem + L.a_off + i * L.a_bytes, T); };
    auto slot_b = [&](int i) { return slotb_at(smem + L.b_off + i * L.b_bytes, T); };
    int4* segtab = reinterpret_cast<int4*>(smem + L.seg_off);   // {position, length, table, bucket mask}
    uint32_t* region = reinterpret_cast<uint32_t*>(smem + L.region_off);
    __shared__ int s_claim[2];

    const int tid = threadIdx.x;
    const int K = a.K;
    Checks chk;

    // First copies of batch b into an A slot: descriptor (validated), token
    // list and tags, document and table offsets.  A batch id past the end
    // leaves the slot empty.
    auto stage1 = [&](int b, const SlotA& s) {
        int4 br = make_int4(0, 0, 0, 0);
        bool ok = b < nbatch;
        if (ok) {
            br = desc[b];   // {first, nseg | words << 16, base, ntok}
            const int nseg = br.y & 0xFFFF, words = (int)((uint32_t)br.y >> 16);
            ok = chk(br.x >= 0 && nseg >= 1 && nseg <= kDocSegs && (int64_t)br.x + nseg <= a.nseg_total &&
                         words <= region_words && br.z >= 0 && br.w >= 1 && br.w <= T - 3 &&
                         (int64_t)br.z + br.w <= a.N, 0);
        }
        const int nseg = ok ? (br.y & 0xFFFF) : 0;
        if (tid == 0) {
            s.d[0] = ok ? make_int4(br.x, nseg, br.z, br.w) : make_int4(0, 0, 0, 0);
            s.d[1] = make_int4(ok ? (int)((uint32_t)br.y >> 16) : 0, 0, 0, 0);
        }
        if (!ok) return;
        const int abase = br.z & ~3;
        const int nch = (br.z - abase + br.w + 3) >> 2;   // 16-byte chunks covering the batch
        for (int c = tid; c < nch; c += kThreads) {
            cp_async16(s.tk + 4 * c, a.sperm + abase + 4 * c);
            cp_async16(s.info + 4 * c, a.sinfo + abase + 4 * c);
        }
        for (int i = tid; i <= nseg; i += kThreads) cp_async4(s.so + i, a.seg_off + br.x + i);
        for (int i = tid; i < nseg; i += kThreads) cp_async4(s.sr + i, seg_region + br.x + i);
    };

    // Gathers of a batch's z and proposals through its token list (its first
    // copies have landed).
    auto gathers = [&](const SlotA& s, const SlotB& g) {
        const int4 d0 = s.d[0];
        const int ntok = d0.w, o = d0.z & 3;
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int p = tid + j * kThreads;
            if (p >= ntok) continue;
            const int t = s.tk[o + p];
            if (!chk.tok((uint32_t)t < (uint32_t)a.N, 4)) continue;
            cp_async4(g.z + p, a.z + t);
            cp_async_props<M>(g.prop + M * p, a.prop + (int64_t)t * M);
        }
    };

    // Segment table and cleared count tables of a batch (its first copies
    // have landed; the previous batch no longer reads either).
    auto setup = [&](const SlotA& s) {
        const int4 d0 = s.d[0];
        const int nseg = d0.y, base = d0.z, ntok = d0.w, words = s.d[1].x;
        for (int i = tid; i < nseg; i += kThreads) {
            const int o0 = s.so[i], Ls = s.so[i + 1] - o0, reg = s.sr[i];
            int w = 0;
            if (Ls > 0) w = kDense ? (K + 1) / 2 : (int)pow2_above((uint32_t)min(2 * Ls, K));
            const bool ok = chk(o0 >= base && Ls >= 0 && (int64_t)o0 + Ls <= (int64_t)base + ntok && reg >= 0 &&
                                    reg + w <= words && (kDense || Ls == 0 || ((reg & 3) == 0 && w >= 4)), 3);
            segtab[i] = ok ? make_int4(o0 - base, Ls, reg, kDense ? 0 : (w >> 2) - 1) : make_int4(0, -1, 0, 0);
        }
        for (int i = tid; i < ((words + 3) >> 2); i += kThreads)
            reinterpret_cast<uint4*>(region)[i] = make_uint4(0u, 0u, 0u, 0u);
    };

    if (kDense) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    if (tid == 0) {
        s_claim[0] = atomicAdd(counter, 1);
        s_claim[1] = atomicAdd(counter, 1);
    }
    __syncthreads();
    int b0 = s_claim[0], b1 = s_claim[1];   // batches i, i+1
    stage1(b0, slot_a(0));
    stage1(b1, slot_a(1));
    cp_commit();
    cp_wait_all();
    __syncthreads();
    gathers(slot_a(0), slot_b(0));
    cp_commit();
    setup(slot_a(0));

    // Batch i lives in slots i % 2.  Three barriers per batch: (1) its
    // gathers and table set-up are complete, and so are the next batch's
    // first copies; (2) its count tables are built; (3) its chains are done
    // -- then batch i+2 gets its first copies in this batch's A slot, this
    // batch is written back and the next one's tables are set up.
    const uint32_t phase = kPhaseDoc;
    int cur = 0;
    while (b0 < nbatch) {
        cp_wait_all();
        __syncthreads();                                                   // (1)
        gathers(slot_a(cur ^ 1), slot_b(cur ^ 1));   // in flight while this batch is sampled
        cp_commit();
        const SlotA s = slot_a(cur);
        const SlotB g = slot_b(cur);
        const int4 d0 = s.d[0];
        const int nseg = d0.y, ntok = d0.w, o = d0.z & 3;

        // C_d of the phase-start topics; each token keeps its topic and, with
        // hash tables, its own entry
        uint32_t ent[TPT];
        int z0v[TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int p = tid + j * kThreads;
            ent[j] = 0u;
            z0v[j] = 0;
            if (p >= ntok) continue;
            const uint32_t inf = s.info[o + p];
            const int sl = (int)(inf >> 16);
            if (!chk.tok(sl < nseg, 5)) continue;
            const int4 sg = segtab[sl];
            if (sg.y <= 0) continue;
            const uint32_t k = (uint32_t)chk.topic(g.z[p], K, 6);
            z0v[j] = (int)k;
            if (kDense) atomicAdd(&region[sg.z + (int)(k >> 1)], dense_unit2(k));
            else ent[j] = (uint32_t)sg.z + bucket_add(region + sg.z, (uint32_t)sg.w, k);
        }
        __syncthreads();                                                   // (2)
        if (tid == 0) s_claim[0] = atomicAdd(counter, 1);

        // M chained MH steps per token (Eq. 7) and the picks of Eq. 6: a
        // topic, or -(position + 1) of a token of the post-acceptance
        // document.  The post-acceptance topics go to g.z by position.
        int32_t* const stage = g.z;
        int tkv[TPT], sv[TPT], pk[TPT][M];
        bool mine[TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int p = tid + j * kThreads;
            mine[j] = false;
            tkv[j] = 0;
            sv[j] = 0;
#pragma unroll
            for (int i = 0; i < M; ++i) pk[j][i] = 0;
            if (p >= ntok) continue;
            const uint32_t inf = s.info[o + p];
            const int sl = (int)(inf >> 16), lp = (int)(inf & 0xFFFFu);
            if (!chk.tok(sl < nseg && lp < ntok, 5)) continue;
            const int4 sg = segtab[sl];
            if (sg.y <= 0) continue;
            const int t = s.tk[o + p];
            if (!chk.tok((uint32_t)t < (uint32_t)a.N, 4)) continue;
            const int z0 = z0v[j];
            int pr[M];
#pragma unroll
            for (int i = 0; i < M; ++i) pr[i] = chk.topic(g.prop[M * p + i], K, 7);
            const uint32_t* tab = region + sg.z;
            int cnt[M + 1];
            float ckv[M + 1];
            uint4 rr[M];
            if (kDense) {
#pragma unroll
                for (int i = 0; i <= M; ++i) {
                    const uint32_t k = (uint32_t)(i == 0 ? z0 : pr[i - 1]);
                    cnt[i] = (int)((tab[k >> 1] >> ((k & 1u) * 16u)) & 0xFFFFu);
                    ckv[i] = ckb_s[k];
                }
#pragma unroll
                for (int i = 0; i < M; ++i) rr[i] = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
            } else {
                // the loads first (own entry, the proposals' first buckets,
                // c_k), then the Philox blocks while they are in flight, then
                // the bucket matches
                uint4 eb[M];
                cnt[0] = (int)(region[ent[j]] & kCountMask);
                ckv[0] = __ldg(a.ckb + z0);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    eb[i] = reinterpret_cast<const uint4*>(tab)[(uint32_t)pr[i] & (uint32_t)sg.w];
                    ckv[i + 1] = __ldg(a.ckb + pr[i]);
                }
#pragma unroll
                for (int i = 0; i < M; ++i) rr[i] = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
#pragma unroll
                for (int i = 0; i < M; ++i) cnt[i + 1] = bucket_resolve(tab, (uint32_t)sg.w, (uint32_t)pr[i], eb[i]);
            }
            const float Lf = __int2float_rn(sg.y);
            const float LG = __fadd_rn(Lf, a.G);
            int sc = z0, cs = cnt[0];
            float ks = ckv[0];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const uint4 r = rr[i];
                const int tp = pr[i];
                const bool acc = (tp != sc) && accept(r.x, cs, cnt[i + 1], a.g, ks, ckv[i + 1]);
                sc = acc ? tp : sc;
                cs = acc ? cnt[i + 1] : cs;
                ks = acc ? ckv[i + 1] : ks;
                pk[j][i] = coin(r.y, Lf, LG) ? -(sg.x + (int)dice(r.z, (uint32_t)sg.y) + 1)
                                             : (int)dice(r.z, (uint32_t)K);
            }
            mine[j] = true;
            tkv[j] = t;
            sv[j] = sc;
            if (sc != z0) {
                if (kDense) {
                    atomicSub(&dck_s[z0], 1);
                    atomicAdd(&dck_s[sc], 1);
                } else if (a.ck_delta) {
                    atomicSub(&a.ck[z0], 1);
                    atomicAdd(&a.ck[sc], 1);
                }
            }
        }
        // every thread has read its g.z entries (before barrier (2)); the
        // stores by position start now
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            if (!mine[j]) continue;
            const int p = tid + j * kThreads;
            stage[(int)(s.info[o + p] & 0xFFFFu)] = sv[j];
        }
        __syncthreads();                                                   // (3)
        const int b2 = s_claim[0];
        stage1(b2, s);              // batch i+2 takes this A slot
        cp_commit();

        // resolve the picks against the post-acceptance document and write
        // back through the token list (z only where the chain moved it)
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            if (!mine[j]) continue;
            int v[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const int q = pk[j][i];
                int pos = q < 0 ? -q - 1 : 0;
                if (!chk.tok(pos < ntok, 8)) pos = 0;
                v[i] = q < 0 ? stage[pos] : q;
            }
            store_picks<M>(a.prop, tkv[j], v);
            if (sv[j] != z0v[j]) a.z[tkv[j]] = sv[j];
        }
        setup(slot_a(cur ^ 1));     // the next batch's tables (this one's are done)
        b0 = b1;
        b1 = b2;
        cur ^= 1;
    }
    cp_wait_all();

    if (kDense) {
        __syncthreads();
        for (int k = tid; k < K; k += kThreads) {
            const int d = dck_s[k];
            if (d != 0) atomicAdd(&a.ck[k], d);
        }
    }
    chk.publish(a.fault, kSiteDocBatch);
}

int docpipe_smem_bytes(int K, int dense, int region_words, int tpt, int M) {
    return docpipe_layout(K, dense, region_words, kThreads * tpt, M).total;
}

template <bool kDense, int M, int TPT>
static const void* docpipe_ptr() {
    return (const void*)doc_pipe_kernel<kDense, M, TPT>;
}

static const void* docpipe_pick(bool dense, int tpt, int M) {
#define WL_DP(DN, TP)                                          \
    if (dense == DN && tpt == TP) {                            \
        switch (M) {                                           \
            case 1: return docpipe_ptr<DN, 1, TP>();           \
            case 2: return docpipe_ptr<DN, 2, TP>();           \
            case 3: return docpipe_ptr<DN, 3, TP>();           \
            case 4: return docpipe_ptr<DN, 4, TP>();           \
            default: return nullptr;                           \
        }                                                      \
    }
    WL_DP(true, 2) WL_DP(false, 2) WL_DP(true, 4) WL_DP(false, 4)
#undef WL_DP
    return nullptr;
}

int docpipe_blocks_per_sm(int K, int dense, int region_words, int tpt, int M) {
    const void* f = docpipe_pick(dense != 0, tpt, M);
    if (!f) return 0;
    const int smem = docpipe_smem_bytes(K, dense, region_words, tpt, M);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_doc_pipe(bool dense, int tpt, const PhaseArgs& a, const int4* desc, int nbatch,
                            int* counter, const int32_t* seg_region, int region_words, int grid,
                            cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (nbatch <= 0) return cudaSuccess;
    const void* f = docpipe_pick(dense, tpt, a.M);
    if (!f) return cudaErrorInvalidValue;
    const int smem = docpipe_smem_bytes(a.K, dense ? 1 : 0, region_words, tpt, a.M);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    PhaseArgs args = a;
    void* params[] = {&args, (void*)&desc, &nbatch, &counter, (void*)&seg_region, &region_words};
    return cudaLaunchKernel(f, dim3(grid), dim3(kThreads), params, (size_t)smem, st);
}

}  // namespace wl
