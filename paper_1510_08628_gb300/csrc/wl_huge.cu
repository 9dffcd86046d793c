// Multi-pass tier of the document and word phases for segments with more
// tokens than one block batch holds (the paper's intra-word parallelism for
// frequent words, Sec. 5.4).  The tier's tokens are cut into equal ranges of
// consecutive tokens; a range is a list of pieces, each piece a run of one
// segment's tokens.  Blocks take ranges from a work counter, so a block
// walks long runs of one segment and loads that segment's count row (K ints,
// global memory) once per piece.  Per phase:
//   hist   : row = histogram of the segment's z (before acceptance; for
//            words, once more after acceptance)
//   accept : M chained MH steps per token against the phase-start row
//            (Eq. 7), z written
//   draw   : M proposals per token from Eq. 6 -- positioning through perm
//            over the post-acceptance document, or the j-th smallest
//            post-acceptance topic of the word (inverse CDF of its row).
// Word pieces are contiguous in the word-major arrays and are streamed with
// 128-bit loads and stores, the next vectors loaded while the current ones
// are processed.  For words, the accept pass draws each token's Philox
// blocks once and stores its picks in the consumed proposal slots; the draw
// pass only resolves ranks.  For long documents the draw pass recomputes the
// blocks.
#include <algorithm>

#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

// 16-byte vectors per thread per array per step: two in the histogram
// pass, one in the accept and draw passes, whose next vectors are already
// loaded while the current ones are processed (two there held 80 registers
// for three blocks per SM; one: PubMed-shaped accept 5.82 -> 5.34 ms, draw
// 4.50 -> 4.41 ms per sweep, the histograms 0.70 -> 0.79 ms)
constexpr int kHistUnroll = 2;
constexpr int kVecUnroll = 1;

__device__ __forceinline__ int elem(const int4& v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// A piece {row, segment, first position, length}: valid when it lies in its
// segment and names an existing count row.
__device__ __forceinline__ bool piece_ok(const PhaseArgs& a, const int4& ch, int nrows) {
    if (ch.x < 0 || ch.x >= nrows || ch.y < 0 || (int64_t)ch.y >= a.nseg_total || ch.w < 0) return false;
    const int s0 = a.seg_off[ch.y], s1 = a.seg_off[ch.y + 1];
    return ch.z >= s0 && (int64_t)ch.z + ch.w <= s1;
}

// The next range of the block (uniform over the block): its pieces
// [*pc0, *pc1), or false when the ranges are exhausted.
__device__ __forceinline__ bool next_range(const HugeWork& w, int* s_r, Checks& chk, int* pc0,
                                           int* pc1) {
    if (threadIdx.x == 0) *s_r = atomicAdd(w.counter, 1);
    __syncthreads();
    const int r = *s_r;
    __syncthreads();
    if (r >= w.nranges) return false;
    *pc0 = w.range_off[r];
    *pc1 = w.range_off[r + 1];
    if (!chk(0 <= *pc0 && *pc0 <= *pc1 && *pc1 <= w.npieces, 0)) *pc1 = *pc0;
    return true;
}

__device__ __forceinline__ int4 get_piece(const PhaseArgs& a, const HugeWork& w, int pc, Checks& chk) {
    int4 ch = w.pieces[pc];
    if (!chk(piece_ok(a, ch, w.nrows), 1)) ch = make_int4(0, 0, 0, 0);
    return ch;
}

// Buckets of the rank guide table of the word draw: the power of two of at
// least 2K (so that a bucket spans about half a topic or less), 4096 to 8192.
// Capped at 8192: with K = 10^4 a 16384-bucket guide took 64 KB and left two
// blocks per SM, the 8192-bucket one three (draw 4.97 -> 4.50 ms per
// PubMed-shaped sweep; 4096 buckets made the walks longer: 5.08 ms).
int huge_guide_bits(int K) {
    int b = 12;
    while (b < 13 && (1 << b) < 2 * K) ++b;
    return b;
}

int huge_smem_bytes(int K, int stage_ck, int pass, bool doc) {
    // pass 0 hist: K; pass 1 accept: row + staged c_k and deltas; pass 2
    // draw: (words) K+1 prefix + guide table
    int words = 0;
    if (pass == 0) words = K;
    else if (pass == 1) words = K + (stage_ck ? 2 * K : 0);
    else words = doc ? 0 : K + 1 + (1 << huge_guide_bits(K));
    return ((words * 4) + 15) & ~15;
}

template <bool kDoc>
__global__ void __launch_bounds__(kThreads) huge_hist_kernel(PhaseArgs a, HugeWork w,
                                                             int32_t* __restrict__ rows) {
    extern __shared__ __align__(16) int hist[];
    __shared__ int s_r;
    const int K = a.K, tid = threadIdx.x;
    Checks chk;
    int pc0, pc1;
    while (next_range(w, &s_r, chk, &pc0, &pc1)) {
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 ch = get_piece(a, w, pc, chk);
            const int p0 = ch.z, p1 = ch.z + ch.w;
            for (int k = tid; k < K; k += kThreads) hist[k] = 0;
            __syncthreads();
            if (kDoc) {
                for (int p = p0 + tid; p < p1; p += kThreads) {
                    const int t = a.perm[p];
                    if (!chk.tok((uint32_t)t < (uint32_t)a.N, 2)) continue;
                    atomicAdd(&hist[chk.topic(a.z[t], K, 3)], 1);
                }
            } else {
                const int v0 = p0 >> 2, v1 = (p1 + 3) >> 2;
                const int4* zv = reinterpret_cast<const int4*>(a.z);
                for (int vb = v0 + tid; vb < v1; vb += kThreads * kHistUnroll) {
                    int4 x[kHistUnroll];
#pragma unroll
                    for (int u = 0; u < kHistUnroll; ++u) {
                        const int v = vb + u * kThreads;
                        if (v < v1) x[u] = zv[v];
                    }
#pragma unroll
                    for (int u = 0; u < kHistUnroll; ++u) {
                        const int v = vb + u * kThreads;
                        if (v >= v1) continue;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = 4 * v + e;
                            if (q >= p0 && q < p1) atomicAdd(&hist[chk.topic(elem(x[u], e), K, 3)], 1);
                        }
                    }
                }
            }
            __syncthreads();
            int32_t* row = rows + (int64_t)ch.x * K;
            for (int k = tid; k < K; k += kThreads)
                if (hist[k] != 0) atomicAdd(&row[k], hist[k]);
            __syncthreads();
        }
    }
    chk.publish(a.fault, kSiteHugeHist);
}

// M chained MH steps of one token from z0 against the count row (Eq. 7).
template <int M>
__device__ __forceinline__ int mh_chain(const PhaseArgs& a, uint32_t t, uint32_t phase, int z0,
                                        const int* pr, const int* row, const float* ckb_s) {
    int s = z0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int tp = pr[i];
        if (tp != s) {
            const uint4 r = draw(t, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
            const float cs = a.stage_ck ? ckb_s[s] : __ldg(a.ckb + s);
            const float ct = a.stage_ck ? ckb_s[tp] : __ldg(a.ckb + tp);
            if (accept(r.x, row[s], row[tp], a.g, cs, ct)) s = tp;
        }
    }
    return s;
}

template <bool kDoc, int M>
__global__ void __launch_bounds__(kThreads, (M <= 2 ? 3 : 2)) huge_accept_kernel(PhaseArgs a, HugeWork w,
                                                               const int32_t* __restrict__ rows_pre) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_r;
    const int K = a.K, tid = threadIdx.x;
    int* row = sm;
    float* ckb_s = reinterpret_cast<float*>(sm + K);
    int* dck_s = sm + 2 * K;   // c_k deltas (with stage_ck)
    Checks chk;
    if (a.stage_ck) {
        for (int k = tid; k < K; k += kThreads) {
            ckb_s[k] = a.ckb[k];
            dck_s[k] = 0;
        }
    }
    auto delta = [&](int z0, int s) {
        if (a.stage_ck && s != z0) {
            atomicSub(&dck_s[z0], 1);
            atomicAdd(&dck_s[s], 1);
        } else if (a.ck_delta && s != z0) {
            atomicSub(&a.ck[z0], 1);
            atomicAdd(&a.ck[s], 1);
        }
    };
    const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
    int pc0, pc1;
    while (next_range(w, &s_r, chk, &pc0, &pc1)) {
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 ch = get_piece(a, w, pc, chk);
            const int p0 = ch.z, p1 = ch.z + ch.w;
            const int4* rp = reinterpret_cast<const int4*>(rows_pre + (int64_t)ch.x * K);
            if ((K & 3) == 0) {
                for (int k = tid; k < (K >> 2); k += kThreads) reinterpret_cast<int4*>(row)[k] = rp[k];
            } else {
                for (int k = tid; k < K; k += kThreads) row[k] = rows_pre[(int64_t)ch.x * K + k];
            }
            __syncthreads();
            if (kDoc) {
                for (int p = p0 + tid; p < p1; p += kThreads) {
                    const int t = a.perm[p];
                    if (!chk.tok((uint32_t)t < (uint32_t)a.N, 2)) continue;
                    const int z0 = chk.topic(a.z[t], K, 3);
                    int pr[M];
#pragma unroll
                    for (int i = 0; i < M; ++i) pr[i] = chk.topic(a.prop[(int64_t)t * M + i], K, 4);
                    const int s = mh_chain<M>(a, (uint32_t)t, phase, z0, pr, row, ckb_s);
                    if (s != z0) a.z[t] = s;
                    delta(z0, s);
                }
            } else {
                // word piece: 128-bit loads of z and of the proposals, the next
                // step's vectors in flight while this step's are processed; the
                // M blocks of each token are drawn here once, the accept uses r0
                // and the pick of Eq. 6 (a topic, or -(rank + 1) resolved by the
                // draw pass) is written over the consumed proposal
                const int Ls = a.seg_off[ch.y + 1] - a.seg_off[ch.y];
                const float Lf = __int2float_rn(Ls);
                const float LG = __fadd_rn(Lf, a.G);
                const int v0 = p0 >> 2, v1 = (p1 + 3) >> 2;
                int4* zv = reinterpret_cast<int4*>(a.z);
                int4* pv = reinterpret_cast<int4*>(a.prop);
                constexpr int kStep = kThreads * kVecUnroll;
                int4 xn[kVecUnroll], yn[kVecUnroll][M];
                auto load = [&](int vb) {
#pragma unroll
                    for (int u = 0; u < kVecUnroll; ++u) {
                        const int v = vb + u * kThreads;
                        if (v < v1) {
                            xn[u] = zv[v];
#pragma unroll
                            for (int i = 0; i < M; ++i) yn[u][i] = pv[(int64_t)v * M + i];
                        }
                    }
                };
                load(v0 + tid);
                for (int vb = v0 + tid; vb < v1; vb += kStep) {
                    int4 x[kVecUnroll], y[kVecUnroll][M];
#pragma unroll
                    for (int u = 0; u < kVecUnroll; ++u) {
                        x[u] = xn[u];
#pragma unroll
                        for (int i = 0; i < M; ++i) y[u][i] = yn[u][i];
                    }
                    if (vb + kStep < v1) load(vb + kStep);
#pragma unroll
                    for (int u = 0; u < kVecUnroll; ++u) {
                        const int v = vb + u * kThreads;
                        if (v >= v1) continue;
                        int out[4], pk[4 * M];
                        bool full = true;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = 4 * v + e;
                            out[e] = elem(x[u], e);
#pragma unroll
                            for (int i = 0; i < M; ++i) pk[e * M + i] = 0;
                            if (q < p0 || q >= p1) { full = false; continue; }
                            const int z0 = chk.topic(out[e], K, 3);
                            // the counts and c_k of z and of every proposal
                            // are loaded first, then the Philox blocks are
                            // drawn while the loads are in flight
                            int tpv[M], rt[M];
                            float kt[M];
                            const int rz = row[z0];
                            const float kz = a.stage_ck ? ckb_s[z0] : __ldg(a.ckb + z0);
#pragma unroll
                            for (int i = 0; i < M; ++i) {
                                tpv[i] = chk.topic(elem(y[u][(e * M + i) / 4], (e * M + i) % 4), K, 4);
                                rt[i] = row[tpv[i]];
                                kt[i] = a.stage_ck ? ckb_s[tpv[i]] : __ldg(a.ckb + tpv[i]);
                            }
                            uint4 rr[M];
#pragma unroll
                            for (int i = 0; i < M; ++i) rr[i] = draw((uint32_t)q, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
                            int s = z0, cs = rz;
                            float ks = kz;
#pragma unroll
                            for (int i = 0; i < M; ++i) {
                                if (tpv[i] != s && accept(rr[i].x, cs, rt[i], a.g, ks, kt[i])) {
                                    s = tpv[i];
                                    cs = rt[i];
                                    ks = kt[i];
                                }
                                pk[e * M + i] = coin(rr[i].y, Lf, LG) ? -(int)(dice(rr[i].z, (uint32_t)Ls) + 1)
                                                                      : (int)dice(rr[i].z, (uint32_t)K);
                            }
                            delta(z0, s);
                            out[e] = s;
                        }
                        if (full) {
                            zv[v] = make_int4(out[0], out[1], out[2], out[3]);
#pragma unroll
                            for (int i = 0; i < M; ++i)
                                pv[(int64_t)v * M + i] = make_int4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int q = 4 * v + e;
                                if (q < p0 || q >= p1) continue;
                                a.z[q] = out[e];
#pragma unroll
                                for (int i = 0; i < M; ++i) a.prop[(int64_t)q * M + i] = pk[e * M + i];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (a.stage_ck) {
        __syncthreads();
        for (int k = tid; k < K; k += kThreads)
            if (dck_s[k] != 0) atomicAdd(&a.ck[k], dck_s[k]);
    }
    chk.publish(a.fault, kSiteHugeAccept);
}

template <bool kDoc, int M>
__global__ void __launch_bounds__(kThreads) huge_draw_kernel(PhaseArgs a, HugeWork w,
                                                             const int32_t* __restrict__ rows_post) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int warp_tot[kWarps];
    __shared__ int s_total, s_r;
    const int K = a.K, tid = threadIdx.x;
    int* P = sm;   // word phase: exclusive prefix of the post-acceptance row, P[K] = L_w
    int* guide = P + K + 1;
    const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
    Checks chk;
    int pc0, pc1;
    while (next_range(w, &s_r, chk, &pc0, &pc1)) {
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 ch = get_piece(a, w, pc, chk);
            const int sb = a.seg_off[ch.y];
            const int Ls = max(a.seg_off[ch.y + 1] - sb, 1);
            const int p0 = ch.z, p1 = ch.z + ch.w;
            const float Lf = __int2float_rn(Ls);
            const float LG = __fadd_rn(Lf, a.G);
            if (kDoc) {
                for (int p = p0 + tid; p < p1; p += kThreads) {
                    const int t = a.perm[p];
#pragma unroll
                    for (int i = 0; i < M; ++i) {
                        const uint4 r = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
                        int k = (int)dice(r.z, (uint32_t)K);
                        if (coin(r.y, Lf, LG)) {
                            const int tq = a.perm[sb + (int)dice(r.z, (uint32_t)Ls)];
                            if (chk.tok((uint32_t)tq < (uint32_t)a.N, 2)) k = a.z[tq];
                        }
                        a.prop[(int64_t)t * M + i] = k;
                    }
                }
                continue;   // no shared state between pieces
            }
            const bool storage = a.word_storage != 0;   // uniform
            const int gb = w.guide_bits, nb = 1 << gb;
            const uint64_t mult = (1ull << (32 + gb)) / (uint64_t)Ls;
            auto bucket_of = [&](int j) { return j < 0 ? -1 : (int)(((uint64_t)j * mult) >> 32); };
            // exclusive prefix of the word's post-acceptance row: the row is
            // copied in, each thread sums a contiguous run of topics, one
            // block scan, then the runs become prefixes
            const int32_t* rq = rows_post + (int64_t)ch.x * K;
            if (!storage) {
            for (int k = tid; k < K; k += kThreads) P[k] = rq[k];
            __syncthreads();
            const int per = (K + kThreads - 1) / kThreads;
            const int k0 = min(K, tid * per), k1 = min(K, k0 + per);
            int sum = 0;
            for (int k = k0; k < k1; ++k) sum += P[k];
            int run = block_excl_scan(sum, warp_tot, &s_total);
            for (int k = k0; k < k1; ++k) {
                const int c = P[k];
                P[k] = run;
                run += c;
            }
            if (tid == 0) P[K] = s_total;
            __syncthreads();
            // rank j lies in bucket B(j) = (j * floor(2^(32+gb) / L)) >> 32
            // (non-decreasing in j).  Topic k fills the buckets that first
            // occur inside its ranks, (B(P[k]-1), B(P[k+1]-1)], so guide[b]
            // is the topic of the smallest rank of bucket b: a lower bound
            // for every rank of the bucket, from which the lookup walks up

            for (int k = k0; k < k1; ++k) {
                const int b0 = bucket_of(P[k] - 1) + 1, b1 = min(bucket_of(P[k + 1] - 1), nb - 1);
                for (int b = b0; b <= b1; ++b) guide[b] = k;
            }
            for (int b = max(0, bucket_of(Ls - 1) + 1) + tid; b < nb; b += kThreads) guide[b] = K - 1;
            __syncthreads();
            }
            // resolve the picks the accept pass stored: a rank j < L_w becomes
            // the j-th smallest post-acceptance topic of the word
            const int v0 = p0 >> 2, v1 = (p1 + 3) >> 2;
            int4* pv = reinterpret_cast<int4*>(a.prop);
            constexpr int kStep = kThreads * kVecUnroll;
            int4 yn[kVecUnroll][M];
            auto load = [&](int vb) {
#pragma unroll
                for (int u = 0; u < kVecUnroll; ++u) {
                    const int v = vb + u * kThreads;
                    if (v < v1)
#pragma unroll
                        for (int i = 0; i < M; ++i) yn[u][i] = pv[(int64_t)v * M + i];
                }
            };
            load(v0 + tid);
            for (int vb = v0 + tid; vb < v1; vb += kStep) {
                int4 y[kVecUnroll][M];
#pragma unroll
                for (int u = 0; u < kVecUnroll; ++u)
#pragma unroll
                    for (int i = 0; i < M; ++i) y[u][i] = yn[u][i];
                if (vb + kStep < v1) load(vb + kStep);
#pragma unroll
                for (int u = 0; u < kVecUnroll; ++u) {
                    const int v = vb + u * kThreads;
                    if (v >= v1) continue;
                    int out[4 * M], jv[4 * M], kg[4 * M], nx[4 * M];
#pragma unroll
                    for (int n = 0; n < 4 * M; ++n) {
                        // only this piece's tokens: an edge vector's other
                        // entries belong to a neighbouring piece or word
                        const int q = 4 * v + n / M;
                        int pk = elem(y[u][n / 4], n % 4);
                        if (q < p0 || q >= p1) pk = 0;
                        out[n] = pk;
                        int j = pk < 0 ? -pk - 1 : -1;
                        if (pk < 0 && !chk.tok((uint32_t)j < (uint32_t)Ls, 5)) j = 0;
                        jv[n] = j;
                    }
                    if (storage) {
#pragma unroll
                        for (int n = 0; n < 4 * M; ++n)   // positioning: the j-th token's new topic
                            if (jv[n] >= 0) out[n] = a.z[sb + min(jv[n], Ls - 1)];
                    } else {
                        // every pick's guide entry and the prefix after it
                        // are loaded first, then the short walks
#pragma unroll
                        for (int n = 0; n < 4 * M; ++n) kg[n] = jv[n] >= 0 ? guide[bucket_of(jv[n])] : 0;
#pragma unroll
                        for (int n = 0; n < 4 * M; ++n) nx[n] = P[kg[n] + 1];
#pragma unroll
                        for (int n = 0; n < 4 * M; ++n) {
                            if (jv[n] < 0) continue;
                            int k = kg[n], next = nx[n];
                            while (k + 1 < K && next <= jv[n]) next = P[++k + 1];
                            out[n] = chk.tok(next > jv[n], 6) ? k : 0;
                        }
                    }
                    const bool full = (4 * v >= p0) && (4 * v + 3 < p1);
                    if (full) {
#pragma unroll
                        for (int i = 0; i < M; ++i)
                            pv[(int64_t)v * M + i] = make_int4(out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = 4 * v + e;
                            if (q < p0 || q >= p1) continue;
#pragma unroll
                            for (int i = 0; i < M; ++i) a.prop[(int64_t)q * M + i] = out[e * M + i];
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    chk.publish(a.fault, kSiteHugeDraw);
}

template <typename F>
static cudaError_t set_smem(F f, int smem) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_huge_hist(bool doc, const PhaseArgs& a, const HugeWork& w, int32_t* rows,
                             int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (w.npieces <= 0) return cudaSuccess;
    const int smem = huge_smem_bytes(a.K, a.stage_ck, 0, doc);
    if (doc) {
        cudaError_t e = set_smem(huge_hist_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        huge_hist_kernel<true><<<grid, kThreads, smem, st>>>(a, w, rows);
    } else {
        cudaError_t e = set_smem(huge_hist_kernel<false>, smem);
        if (e != cudaSuccess) return e;
        huge_hist_kernel<false><<<grid, kThreads, smem, st>>>(a, w, rows);
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

cudaError_t launch_huge_accept(bool doc, const PhaseArgs& a, const HugeWork& w,
                               const int32_t* rows_pre, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (w.npieces <= 0) return cudaSuccess;
    const int smem = huge_smem_bytes(a.K, a.stage_ck, 1, doc);
    cudaError_t e = cudaSuccess;
    if (doc) {
        WL_M_SWITCH({
            e = set_smem(huge_accept_kernel<true, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_accept_kernel<true, MM><<<grid, kThreads, smem, st>>>(a, w, rows_pre);
        })
    } else {
        WL_M_SWITCH({
            e = set_smem(huge_accept_kernel<false, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_accept_kernel<false, MM><<<grid, kThreads, smem, st>>>(a, w, rows_pre);
        })
    }
    return cudaGetLastError();
}

cudaError_t launch_huge_draw(bool doc, const PhaseArgs& a, const HugeWork& w,
                             const int32_t* rows_post, int grid, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (w.npieces <= 0) return cudaSuccess;
    // storage-order word positioning reads z directly: no prefix, no guide
    const int smem = a.word_storage ? 0 : huge_smem_bytes(a.K, a.stage_ck, 2, doc);
    cudaError_t e = cudaSuccess;
    if (doc) {
        WL_M_SWITCH({
            e = set_smem(huge_draw_kernel<true, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_draw_kernel<true, MM><<<grid, kThreads, smem, st>>>(a, w, rows_post);
        })
    } else {
        WL_M_SWITCH({
            e = set_smem(huge_draw_kernel<false, MM>, smem);
            if (e != cudaSuccess) return e;
            huge_draw_kernel<false, MM><<<grid, kThreads, smem, st>>>(a, w, rows_post);
        })
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sparse count rows (K above what a shared-memory row holds): a long
// segment's counts live in an open-addressing hash in global memory, one
// 64-bit slot per entry ((topic + 1) << 32 | count), capacity a power of two
// above min(2 L, K) (so that probing ends), multiplicative hash, linear
// probing.  A token costs one atomic when its topic is present.  Word
// proposals then use positioning in storage order (reads z), so no
// post-acceptance row is needed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sparse_slot(uint32_t k, uint32_t mask) {
    return (k * 2654435761u) & mask;   // cap <= 2^31: the low bits of the product
}

__device__ __forceinline__ void sparse_add(unsigned long long* slots, uint32_t cap, uint32_t k, uint32_t n) {
    const uint32_t mask = cap - 1u;
    const unsigned long long key = (unsigned long long)(k + 1u) << 32;
    uint32_t h = sparse_slot(k, mask);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        // a stale empty read is settled by the CAS below
        const unsigned long long v = __ldcg(slots + h);
        if ((v >> 32) == (k + 1u)) {
            atomicAdd(slots + h, (unsigned long long)n);
            return;
        }
        if (v == 0ull) {
            const unsigned long long old = atomicCAS(slots + h, 0ull, key | n);
            if (old == 0ull) return;
            if ((old >> 32) == (k + 1u)) {
                atomicAdd(slots + h, (unsigned long long)n);
                return;
            }
        }
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int sparse_get(const unsigned long long* slots, uint32_t cap, uint32_t k) {
    const uint32_t mask = cap - 1u;
    uint32_t h = sparse_slot(k, mask);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const unsigned long long v = __ldg(slots + h);
        if ((v >> 32) == (k + 1u)) return (int)(uint32_t)v;
        if (v == 0ull) return 0;
        h = (h + 1) & mask;
    }
    return 0;
}

// sparse_get given the key's first slot v0 (already loaded).
__device__ __forceinline__ int sparse_resolve(const unsigned long long* slots, uint32_t cap, uint32_t k,
                                              unsigned long long v) {
    const uint32_t mask = cap - 1u;
    uint32_t h = sparse_slot(k, mask);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        if ((v >> 32) == (k + 1u)) return (int)(uint32_t)v;
        if (v == 0ull) return 0;
        h = (h + 1) & mask;
        v = __ldg(slots + h);
    }
    return 0;
}

template <bool kDoc>
__global__ void __launch_bounds__(kThreads) sparse_hist_kernel(PhaseArgs a, HugeWork w, SparseRows r) {
    __shared__ int s_r;
    const int K = a.K, tid = threadIdx.x;
    Checks chk;
    int pc0, pc1;
    while (next_range(w, &s_r, chk, &pc0, &pc1)) {
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 ch = get_piece(a, w, pc, chk);
            const int64_t base = r.off[ch.x];
            const uint32_t cap = (uint32_t)(r.off[ch.x + 1] - base);
            if (!chk(cap > 0 && (cap & (cap - 1)) == 0, 7)) continue;
            unsigned long long* slots = r.slots + base;
            for (int p = ch.z + tid; p < ch.z + ch.w; p += kThreads) {
                int t = kDoc ? a.perm[p] : p;
                if (!chk.tok((uint32_t)t < (uint32_t)a.N, 2)) continue;
                // lanes of a warp count tokens of the same segment: one
                // insert per distinct topic among them
                const uint32_t k = (uint32_t)chk.topic(a.z[t], K, 3);
                const unsigned m = __match_any_sync(__activemask(), k);
                if ((threadIdx.x & 31) == __ffs(m) - 1) sparse_add(slots, cap, k, (uint32_t)__popc(m));
            }
        }
    }
    chk.publish(a.fault, kSiteHugeHist);
}

template <bool kDoc, int M>
__global__ void __launch_bounds__(kThreads) sparse_accept_kernel(PhaseArgs a, HugeWork w, SparseRows r) {
    __shared__ int s_r;
    const int K = a.K, tid = threadIdx.x;
    const uint32_t phase = kDoc ? kPhaseDoc : kPhaseWord;
    Checks chk;
    int pc0, pc1;
    while (next_range(w, &s_r, chk, &pc0, &pc1)) {
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 ch = get_piece(a, w, pc, chk);
            const int64_t base = r.off[ch.x];
            const uint32_t cap = (uint32_t)(r.off[ch.x + 1] - base);
            if (!chk(cap > 0 && (cap & (cap - 1)) == 0, 7)) continue;
            const unsigned long long* slots = r.slots + base;
            const int Ls = a.seg_off[ch.y + 1] - a.seg_off[ch.y];
            const float Lf = __int2float_rn(Ls);
            const float LG = __fadd_rn(Lf, a.G);
            for (int p = ch.z + tid; p < ch.z + ch.w; p += kThreads) {
                const int t = kDoc ? a.perm[p] : p;
                if (!chk.tok((uint32_t)t < (uint32_t)a.N, 2)) continue;
                const int z0 = chk.topic(a.z[t], K, 3);
                // first slots and c_k of z and of every proposal loaded
                // first, the Philox blocks drawn while they are in flight,
                // then the probes resolved
                const uint32_t mask = cap - 1u;
                int tpv[M];
                unsigned long long v0[M + 1];
                float kv[M + 1];
                v0[0] = __ldg(slots + sparse_slot((uint32_t)z0, mask));
                kv[0] = __ldg(a.ckb + z0);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    tpv[i] = chk.topic(a.prop[(int64_t)t * M + i], K, 4);
                    v0[i + 1] = __ldg(slots + sparse_slot((uint32_t)tpv[i], mask));
                    kv[i + 1] = __ldg(a.ckb + tpv[i]);
                }
                uint4 rv[M];
#pragma unroll
                for (int i = 0; i < M; ++i) rv[i] = draw((uint32_t)t, a.iter, phase, (uint32_t)(i + 1), 0u, a.rk);
                int s = z0;
                int cs = sparse_resolve(slots, cap, (uint32_t)z0, v0[0]);
                float ks = kv[0];
                int pk[M];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const uint4 rr = rv[i];
                    const int tp = tpv[i];
                    if (tp != s) {
                        const int ct = sparse_resolve(slots, cap, (uint32_t)tp, v0[i + 1]);
                        const float kt = kv[i + 1];
                        if (accept(rr.x, cs, ct, a.g, ks, kt)) {
                            s = tp;
                            cs = ct;
                            ks = kt;
                        }
                    }
                    // words: the pick of Eq. 6 (a topic, or -(rank + 1)) over the
                    // consumed proposal, resolved by the draw pass
                    if (!kDoc)
                        pk[i] = coin(rr.y, Lf, LG) ? -(int)(dice(rr.z, (uint32_t)Ls) + 1) : (int)dice(rr.z, (uint32_t)K);
                }
                if (s != z0) {
                    a.z[t] = s;
                    if (a.ck_delta) {
                        atomicSub(&a.ck[z0], 1);
                        atomicAdd(&a.ck[s], 1);
                    }
                }
                if (!kDoc) {
#pragma unroll
                    for (int i = 0; i < M; ++i) a.prop[(int64_t)t * M + i] = pk[i];
                }
            }
        }
    }
    chk.publish(a.fault, kSiteHugeAccept);
}

cudaError_t launch_sparse_hist(bool doc, const PhaseArgs& a, const HugeWork& w, const SparseRows& r, int grid,
                               cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (w.npieces <= 0) return cudaSuccess;
    if (doc) sparse_hist_kernel<true><<<grid, kThreads, 0, st>>>(a, w, r);
    else sparse_hist_kernel<false><<<grid, kThreads, 0, st>>>(a, w, r);
    return cudaGetLastError();
}

cudaError_t launch_sparse_accept(bool doc, const PhaseArgs& a, const HugeWork& w, const SparseRows& r, int grid,
                                 cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (w.npieces <= 0) return cudaSuccess;
    if (doc) {
        WL_M_SWITCH({ sparse_accept_kernel<true, MM><<<grid, kThreads, 0, st>>>(a, w, r); })
    } else {
        WL_M_SWITCH({ sparse_accept_kernel<false, MM><<<grid, kThreads, 0, st>>>(a, w, r); })
    }
    return cudaGetLastError();
}

// Log-likelihood terms of sparse rows: sum over entries with a count of
// lnG(g + count) - lnG(g).
__global__ void sparse_loglik_kernel(const unsigned long long* __restrict__ slots, int64_t n, double g,
                                     double* out) {
    __shared__ double red[kWarps];
    const double lg = lgamma(g);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(uint32_t)slots[i];
        if (c > 0) acc += lgamma(g + (double)c) - lg;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kWarps; ++i) s += red[i];
        atomicAdd(out, s);
    }
}

cudaError_t launch_sparse_loglik(const unsigned long long* slots, int64_t n, double g, double* out,
                                 cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(4096, (n + kThreads - 1) / kThreads);
    sparse_loglik_kernel<<<grid, kThreads, 0, st>>>(slots, n, g, out);
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
