// The fold-in encoder (the learned document proposal; not in the paper):
// hashed bag of words -> H ReLU -> K softmax, BF16 weights, FP32
// accumulation, trained with soft cross-entropy against theta of Eq. 4 and
// Adam.  Readings (the oracle's L1-L5):
//   feature f(w) = ((w * 2654435761) mod 2^32) >> (32 - log2F), input
//   x_f = (# tokens with f(w) = f) / L_d;
//   h_pre = b1 + W1^T x, h = ReLU(h_pre), logits = b2 + W2^T bf16(h),
//   q = softmax(logits); loss = -(1/B) sum theta log q.
// Layer 1 is a gather: one block per document sums the W1 rows of its
// tokens.  Layer 2 and its two backward products are tensor-core GEMMs
// (wl_gemm.cu).  The layer-1 weight gradient is scattered with FP32 atomics
// into a dense buffer; Adam then updates every parameter and refreshes the
// BF16 copies (W2 in both the [K, H] and [H, K] layouts the GEMMs read).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "wl_block.cuh"
#include "wl_kernels.h"

namespace wl {

constexpr int kEncThreads = 128;

__device__ __forceinline__ uint16_t to_bf16(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float from_bf16(uint16_t b) {
    return __uint_as_float((uint32_t)b << 16);
}

__device__ __forceinline__ int enc_feature(int w, int log2F) {
    return (int)(((uint32_t)w * 2654435761u) >> (32 - log2F));
}

// Word id of every document-major token: the word whose word-major range
// holds perm[p].
__global__ void enc_docword_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ word_off,
                                   int64_t N, int64_t V, int32_t* __restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int t = perm[p];
        int64_t lo = 0, hi = V - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (word_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        out[p] = (int32_t)lo;
    }
}

// Layer 1 for a batch: row r of the batch is document docs[r] (r < nreal),
// else padding (h = 0).  One block per row: the document's tokens are dealt
// to the block's warps (token t to warp t mod 8), each warp reading whole
// W1 rows (a lane's 8 columns of each 256-column slice, one 16-byte load)
// with four rows in flight; the warps' partial sums are added in warp
// order.  The order of every sum depends only on the document, not on the
// batch it is in.
constexpr int kL1Threads = 256;
constexpr int kL1Warps = kL1Threads / 32;

__global__ void __launch_bounds__(kL1Threads) enc_l1_fwd_kernel(EncBatch b, const uint16_t* __restrict__ W1b,
                                                                const float* __restrict__ b1, int H, int log2F,
                                                                float* __restrict__ h_pre, uint16_t* __restrict__ hb,
                                                                uint16_t* __restrict__ hbT) {
    __shared__ float part[kL1Warps][256];
    const int r = blockIdx.x;
    const int B = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int d0 = 0, d1 = 0;
    if (r < b.nreal) {
        const int d = b.docs[r];
        d0 = b.doc_off[d];
        d1 = b.doc_off[d + 1];
    }
    const float invL = d1 > d0 ? 1.0f / (float)(d1 - d0) : 0.0f;
    for (int c0 = 0; c0 < H; c0 += 256) {
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
        // a slice may be half used (H a multiple of 128): lanes past H idle
        const bool cols = c0 + lane * 8 < H;
        const uint16_t* Wc = W1b + c0 + (cols ? lane * 8 : 0);
        int t = cols ? d0 + w : d1;
        for (; t + 3 * kL1Warps < d1; t += 4 * kL1Warps) {
            uint4 x[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int f = enc_feature(b.words[t + v * kL1Warps], log2F);
                x[v] = *reinterpret_cast<const uint4*>(Wc + (int64_t)f * H);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint32_t e[4] = {x[v].x, x[v].y, x[v].z, x[v].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc[2 * u] += __uint_as_float(e[u] << 16);
                    acc[2 * u + 1] += __uint_as_float(e[u] & 0xFFFF0000u);
                }
            }
        }
        for (; t < d1; t += kL1Warps) {
            const int f = enc_feature(b.words[t], log2F);
            const uint4 x = *reinterpret_cast<const uint4*>(Wc + (int64_t)f * H);
            const uint32_t e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[2 * u] += __uint_as_float(e[u] << 16);
                acc[2 * u + 1] += __uint_as_float(e[u] & 0xFFFF0000u);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) part[w][lane * 8 + u] = acc[u];
        __syncthreads();
        if (c0 + (int)threadIdx.x < H) {
            const int jj = threadIdx.x;   // one column of the slice per thread
            float sum = 0.0f;
#pragma unroll
            for (int v = 0; v < kL1Warps; ++v) sum += part[v][jj];
            const int j = c0 + jj;
            const float hp = r < b.nreal ? b1[j] + sum * invL : 0.0f;
            h_pre[(int64_t)r * H + j] = hp;
            const uint16_t hv = to_bf16(hp > 0.0f ? hp : 0.0f);
            hb[(int64_t)r * H + j] = hv;
            hbT[(int64_t)j * B + r] = hv;
        }
        __syncthreads();
    }
}

// Softmax of each row's first K logits; with targets, the soft cross-entropy
// and dlogits = (q - theta) / nreal (FP32 into gb2, BF16 into dl and dlT).
// Targets are given rows (tgt) or theta of Eq. 4 of the document's current
// assignments (z through perm).
__global__ void __launch_bounds__(kEncThreads) enc_softmax_kernel(
    EncBatch b, const float* __restrict__ logits, int K, int Kp, float* __restrict__ q_out,
    const float* __restrict__ tgt, const int32_t* __restrict__ z, const int32_t* __restrict__ perm,
    float alpha, float abar, uint16_t* __restrict__ dl, uint16_t* __restrict__ dlT,
    float* __restrict__ gb2, double* __restrict__ loss, int32_t* __restrict__ cnt_scratch) {
    __shared__ float red[kEncThreads / 32];
    __shared__ float s_val;
    const int r = blockIdx.x, B = gridDim.x, tid = threadIdx.x;
    const float* lg = logits + (int64_t)r * Kp;
    if (r >= b.nreal) {
        if (dl)
            for (int k = tid; k < Kp; k += kEncThreads) {
                dl[(int64_t)r * Kp + k] = 0;
                dlT[(int64_t)k * B + r] = 0;
            }
        return;
    }
    // max
    float m = -INFINITY;
    for (int k = tid; k < K; k += kEncThreads) m = fmaxf(m, lg[k]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        float v = red[0];
        for (int i = 1; i < kEncThreads / 32; ++i) v = fmaxf(v, red[i]);
        s_val = v;
    }
    __syncthreads();
    m = s_val;
    __syncthreads();
    float s = 0.f;
    for (int k = tid; k < K; k += kEncThreads) s += expf(lg[k] - m);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int i = 0; i < kEncThreads / 32; ++i) v += red[i];
        s_val = v;
    }
    __syncthreads();
    const float inv = 1.0f / s_val;
    if (q_out)
        for (int k = tid; k < K; k += kEncThreads) q_out[(int64_t)r * K + k] = expf(lg[k] - m) * inv;
    if (!dl) return;
    // targets: given rows, or theta of Eq. 4 from the document's assignments
    const int d = b.docs[r];
    float Lf = 0.f;
    int32_t* cnt = cnt_scratch + (int64_t)blockIdx.x * K;
    if (!tgt) {
        for (int k = tid; k < K; k += kEncThreads) cnt[k] = 0;
        __syncthreads();
        const int p0 = b.doc_off[d], p1 = b.doc_off[d + 1];
        for (int p = p0 + tid; p < p1; p += kEncThreads) {
            const uint32_t k = min((uint32_t)z[perm[p]], (uint32_t)(K - 1));
            atomicAdd(&cnt[k], 1);
        }
        __syncthreads();
        Lf = (float)(p1 - p0);
    }
    const float scale = 1.0f / (float)b.nreal;
    float ce = 0.f;
    for (int k = tid; k < Kp; k += kEncThreads) {
        float g = 0.f;
        if (k < K) {
            const float qk = expf(lg[k] - m) * inv;
            const float th = tgt ? tgt[(int64_t)d * K + k] : ((float)cnt[k] + alpha) / (Lf + abar);
            ce -= th * logf(fmaxf(qk, 1e-30f));
            g = (qk - th) * scale;
            atomicAdd(&gb2[k], g);
        }
        const uint16_t gv = to_bf16(g);
        dl[(int64_t)r * Kp + k] = gv;
        dlT[(int64_t)k * B + r] = gv;
    }
    for (int o = 16; o; o >>= 1) ce += __shfl_xor_sync(0xFFFFFFFFu, ce, o);
    if ((tid & 31) == 0) atomicAdd(loss, (double)ce * (double)scale);
}

// Layer-1 backward: dh_pre = dH * [h_pre > 0]; gb1 += dh_pre; each token adds
// dh_pre / L_d into its feature's gradient row.
__global__ void __launch_bounds__(kEncThreads) enc_l1_bwd_kernel(EncBatch b, const float* __restrict__ dH,
                                                                 const float* __restrict__ h_pre, int H, int log2F,
                                                                 float* __restrict__ gW1, float* __restrict__ gb1) {
    const int r = blockIdx.x;
    if (r >= b.nreal) return;
    const int d = b.docs[r];
    const int d0 = b.doc_off[d], d1 = b.doc_off[d + 1];
    const float invL = d1 > d0 ? 1.0f / (float)(d1 - d0) : 0.0f;
    for (int j = threadIdx.x; j < H; j += kEncThreads) {
        const float g = h_pre[(int64_t)r * H + j] > 0.0f ? dH[(int64_t)r * H + j] : 0.0f;
        if (g == 0.0f) continue;
        atomicAdd(&gb1[j], g);
        const float gs = g * invL;
        for (int t = d0; t < d1; ++t) atomicAdd(&gW1[(int64_t)enc_feature(b.words[t], log2F) * H + j], gs);
    }
}

// Adam (Kingma & Ba, Alg. 1) on n FP32 parameters; optional BF16 copy.
__global__ void enc_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int64_t n, float lr, float c1, float c2,
                                uint16_t* __restrict__ wb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        w[i] = wi;
        if (wb) wb[i] = to_bf16(wi);
    }
}

// BF16 copies of W2 ([Kp, H] master) in both GEMM layouts.
__global__ void enc_w2_copies_kernel(const float* __restrict__ W2t, int Kp, int H, uint16_t* __restrict__ W2tb,
                                     uint16_t* __restrict__ W2nb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)Kp * H;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / H), j = (int)(i % H);
        const uint16_t v = to_bf16(W2t[i]);
        W2tb[i] = v;
        W2nb[(int64_t)j * Kp + k] = v;
    }
}

__global__ void enc_to_bf16_kernel(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = to_bf16(x[i]);
}

// Walker alias tables of the proposal rows q[d, 0..K) (Vose's construction,
// in the oracle's order and FP32 operations): one block per document, its
// scaled row p, the two stacks (small from the front, large from the back)
// and the aliases in shared memory; out: {bits of the cut p, alias} per
// topic, so that a draw reads one 8-byte entry.  The block scales the row and fills the stacks in
// parallel -- a block scan gives each topic its place, in increasing topic
// order as the serial construction pushes them -- then one thread pairs
// them, a chain of dependent steps that only shared-memory latency keeps
// short.
constexpr int kAliasThreads = 256;

__global__ void __launch_bounds__(kAliasThreads) enc_alias_kernel(const float* __restrict__ q, int64_t Dn, int K,
                                                                  int2* __restrict__ atab) {
    extern __shared__ __align__(16) unsigned char sm[];
    float* p = reinterpret_cast<float*>(sm);
    int32_t* stk = reinterpret_cast<int32_t*>(p + K);
    int32_t* al = stk + K;
    __shared__ int warp_s[kAliasThreads / 32], warp_l[kAliasThreads / 32];
    __shared__ int s_ns, s_nl;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float Kf = (float)K;
    for (int64_t d = blockIdx.x; d < Dn; d += gridDim.x) {
        const float* qd = q + d * K;
        if (tid == 0) {
            s_ns = 0;
            s_nl = 0;
        }
        __syncthreads();
        for (int base = 0; base < K; base += kAliasThreads) {
            const int k = base + tid;
            float pk = 0.0f;
            if (k < K) {
                pk = __fmul_rn(qd[k], Kf);
                p[k] = pk;
            }
            const bool small = k < K && pk < 1.0f, large = k < K && !(pk < 1.0f);
            const unsigned bs = __ballot_sync(0xFFFFFFFFu, small), bl = __ballot_sync(0xFFFFFFFFu, large);
            if (lane == 0) {
                warp_s[w] = __popc(bs);
                warp_l[w] = __popc(bl);
            }
            __syncthreads();
            int os = s_ns, ol = s_nl;
            for (int i = 0; i < w; ++i) {
                os += warp_s[i];
                ol += warp_l[i];
            }
            const unsigned below = (1u << lane) - 1u;
            if (small) stk[os + __popc(bs & below)] = k;
            if (large) stk[K - 1 - (ol + __popc(bl & below))] = k;
            __syncthreads();
            if (tid == 0) {
                int ts = 0, tl = 0;
                for (int i = 0; i < kAliasThreads / 32; ++i) {
                    ts += warp_s[i];
                    tl += warp_l[i];
                }
                s_ns += ts;
                s_nl += tl;
            }
            __syncthreads();
        }
        if (tid == 0) {
            int ns = s_ns, nl = s_nl;
            while (ns > 0 && nl > 0) {
                const int l = stk[--ns];
                const int g = stk[K - nl--];
                al[l] = g;
                p[g] = __fsub_rn(__fadd_rn(p[g], p[l]), 1.0f);
                if (p[g] < 1.0f) stk[ns++] = g; else stk[K - 1 - nl++] = g;
            }
            while (nl > 0) {
                const int g = stk[K - nl--];
                p[g] = 1.0f;
                al[g] = g;
            }
            while (ns > 0) {
                const int l = stk[--ns];
                p[l] = 1.0f;
                al[l] = l;
            }
        }
        __syncthreads();
        int2* td = atab + d * K;
        for (int k = tid; k < K; k += kAliasThreads) td[k] = make_int2(__float_as_int(p[k]), al[k]);
        __syncthreads();
    }
}

static int grid_n(int64_t n) { return (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256)); }

cudaError_t launch_enc_docword(const int32_t* perm, const int32_t* word_off, int64_t N, int64_t V,
                               int32_t* out, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (N <= 0) return cudaSuccess;
    enc_docword_kernel<<<grid_n(N), 256, 0, st>>>(perm, word_off, N, V, out);
    return cudaGetLastError();
}

cudaError_t launch_enc_l1_fwd(const EncBatch& b, int B, const uint16_t* W1b, const float* b1, int H, int log2F,
                              float* h_pre, uint16_t* hb, uint16_t* hbT, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (H % 128 != 0) return cudaErrorInvalidValue;
    enc_l1_fwd_kernel<<<B, kL1Threads, 0, st>>>(b, W1b, b1, H, log2F, h_pre, hb, hbT);
    return cudaGetLastError();
}

cudaError_t launch_enc_softmax(const EncBatch& b, int B, const float* logits, int K, int Kp, float* q_out,
                               const float* tgt, const int32_t* z, const int32_t* perm, float alpha, float abar,
                               uint16_t* dl, uint16_t* dlT, float* gb2, double* loss, int32_t* cnt,
                               cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    enc_softmax_kernel<<<B, kEncThreads, 0, st>>>(b, logits, K, Kp, q_out, tgt, z, perm, alpha, abar, dl, dlT,
                                                  gb2, loss, cnt);
    return cudaGetLastError();
}

cudaError_t launch_enc_l1_bwd(const EncBatch& b, int B, const float* dH, const float* h_pre, int H, int log2F,
                              float* gW1, float* gb1, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    enc_l1_bwd_kernel<<<B, kEncThreads, 0, st>>>(b, dH, h_pre, H, log2F, gW1, gb1);
    return cudaGetLastError();
}

cudaError_t launch_enc_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, int step,
                            uint16_t* wb, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    const float c1 = (float)(1.0 - std::pow(0.9, step)), c2 = (float)(1.0 - std::pow(0.999, step));
    enc_adam_kernel<<<grid_n(n), 256, 0, st>>>(w, m, v, g, n, lr, c1, c2, wb);
    return cudaGetLastError();
}

cudaError_t launch_enc_w2_copies(const float* W2t, int Kp, int H, uint16_t* W2tb, uint16_t* W2nb,
                                 cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    enc_w2_copies_kernel<<<grid_n((int64_t)Kp * H), 256, 0, st>>>(W2t, Kp, H, W2tb, W2nb);
    return cudaGetLastError();
}

cudaError_t launch_enc_to_bf16(const float* x, int64_t n, uint16_t* y, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    enc_to_bf16_kernel<<<grid_n(n), 256, 0, st>>>(x, n, y);
    return cudaGetLastError();
}

cudaError_t launch_enc_alias(const float* q, int64_t Dn, int K, int2* atab, cudaStream_t st) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (Dn <= 0) return cudaSuccess;
    const int smem = K * 12;
    cudaError_t e = cudaFuncSetAttribute(enc_alias_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(Dn, 152 * 8);
    enc_alias_kernel<<<grid, kAliasThreads, smem, st>>>(q, Dn, K, atab);
    return cudaGetLastError();
}

}  // namespace wl
