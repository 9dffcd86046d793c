// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05), the second
// layer of the fold-in encoder and its two backward products:
//   C[M, N] (FP32) = A[M, K] * B[N, K]^T (+ bias[N]),  A, B BF16 row-major.
// One CTA of four warps per 128 x 128 tile of C.  K advances in chunks of 64:
// all threads stage the A and B chunks in shared memory in the canonical
// K-major, no-swizzle layout (8 x 16-byte core matrices; core matrices along
// K 128 B apart, 8-row groups 1 KB apart), then one thread issues four
// tcgen05.mma (M=128, N=128, K=16 each) accumulating in tensor memory, and
// tcgen05.commit arrives on the chunk's mbarrier.  Two stages: the next
// chunk is staged while the tensor cores work on the current one.  The
// epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = rows of the tile).  Every mbarrier wait is bounded; a wait
// that runs out records an error and the CTA returns after freeing its TMEM.
// Split K: the encoder's products have few 128 x 128 tiles (16 for a batch
// of 256 rows against K = 1000 topics), so the K chunks are divided among
// `splits` CTAs per tile (blockIdx.z), each writing its partial tile to a
// workspace, and a second kernel adds the partials in split order (a fixed
// order: the result does not depend on scheduling) plus the bias.
#include <algorithm>

#include "wl_kernels.h"

namespace wl {

constexpr int kGemmTile = 128;           // M and N of a tile
constexpr int kGemmChunk = 64;           // K per staged chunk (128 bytes of BF16)
constexpr int kGemmThreads = 128;
constexpr int kStageBytes = kGemmTile * kGemmChunk * 2;   // 16 KB per operand per stage
constexpr uint32_t kGemmWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address,
// leading byte offset (next core matrix along K), stride byte offset (next
// 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// Bounded wait for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kGemmWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity));
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(
    const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, float* __restrict__ C,
    const float* __restrict__ bias, int M, int N, int K, int kc_per_split, int32_t* status) {
    extern __shared__ __align__(1024) uint8_t gsm[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGemmTile, n0 = blockIdx.x * kGemmTile;
    uint8_t* stageA[2] = {gsm, gsm + 2 * kStageBytes};
    uint8_t* stageB[2] = {gsm + kStageBytes, gsm + 3 * kStageBytes};

    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(kGemmTile));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = umma_idesc_bf16(kGemmTile, kGemmTile);

    // this CTA's K chunks; with splits, C is its slice of the workspace
    const int kbeg = blockIdx.z * kc_per_split;
    const int nk = min(K / kGemmChunk - kbeg, kc_per_split);
    C += (int64_t)blockIdx.z * M * N;
    A += (int64_t)kbeg * kGemmChunk;
    B += (int64_t)kbeg * kGemmChunk;
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc & 1;
        // the stage is free once the MMAs of chunk kc - 2 are done; the
        // outcome of the bounded wait is agreed on by the whole CTA
        bool w = true;
        if (kc >= 2) w = mbar_wait(smem_u32(&bars[st]), (uint32_t)(((kc - 2) >> 1) & 1));
        ok = __syncthreads_and(w) != 0;
        if (!ok) break;
        // stage chunk kc: 16-byte vector v = (row r, k-group g) goes to core
        // matrix (r / 8, g) at (r / 8) * 1024 + g * 128 + (r % 8) * 16
        const int k0 = kc * kGemmChunk;
#pragma unroll
        for (int it = 0; it < (kGemmTile * kGemmChunk / 8) / kGemmThreads; ++it) {
            const int v = it * kGemmThreads + tid;
            const int r = v >> 3, g = v & 7;
            const int off = (r >> 3) * 1024 + g * 128 + (r & 7) * 16;
            const uint4 a = *reinterpret_cast<const uint4*>(A + (int64_t)(m0 + r) * K + k0 + g * 8);
            const uint4 b = *reinterpret_cast<const uint4*>(B + (int64_t)(n0 + r) * K + k0 + g * 8);
            *reinterpret_cast<uint4*>(stageA[st] + off) = a;
            *reinterpret_cast<uint4*>(stageB[st] + off) = b;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(stageA[st]), b0 = smem_u32(stageB[st]);
#pragma unroll
            for (int s = 0; s < kGemmChunk / 16; ++s) {
                const uint64_t ad = umma_desc(a0 + s * 256, 128, 1024);
                const uint64_t bd = umma_desc(b0 + s * 256, 128, 1024);
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&bars[st])) : "memory");
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && nk > 0) {
        const bool w = mbar_wait(smem_u32(&bars[(nk - 1) & 1]), (uint32_t)(((nk - 1) >> 1) & 1));
        ok = __syncthreads_and(w) != 0;
    }
    if (!ok) {
        if (tid == 0) {
            s_abort = 1;
            if (status) atomicExch(status, 1);
        }
        // give MMAs in flight a second bounded wait before the memory goes
        if (nk > 0) mbar_wait(smem_u32(&bars[(nk - 1) & 1]), (uint32_t)(((nk - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_abort) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < kGemmTile; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float* out = C + (int64_t)row * N + n0 + c0;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
                float4 v;
                v.x = __uint_as_float(r[j]);
                v.y = __uint_as_float(r[j + 1]);
                v.z = __uint_as_float(r[j + 2]);
                v.w = __uint_as_float(r[j + 3]);
                if (bias) {
                    v.x += bias[n0 + c0 + j];
                    v.y += bias[n0 + c0 + j + 1];
                    v.z += bias[n0 + c0 + j + 2];
                    v.w += bias[n0 + c0 + j + 3];
                }
                *reinterpret_cast<float4*>(out + j) = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGemmTile));
    }
}

// C = sum over splits s of part[s] (in order s = 0, 1, ...) + bias.
__global__ void gemm_reduce_kernel(const float* __restrict__ part, int splits, int M, int N,
                                   const float* __restrict__ bias, float* __restrict__ C) {
    const int64_t n4 = (int64_t)M * N / 4;
    const int64_t plane = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = reinterpret_cast<const float4*>(part)[i];
        for (int s = 1; s < splits; ++s) {
            const float4 b = reinterpret_cast<const float4*>(part + s * plane)[i];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
        if (bias) {
            const int col = (int)((i * 4) % N);
            a.x += bias[col];
            a.y += bias[col + 1];
            a.z += bias[col + 2];
            a.w += bias[col + 3];
        }
        reinterpret_cast<float4*>(C)[i] = a;
    }
}

int gemm_smem_bytes() { return 4 * kStageBytes; }

// Splits of K for an M x N product: the smallest divisor of the chunk count
// (up to 8) that gives 64 CTAs, else the largest, within the workspace.
int gemm_splits(int M, int N, int K, int64_t work_floats) {
    const int tiles = (M / kGemmTile) * (N / kGemmTile), nk = K / kGemmChunk;
    int s = 1;
    for (int d = 2; d <= 8 && d <= nk && tiles * s < 64; ++d)
        if (nk % d == 0 && (int64_t)d * M * N <= work_floats) s = d;
    return s;
}

cudaError_t launch_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, const float* bias,
                             int M, int N, int K, int32_t* status, cudaStream_t st, float* work,
                             int64_t work_floats) {
    if (const cudaError_t g_ = launch_gate()) return g_;
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (M % kGemmTile || N % kGemmTile || K % kGemmChunk) return cudaErrorInvalidValue;
    const int smem = gemm_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int splits = work ? gemm_splits(M, N, K, work_floats) : 1;
    const int per = (K / kGemmChunk) / splits;
    if (splits == 1) {
        gemm_bf16_kernel<<<dim3(N / kGemmTile, M / kGemmTile, 1), kGemmThreads, smem, st>>>(A, B, C, bias, M, N, K,
                                                                                            per, status);
        return cudaGetLastError();
    }
    gemm_bf16_kernel<<<dim3(N / kGemmTile, M / kGemmTile, splits), kGemmThreads, smem, st>>>(A, B, work, nullptr, M,
                                                                                            N, K, per, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t n4 = (int64_t)M * N / 4;
    gemm_reduce_kernel<<<(unsigned)std::min<int64_t>((n4 + 255) / 256, 152 * 8), 256, 0, st>>>(work, splits, M, N,
                                                                                                bias, C);
    return cudaGetLastError();
}

}  // namespace wl
