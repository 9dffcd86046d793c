// Host-side launchers of the sampler kernels (internal to libwarplda.so).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wl_common.cuh"

namespace wl {

// Host-side fault injection, for tests of the error paths (nothing is run
// on the GPU to fail): with WARPLDA_FAIL_LAUNCH=k in the environment the
// k-th kernel launcher called from then on returns a launch error instead of
// launching, and with WARPLDA_FAIL_ALLOC=k the k-th device or pinned host
// allocation the library asks for fails as out of memory.  "From then on"
// counts from the first call that sees the variable with its current value;
// unset, empty or 0 disables it.  Every launcher starts with launch_gate().
cudaError_t launch_gate();
cudaError_t alloc_gate();

// On-chip batch tier (wl_batch.cu).  A batch is {first segment, end
// segment, table words, 0}; seg_region[s] is segment s's table offset in its
// batch; dense selects 16-bit dense tables (else hash tables).
int batch_smem_bytes(int K, int stage_ck, int region_words, int tpt, int word_phase, int dense);
int batch_blocks_per_sm(int K, int stage_ck, int region_words, int tpt, int word_phase, int M,
                        int dense);
cudaError_t launch_batch_phase(bool doc, bool dense, int tpt, const PhaseArgs& a,
                               const int4* batches, int nbatch, int* counter,
                               const int32_t* seg_region, int region_words, int kbits, int grid,
                               cudaStream_t st);

// Pipelined document batches (wl_docpipe.cu): desc[b] = {first document,
// documents | table words << 16, first token, tokens}.
int docpipe_smem_bytes(int K, int dense, int region_words, int tpt, int M);
int docpipe_blocks_per_sm(int K, int dense, int region_words, int tpt, int M);
cudaError_t launch_doc_pipe(bool dense, int tpt, const PhaseArgs& a, const int4* desc, int nbatch,
                            int* counter, const int32_t* seg_region, int region_words, int grid,
                            cudaStream_t st);

// Heavy words on a thread-block cluster (wl_cluster.cu): one cluster of C
// blocks per word of words[0..nwords), T tokens per block at most, smem
// bytes of dynamic shared memory per block.
int cluster_slice_capacity(int K, int M, int stage_ck, int smem_max);
int cluster_size_supported(int K, int M, int stage_ck, int C, int smem);
cudaError_t launch_cluster_word(const PhaseArgs& a, const int32_t* words, int nwords, int C, int T, int smem,
                                cudaStream_t st);

// Warp tier of the document phase (wl_docwarp.cu): docs = ids of documents
// with 1..32*tpl tokens.
int docwarp_table_words(int K, int tpl, int dense);
int docwarp_smem_bytes(int K, int stage_ck, int tpl, int dense);
int docwarp_blocks_per_sm(int K, int stage_ck, int tpl, int M, int dense);
cudaError_t launch_doc_warp(int tpl, bool dense, const PhaseArgs& a, const int32_t* docs, int ndocs,
                            int* counter, int grid, cudaStream_t st);

// Multi-pass tier for segments too long for one block (wl_huge.cu); rows
// are count rows of K ints, one per long segment.
int huge_guide_bits(int K);
int huge_smem_bytes(int K, int stage_ck, int pass, bool doc);
int huge_blocks_per_sm(int K, int stage_ck, int pass, bool doc, int M);
cudaError_t launch_huge_hist(bool doc, const PhaseArgs& a, const HugeWork& w, int32_t* rows,
                             int grid, cudaStream_t st);
cudaError_t launch_huge_accept(bool doc, const PhaseArgs& a, const HugeWork& w,
                               const int32_t* rows_pre, int grid, cudaStream_t st);
cudaError_t launch_huge_draw(bool doc, const PhaseArgs& a, const HugeWork& w,
                             const int32_t* rows_post, int grid, cudaStream_t st);
// Sparse count rows (large K): row r's hash occupies [off[r], off[r+1]) of
// slots, each (topic + 1) << 32 | count (0 = empty); capacities are powers
// of two.
struct SparseRows {
    const int64_t* off;
    unsigned long long* slots;
};
cudaError_t launch_sparse_hist(bool doc, const PhaseArgs& a, const HugeWork& w, const SparseRows& r, int grid,
                               cudaStream_t st);
cudaError_t launch_sparse_accept(bool doc, const PhaseArgs& a, const HugeWork& w, const SparseRows& r, int grid,
                                 cudaStream_t st);
cudaError_t launch_sparse_loglik(const unsigned long long* slots, int64_t n, double g, double* out,
                                 cudaStream_t st);

// Fold-in of new documents against a frozen model (wl_foldin.cu).
struct FoldArgs {
    int32_t* z;              // [Nn] topics, document order
    int32_t* prop;           // [Nn * M] proposals
    const int32_t* words;    // [Nn] word ids
    const int32_t* doc_off;  // [Dn + 1] token offsets
    const int32_t* order;    // [Dn] documents, longest first
    const int64_t* ids;      // [Dn] document ids (Philox stream)
    const int32_t* Cw;       // [V * K] frozen C_w
    const int32_t* Zs;       // [N] frozen topics of each word, ascending (word-major)
    const int32_t* word_off; // [V + 1] token offsets of the words
    const float* ckb;        // [K] frozen (float)c_k + beta_bar
    float* theta;            // [Dn * K] or null
    const float* q;          // learned proposal [Dn * K] or null (plain fold-in)
    const int2* atab;        // its alias tables [Dn * K]: {bits of the FP32 cut, alias}
    int32_t* counter;        // work counter (zero on entry)
    int32_t* fault;          // index-check record
    int Dn, K, M, V, sweeps, Lmax;
    float alpha, abar, beta, kbeta;
    RoundKeys rk;
};

// Fold-in against a frozen model (wl_foldin.cu): Cw = [V, K] trained counts,
// Zs = [N] each word's trained topics in ascending order.
cudaError_t launch_model_build(const int32_t* z, const int32_t* word_off, int64_t V, int K,
                               int32_t* Cw, int32_t* Zs, int32_t* fault, int grid, cudaStream_t st);
int foldin_table_words(int K, int Lmax);
int foldin_warps(int tab_words);
int foldin_blocks_per_sm(int K, int M, int tab_words);
cudaError_t launch_foldin(const FoldArgs& f, int tab_words, int grid, cudaStream_t st);

// Word-major fold-in (plain proposal; wl_foldin.cu): the requests' tokens
// regrouped by word, in pieces of up to 256 tokens of one word (staged: the
// word's frozen row is loaded once into the warp's shared memory) or of the
// words with few tokens (direct loads).
struct FoldWords {
    const int4* rec;          // [Nn] {token index, position in its document, stream id, word}
    const int4* pieces;       // {word or -1, first record, records, staged}
    const int32_t* npieces;   // number of pieces (device)
    int64_t Nn;
    int pstride;              // ints of shared memory per warp for a staged row (0: no staging)
    int per;                  // prefix-sum chunk per lane (odd)
};
constexpr int kFoldStageMaxK = 2048;   // staged rows above this K would cost too many resident warps
int64_t fold_pieces_bound(int64_t Nn, int stage_min);
cudaError_t launch_fold_words_build(const FoldArgs& f, int64_t Nn, int stage_min, int32_t* cnt, int32_t* hc,
                                    int32_t* lc, int32_t* pc, int32_t* cur, int32_t* scan_tmp, int4* rec,
                                    int4* pieces, int32_t* npieces, int grid, cudaStream_t st);
cudaError_t launch_fold_doc(const FoldArgs& f, int tab_words, int it, int mode, int32_t* counter, int grid,
                            cudaStream_t st);
cudaError_t launch_fold_word(const FoldArgs& f, const FoldWords& fw, int it, int grid, cudaStream_t st);
int fold_doc_blocks_per_sm(int K, int M, int tab_words);
int fold_word_blocks_per_sm(int M, const FoldWords& fw);

// Serving slots (continuous batching of fold-in requests): per slot
// info = {token offset in the pool, L, sweeps done, stream id}; the pool holds
// the active requests' word ids, z and proposals; theta (and, with the
// learned proposal, q and its alias table) per slot.
struct ServeSlots {
    int4* info;
    const int32_t* active;   // [nactive] slots advanced by this launch, one warp each
    int nactive, nslots;
    const int32_t* long_active;   // [nlong] slots advanced by a whole block each
    int nlong, long_blocks;       // ... by the launch's first long_blocks blocks
    int32_t* long_counter;        // their work counter (zero on entry)
    int64_t pool_tokens;
    int32_t* z;
    int32_t* prop;
    const int32_t* words;
    float* fin_theta;        // theta rows of the requests finishing in this launch
    int32_t* fin_slot;       // their slots
    int32_t* fin_count;      // rows written (zero on entry)
    const float* q;
    const int2* atab;        // {bits of the FP32 cut, alias} per topic
};
cudaError_t launch_serve_admit(const int32_t* staged, const int4* req, const int32_t* src, int n, int nslots,
                               int64_t pool_tokens, int32_t* pool_words, int4* info, cudaStream_t st);
cudaError_t launch_serve_rows(const void* src, const int32_t* slots, int n, int K, int nslots, void* dst,
                              cudaStream_t st);
cudaError_t launch_serve(const FoldArgs& f, const ServeSlots& sl, int tab_words, int grid, cudaStream_t st);

// Tensor-core BF16 GEMM (wl_gemm.cu): C[M,N] = A[M,K] B[N,K]^T (+ bias[N]),
// FP32 C; M, N multiples of 128, K a multiple of 64; *status set to 1 if a
// bounded wait ran out.
int gemm_smem_bytes();
// work: a float workspace of work_floats for split-K partial tiles (NULL:
// one CTA per tile); the result is the same for every split count up to
// FP32 rounding of the partial sums, and deterministic for a given one.
cudaError_t launch_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, const float* bias,
                             int M, int N, int K, int32_t* status, cudaStream_t st, float* work = nullptr,
                             int64_t work_floats = 0);
int gemm_splits(int M, int N, int K, int64_t work_floats);

// Fold-in encoder (wl_encoder.cu).  A batch is rows r = 0..B-1 of document
// docs[r] (r < nreal; the other rows are padding), tokens at
// [doc_off[d], doc_off[d+1]) of words (document-major word ids).
struct EncBatch {
    const int32_t* docs;
    const int32_t* doc_off;
    const int32_t* words;
    int nreal;
};
cudaError_t launch_enc_docword(const int32_t* perm, const int32_t* word_off, int64_t N, int64_t V,
                               int32_t* out, cudaStream_t st);
cudaError_t launch_enc_l1_fwd(const EncBatch& b, int B, const uint16_t* W1b, const float* b1, int H, int log2F,
                              float* h_pre, uint16_t* hb, uint16_t* hbT, cudaStream_t st);
cudaError_t launch_enc_softmax(const EncBatch& b, int B, const float* logits, int K, int Kp, float* q_out,
                               const float* tgt, const int32_t* z, const int32_t* perm, float alpha, float abar,
                               uint16_t* dl, uint16_t* dlT, float* gb2, double* loss, int32_t* cnt,
                               cudaStream_t st);
cudaError_t launch_enc_l1_bwd(const EncBatch& b, int B, const float* dH, const float* h_pre, int H, int log2F,
                              float* gW1, float* gb1, cudaStream_t st);
cudaError_t launch_enc_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, int step,
                            uint16_t* wb, cudaStream_t st);
cudaError_t launch_enc_w2_copies(const float* W2t, int Kp, int H, uint16_t* W2tb, uint16_t* W2nb,
                                 cudaStream_t st);
cudaError_t launch_enc_to_bf16(const float* x, int64_t n, uint16_t* y, cudaStream_t st);
cudaError_t launch_enc_alias(const float* q, int64_t Dn, int K, int2* atab,
                             cudaStream_t st);

// Initialisation, c_k, export, log-likelihood (wl_misc.cu).
cudaError_t launch_init_z(int32_t* z, int32_t* prop, int64_t N, int K, int M, uint64_t seed,
                          cudaStream_t st);
// c_k = histogram of z (z 16-byte aligned); grid from topic_hist_blocks_per_sm
int topic_hist_blocks_per_sm(int K);
cudaError_t launch_topic_hist(const int32_t* z, int64_t N, int32_t* ck, int K, int grid, cudaStream_t st);
cudaError_t launch_finalize_ck(const int32_t* ck, float* ckb, int K, float beta_bar,
                               int32_t* counters, int ncounters, cudaStream_t st);
cudaError_t launch_zero(int32_t* p, int64_t n, cudaStream_t st);
cudaError_t launch_gather_docmajor(const int32_t* z, const int32_t* perm, int64_t N, int32_t* out,
                                   cudaStream_t st);
cudaError_t launch_check_range(const int32_t* v, int64_t n, int K, int32_t* bad, cudaStream_t st);
cudaError_t launch_loglik_batches(bool doc, const int32_t* z, const int32_t* perm,
                                  const int32_t* seg_off, const int4* batches, int nbatch, int K,
                                  double g, int region_words, int64_t N, int64_t nseg_total,
                                  int32_t* fault, double* out, int grid, cudaStream_t st);
cudaError_t launch_loglik_rows(const int32_t* rows, int64_t nrows, int K, double g, double* out,
                               cudaStream_t st);
cudaError_t launch_loglik_lengths(const int32_t* seg_off, int64_t nseg, double abar, double* out,
                                  cudaStream_t st);
cudaError_t launch_loglik_topics(const int32_t* ck, int K, double bbar, double* out,
                                 cudaStream_t st);
int loglik_smem_bytes(int region_words);

// Sets the message warplda_last_error() returns on this thread; returns code.
int record_error(int code, const char* msg);

// Token store build (wl_build.cu).  launch_token_sort: stable LSD sort of
// (word id, doc-major position) pairs; pass 0 reads keys_a (word ids, values
// implicit), passes alternate between the (a) and (b) buffers, and
// *pos_sorted / *keys_sorted receive the buffers holding the positions and
// the word ids in word-major order ((b) after an odd number of passes,
// token_sort_passes(V)).  scratch holds
// token_sort_scratch(N) words.
// In-place exclusive scan of n int32 entries; tmp holds scan_scratch_words(n).
cudaError_t launch_scan_exclusive(int32_t* d, int64_t n, int32_t* tmp, cudaStream_t st);
int64_t scan_scratch_words(int64_t n);
cudaError_t launch_word_check(const int32_t* w, int64_t N, int32_t V, int32_t* bad, cudaStream_t st);
cudaError_t launch_word_starts(const int32_t* keys_sorted, int64_t N, int32_t V, int32_t* start, cudaStream_t st);
int token_sort_passes(int64_t V);
int64_t token_sort_scratch(int64_t N);
cudaError_t launch_token_sort(int32_t* keys_a, int32_t* vals_a, int32_t* keys_b, int32_t* vals_b, int64_t N,
                              int32_t V, int32_t* scratch, int32_t** pos_sorted, int32_t** keys_sorted,
                              cudaStream_t st);
cudaError_t launch_perm(const int32_t* pos_sorted, int64_t N, int32_t* perm, cudaStream_t st);
cudaError_t launch_batch_lists(const int4* batches, int nb, int max_tokens, const int32_t* doc_off,
                               const int32_t* perm, const int32_t* pos_sorted, int64_t N, int32_t* sperm,
                               uint32_t* sinfo, int32_t* bad, cudaStream_t st);

}  // namespace wl
