/*
 * warplda.h -- C ABI of the GB300 WarpLDA sampler (libwarplda.so).
 *
 * The library implements the hot path of WarpLDA (Chen et al., arXiv
 * 1510.08628): the O(1) Metropolis-Hastings sweep over all tokens, one
 * document phase followed by one word phase (Sec. 4.4), sampling the MCEM
 * E-step target of Eq. 5 with the proposals of Eq. 6 and the acceptance rates
 * of Eq. 7, as in the appendix algorithm (Alg. 2).  All of it runs in CUDA
 * kernels for sm_103a on one GPU; there is no CPU fallback.
 *
 * Conventions
 *  - Every call returns WARPLDA_OK (0) or a negative WARPLDA_E* code; the
 *    message of the last failure on the calling thread is warplda_last_error().
 *  - Host pointers are plain host memory (pageable or pinned); "_dev" calls
 *    take device pointers of the context's device.  Inputs are copied; the
 *    caller keeps ownership of every buffer it passes.  Outputs are
 *    caller-allocated.
 *  - The context owns all device state.  Its work is issued on the stream
 *    given to warplda_init (NULL = the legacy default stream).  Calls that
 *    write host buffers synchronise that stream; warplda_sweep and the _dev
 *    calls do not.
 *  - Index types: document and word ids are int32; token counts int64 at the
 *    boundary.  N must be below 2^31.
 *  - Random numbers: Philox4x32-10 keyed by the 64-bit seed, counter
 *    (token's word-major index, iteration, phase << 8 | MH step, stream), so
 *    results do not depend on the launch configuration.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef WARPLDA_H
#define WARPLDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WARPLDA_OK 0
#define WARPLDA_EINVAL (-1)    /* bad argument or corpus */
#define WARPLDA_ENOMEM (-2)    /* device or host allocation failed */
#define WARPLDA_ECUDA (-3)     /* a CUDA call or kernel failed */
#define WARPLDA_ETIMEDOUT (-4) /* a bounded device wait gave up */
#define WARPLDA_ESTATE (-5)    /* call not valid in the context's state */
#define WARPLDA_EIO (-6)       /* checkpoint file could not be read or written */
#define WARPLDA_EBUSY (-7)     /* no serving slot or pool memory free now: retry later */
#define WARPLDA_EINTERNAL (-8) /* unexpected host-side failure (a library bug) */

#define WARPLDA_PHASE_DOC 1
#define WARPLDA_PHASE_WORD 2

typedef struct warplda_ctx warplda_ctx;
typedef struct warplda_server warplda_server;

/*
 * Launch tuning.  Any field left 0 takes its default.  Results are identical
 * for every valid tuning (the random stream is keyed by token, not by
 * schedule); the fields only move segments between kernel tiers.
 *   batch_max_tokens  documents / words with at most this many tokens are
 *                     processed on chip, several per thread block (<= 4095).
 *   huge_chunk        most tokens in one piece of a longer segment (the
 *                     multi-pass tier cuts such segments into ranges of
 *                     about equal size; 0: no further limit).
 *   region_budget     32-bit words of shared memory for the per-segment
 *                     count tables of one block batch.
 *   doc_warp_max      documents with at most this many tokens (capped at 512
 *                     with dense count tables, 256 with hash tables) are
 *                     sampled one warp per document; 0 (default) or -1: off.
 *   doc_batch_kernel  which kernel samples the document batches of up to
 *                     2045 tokens: 2 = the pipelined document kernel
 *                     (batches of up to 1021 tokens and 128 documents; the
 *                     next batch's tokens are gathered into shared memory
 *                     while the current one is sampled; region_budget
 *                     defaults to 4096 words for them); 1 = the block batch
 *                     kernel; 0 (default) = pipelined with hash count
 *                     tables and 2048 < K <= 16384, else block batch.
 *   cluster_max_tokens  words longer than a block batch and at most this
 *                     long are sampled on a thread-block cluster of 1 to 16
 *                     blocks (their tokens held in the cluster's shared
 *                     memory, the count rows reduced over distributed shared
 *                     memory); longer words take the multi-pass tier.  -1:
 *                     as long as the cluster's shared memory allows; 0
 *                     (default): no cluster tier (the multi-pass tier is
 *                     faster on the workloads measured).  K above 16384 has
 *                     no cluster tier.
 *   foldin_kernel     fold-in with the plain proposal: 0 (default) or 2 =
 *                     word-major phases (per sweep one launch for the
 *                     document phase, one warp per document, and one for
 *                     the word phase over the requests' tokens grouped by
 *                     word, a frequent word's frozen row read once per
 *                     piece of its tokens into shared memory); 1 = one warp
 *                     per document for all sweeps in one launch.  The
 *                     learned proposal and serving always take the
 *                     per-document kernel.
 * One field changes the sampler (a different, equally valid chain):
 *   word_positioning  the word proposal's p_A branch (Eq. 6): 0 (default) =
 *                     the j-th smallest post-acceptance topic of the word;
 *                     1 = the paper's random positioning (Sec. 4.3) over the
 *                     word's tokens in storage order -- the same law, no sort.
 */
typedef struct warplda_tuning {
    int32_t batch_max_tokens;
    int32_t huge_chunk;
    int32_t region_budget;
    int32_t doc_warp_max;
    int32_t word_positioning;
    int32_t doc_batch_kernel;
    int32_t cluster_max_tokens;
    int32_t foldin_kernel;
} warplda_tuning;

/*
 * warplda_init -- build the device state for a corpus (Sec. 2.1 problem
 * statement: W, K, alpha, beta; Sec. 4.3: M proposals per token).
 *   out        receives the new context.
 *   D, V, N    documents, vocabulary size, tokens (N == doc_ptr[D] < 2^31).
 *   doc_ptr    host int64[D+1], doc_ptr[0] = 0, non-decreasing: token CSR by
 *              document.  Empty documents are allowed.
 *   doc_word   host int32[N], word id in [0, V) of each token, in document
 *              order.  Empty words are allowed.
 *   K          topics, 1 <= K <= 1048575 (2^20 - 1).  Above 16384 the
 *              long documents and words of the multi-pass tier count into
 *              hash rows in device memory (capacity the power of two above
 *              min(2 L, K) per row) instead of dense K-wide rows, and word
 *              proposals use positioning in storage order (as tuning
 *              word_positioning = 1, which is forced).  Fold-in, the
 *              encoder, serving and warplda_word_counts keep a dense
 *              [V, K] model and return EINVAL above 16384.
 *   alpha      symmetric document Dirichlet parameter (> 0, FP32; the paper's
 *              alpha after its alpha' - 1 shift, Sec. 4.2).
 *   beta       symmetric word Dirichlet parameter (> 0, FP32).
 *   M          MH steps (proposals) per token per phase, 1 <= M <= 4.
 *   seed       Philox key.
 *   cuda_stream  cudaStream_t for all work of this context, or NULL.
 *   tuning     NULL for defaults.
 * Initialises z = Dice(K) per token and every proposal to z (Alg. 2), and
 * c_k = histogram of z.  Errors: EINVAL (bad sizes, CSR, word id, K, M,
 * alpha, beta), ENOMEM, ECUDA.  On error *out is NULL.
 */
int warplda_init(warplda_ctx** out, int64_t D, int64_t V, int64_t N, const int64_t* doc_ptr,
                 const int32_t* doc_word, int32_t K, float alpha, float beta, int32_t M,
                 uint64_t seed, void* cuda_stream, const warplda_tuning* tuning);

/*
 * warplda_sweep -- run n full sweeps (document phase then word phase each,
 * Sec. 4.4; counts refreshed only at phase boundaries, c_k reduced once per
 * phase).  Asynchronous on the context's stream; n >= 0.  Errors: EINVAL,
 * ESTATE (a single phase is pending, see warplda_phase), ECUDA (launch error).
 */
int warplda_sweep(warplda_ctx* ctx, int32_t n);

/*
 * warplda_phase -- run one phase of the next sweep: WARPLDA_PHASE_DOC, then
 * WARPLDA_PHASE_WORD (which completes the sweep).  For tests and tracing.
 * Errors: EINVAL (unknown phase), ESTATE (phases out of order), ECUDA.
 */
int warplda_phase(warplda_ctx* ctx, int32_t phase);

/*
 * warplda_counts -- copy results to host buffers (each may be NULL):
 *   z_docmajor  int32[N], topic of each token in the caller's doc_ptr order.
 *               Pinned (page-locked) host memory is written directly by the
 *               gather kernel; pageable memory goes through a device buffer
 *               of N int32 allocated on first use.
 *   ck          int32[K], global topic counts c_k (Sec. 2.1).
 * Synchronises the stream.  Errors: ECUDA.
 */
int warplda_counts(warplda_ctx* ctx, int32_t* z_docmajor, int32_t* ck);

/* As warplda_counts with device pointers; asynchronous on the stream. */
int warplda_counts_dev(warplda_ctx* ctx, int32_t* z_docmajor_dev, int32_t* ck_dev);

/*
 * warplda_get_state / warplda_set_state -- the complete sampler state, in
 * word-major token order (tokens sorted by word, then by their doc_ptr
 * position): z int32[N], proposals int32[N*M] (token-major, M per token),
 * c_k int32[K], and the number of completed sweeps.  get_state may be called
 * between the two phases of a sweep (the state after the document phase).
 * set_state recomputes c_k from z and checks that every value lies in [0, K);
 * on a bad value it re-initialises the context and returns EINVAL.  Host
 * buffers; both synchronise.  Errors: EINVAL, ESTATE (set_state while a
 * word phase is pending), ECUDA.
 */
int warplda_get_state(warplda_ctx* ctx, int32_t* z_wordmajor, int32_t* prop_wordmajor,
                      int32_t* ck, uint32_t* sweeps_done);
int warplda_set_state(warplda_ctx* ctx, const int32_t* z_wordmajor, const int32_t* prop_wordmajor,
                      uint32_t sweeps_done);

/* word_ptr int64[V+1] and perm int32[N] (doc_ptr position -> word-major
 * index) of the context's token order (Sec. 5.2 layout).  Host buffers. */
int warplda_token_order(warplda_ctx* ctx, int64_t* word_ptr, int32_t* perm);

/*
 * warplda_doc_batches -- the document batches of the on-chip tier and their
 * tokens in word-major order (the gather lists of the document phase,
 * Sec. 5.2), for tests and tracing.  Host buffers, each may be NULL:
 *   n_batches  receives the number of batches;
 *   batches  int32[4 * n_batches]: {first document, end document, table
 *            words, 0} per batch (both size classes, the 8- or 4-token class
 *            first);
 *   sperm    int32[N]: over the doc-major positions of each batch, that
 *            batch's word-major token indices in ascending order; 0 outside
 *            the batches;
 *   sinfo    uint32[N]: beside each sperm entry, (document slot in the batch
 *            << 16) | (doc-major position - the batch's first position).
 * Synchronises.  Errors: EINVAL, ECUDA.
 */
int warplda_doc_batches(warplda_ctx* ctx, int64_t* n_batches, int32_t* batches, int32_t* sperm,
                        uint32_t* sinfo);

/*
 * warplda_loglik -- joint log-likelihood log p(W, Z | alpha, beta) of Sec. 6.1
 * in FP64 (zero counts contribute zero; alpha_bar = K alpha and
 * beta_bar = V beta in double).  Synchronises.  Errors: ECUDA, ESTATE.
 */
int warplda_loglik(warplda_ctx* ctx, double* out);

/*
 * warplda_save / warplda_load -- checkpoint the state of warplda_get_state to
 * a file and restore it into a context built from the same corpus and
 * parameters.  Resume is bit-exact.  Errors: EIO, EINVAL (mismatch), ECUDA.
 */
int warplda_save(warplda_ctx* ctx, const char* path);
int warplda_load(warplda_ctx* ctx, const char* path);

/* Per-context statistics for benchmarks (host struct, filled on return). */
typedef struct warplda_info {
    int64_t D, V, N;
    int32_t K, M;
    int32_t launches_per_sweep;       /* kernels one warplda_sweep(1) launches */
    int32_t batch_max_tokens;
    int64_t doc_batches, word_batches;
    int64_t huge_docs, huge_doc_tokens;
    int64_t mega_words, mega_word_tokens;   /* words of the multi-pass tier */
    int64_t device_bytes;             /* device memory held by the context */
    int64_t pipe_doc_tokens;          /* tokens of the pipelined document batches */
    int64_t cluster_words, cluster_word_tokens;   /* words sampled on a thread-block cluster */
    int32_t reserved[2];
} warplda_info;
int warplda_get_info(warplda_ctx* ctx, warplda_info* out);

/*
 * Kernel timing for benchmarks.  While enabled, every kernel launch of the
 * context is bracketed by CUDA events recorded on the context's stream.
 * warplda_kernel_times synchronises and reports, for up to `cap` kernel
 * classes, their names, launch counts and total device milliseconds since the
 * last enable.  Returns the number of classes (>= 0) or an error code.
 */
int warplda_profile(warplda_ctx* ctx, int32_t enable);
int warplda_kernel_times(warplda_ctx* ctx, int32_t cap, const char** names, int64_t* launches,
                         double* total_ms);

/*
 * warplda_foldin -- theta (Eq. 4) of Dn new documents, sampled against the
 * model frozen at the call: the word-topic counts C_w and the topic counts
 * c_k of the context's current state (the paper trains only; fold-in is its
 * sampler with the word side frozen).  Each of `sweeps` sweeps is the
 * document phase of Sec. 4.4 (pi^word of Eq. 7 against the document's own
 * phase-start counts and the frozen c_k, then positioning over the
 * post-acceptance assignments) and the word phase with frozen counts (pi^doc
 * against the frozen C_w row of each token's word; word proposals of Eq. 6
 * drawn from that frozen row).  The new documents enter neither C_w nor c_k.
 * Random numbers are keyed by `seed`, the document id and the token's
 * position in its document, so a document's result does not depend on which
 * other documents are folded in with it.
 *   Dn, doc_ptr[Dn+1] (int64, host), doc_word[doc_ptr[Dn]] (int32, host):
 *               the documents as a CSR; word ids in [0, V).
 *   doc_ids     host int64[Dn] stream ids of the documents, or NULL for
 *               0..Dn-1.
 *   sweeps      fold-in sweeps (>= 0).
 *   proposal    WARPLDA_PROPOSAL_PLAIN, or WARPLDA_PROPOSAL_LEARNED: the
 *               document proposal is the encoder's softmax q_d (see
 *               warplda_encoder_init) drawn through a Walker alias table, and
 *               the word phase accepts it with the independence-sampler rate
 *               of Alg. 1, min{1, p(t) q_d(s) / (p(s) q_d(t))}, p the Eq. 5
 *               conditional with the document's phase-start counts, the frozen
 *               C_w and c_k; the chain keeps its target.
 *   theta_out   host float[Dn*K], theta_dk = (C_dk + alpha)/(L_d + K alpha)
 *               of the final assignments; or NULL.
 *   z_out       host int32[doc_ptr[Dn]], final topics in document order; or
 *               NULL.
 * The frozen model (C_w as V*K int32 and each word's topics in ascending
 * order, N int32, held by the context until warplda_destroy) is rebuilt when
 * the context has swept since the last fold-in.  The call's device scratch
 * (the documents' words, z, proposals, theta and the word-major records,
 * about 40 + 12 M bytes per token plus 4 K bytes per document) is kept by
 * the context for the next call and grown when a call needs more; it is
 * freed by warplda_destroy.  Documents may have at most 65535 tokens when
 * K <= 2048, 4095 above.  Synchronous.  Errors: EINVAL (CSR, word id,
 * length, proposal), ESTATE (a word phase is pending), ENOMEM, ECUDA.
 */
#define WARPLDA_PROPOSAL_PLAIN 0
#define WARPLDA_PROPOSAL_LEARNED 1
int warplda_foldin(warplda_ctx* ctx, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                   const int64_t* doc_ids, int32_t sweeps, uint64_t seed, int32_t proposal,
                   float* theta_out, int32_t* z_out);

/*
 * warplda_word_counts -- the word-topic counts C_w of the current state
 * (Sec. 2.1): host int32[V*K], row-major by word.  This is the frozen model
 * fold-in uses (built on the device, kept until the context sweeps again).
 * Errors: EINVAL, ESTATE (a word phase is pending), ENOMEM, ECUDA.
 */
int warplda_word_counts(warplda_ctx* ctx, int32_t* cw);

/*
 * The fold-in encoder: the learned document proposal of fold-in (the paper
 * has no counterpart).  A document's input is its hashed bag of words,
 * x_f = (# tokens whose word w has f(w) = ((w * 2654435761) mod 2^32) >>
 * (32 - log2_features)) / L_d; h = ReLU(b1 + W1^T x) (W1: [F, H]); q =
 * softmax(b2 + W2^T bf16(h)) (W2: [H, K]).  BF16 weights, FP32 accumulation;
 * the second layer and its backward products run on the tensor cores.
 *
 * warplda_encoder_init -- allocate and initialise (W1 ~ U(-1, 1), W2 Glorot
 *   uniform, biases 0; seeded).  log2_features in [6, 20]; hidden and
 *   batch_rows multiples of 128 up to 2048.  ESTATE if already initialised.
 * warplda_encoder_weights -- get (set = 0) or set (set = 1) the FP32 master
 *   weights: W1 host float[F*H] row-major, b1 [H], W2 [H*K] row-major, b2 [K].
 *   Setting leaves the optimiser state as it is.
 * warplda_encoder_grad -- one forward and backward pass on Dn (1..batch_rows)
 *   host documents (CSR, word ids in [0, V)) against host targets
 *   theta[Dn*K]; writes the mean soft cross-entropy and the gradients (same
 *   layouts as the weights); no update.
 * warplda_encoder_train -- `epochs` passes of Adam (lr; beta1 0.9, beta2
 *   0.999, eps 1e-8) over the context's own documents in seeded random
 *   batches of batch_rows, targets theta of Eq. 4 from the current
 *   assignments; epoch_loss[epochs] (or NULL) receives each epoch's mean loss.
 * warplda_encoder_proposal -- q_out[Dn*K] (host) for Dn host documents.
 * All synchronous.  Errors: EINVAL, ESTATE, ENOMEM, ETIMEDOUT (a bounded
 * tensor-core wait ran out), ECUDA.
 */
int warplda_encoder_init(warplda_ctx* ctx, int32_t log2_features, int32_t hidden, int32_t batch_rows,
                         uint64_t seed);
int warplda_encoder_weights(warplda_ctx* ctx, int32_t set, float* W1, float* b1, float* W2, float* b2);
int warplda_encoder_grad(warplda_ctx* ctx, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                         const float* theta, double* loss, float* gW1, float* gb1, float* gW2, float* gb2);
int warplda_encoder_train(warplda_ctx* ctx, int32_t epochs, float lr, uint64_t seed, double* epoch_loss);
int warplda_encoder_proposal(warplda_ctx* ctx, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                             float* q_out);

/*
 * Serving fold-in requests with continuous batching (the paper has no
 * counterpart).  The context's model is frozen when the server is created
 * (as for warplda_foldin); each request is one new document, folded in for
 * `sweeps` sweeps exactly as warplda_foldin would fold it in with doc id =
 * the request id and the same seed and proposal -- bit for bit, alone or in
 * any mix.  Per-request z, proposals and theta stay on the device.
 *
 * warplda_server_create -- `slots` requests in flight at most; a device
 *   token pool of pool_tokens (each admitted request holds L_d contiguous
 *   tokens until its result is polled); requests of at most max_doc_tokens
 *   (<= 65535 when K <= 2048, <= 4095 above).  Errors: EINVAL, ESTATE,
 *   ENOMEM, ECUDA.
 * warplda_server_submit -- admit request `id` (host word ids words[L], in
 *   [0, V); copied on the host, uploaded by the next step).  Returns OK, or
 *   EBUSY when no slot or no contiguous pool range is free: admission is by
 *   memory, the caller retries after a poll has retired finished requests.
 * warplda_server_step -- upload the requests admitted since the last step,
 *   then launch one sweep for every admitted, unfinished request (new ones
 *   are initialised first; a request's last sweep writes its theta);
 *   asynchronous.  With the learned proposal the new requests' encoder
 *   forward and alias tables run on a second stream beside the sweep of the
 *   requests already running (the step ends when both have); with fewer
 *   than 8 sweeps per request their first sweep follows there, in the same
 *   step, else they join the sweeps from the next step on (results are the
 *   same either way).  *active_out (or NULL) = requests advanced or being
 *   admitted.  Requests submitted while a step runs join the next step.
 *   The previous step's results must have been polled (else ESTATE).
 * warplda_server_poll -- wait at most timeout_ms for the last step (else
 *   ETIMEDOUT), then hand over the requests it finished: ids[n] and
 *   theta[n*K] (Eq. 4), *n_out = n <= max_results (else EINVAL; max_results
 *   = slots always suffices); their slots and pool memory are freed.
 * Not thread-safe: one thread drives a server.
 * warplda_server_destroy -- wait for the stream and free the server.
 */
int warplda_server_create(warplda_ctx* ctx, int32_t slots, int64_t pool_tokens, int32_t max_doc_tokens,
                          int32_t sweeps, uint64_t seed, int32_t proposal, warplda_server** out);
int warplda_server_submit(warplda_server* srv, int64_t id, int32_t L, const int32_t* words);
int warplda_server_step(warplda_server* srv, int32_t* active_out);
int warplda_server_poll(warplda_server* srv, int32_t max_results, int64_t* ids, float* theta, int32_t* n_out,
                        int32_t timeout_ms);
void warplda_server_destroy(warplda_server* srv);

/*
 * warplda_gemm_bf16 -- the tensor-core (tcgen05) GEMM of the fold-in
 * encoder's second layer and its backward products, exposed for testing:
 *   C[M, N] = A[M, K] * B[N, K]^T (+ bias[N]).
 *   A_dev, B_dev  device BF16, row-major (K contiguous), 16-byte aligned.
 *   C_dev         device float32 [M, N], row-major.
 *   bias_dev      device float32 [N] or NULL.
 *   M, N multiples of 128, K a multiple of 64.
 * Synchronous on cuda_stream (NULL: the default stream).  Errors: EINVAL
 * (shapes, alignment), ETIMEDOUT (a bounded tensor-core wait ran out), ECUDA.
 * The paper has no counterpart.
 */
int warplda_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, const float* bias_dev,
                      int32_t M, int32_t N, int32_t K, void* cuda_stream);

/*
 * warplda_sync -- wait for the work queued on the context's stream and report
 * the kernels' index checks.  Every sampler kernel validates the indices it
 * takes from stored state (topics, proposals, token pointers, work lists)
 * before it uses them; a failed check skips the access and is recorded.
 * Returns OK, or ECUDA with the kernel site and value of the first failed
 * check since the last report (the record is then cleared).  warplda_counts,
 * warplda_get_state and warplda_loglik report the record the same way.
 * Setting WARPLDA_SYNC_CHECK=1 in the environment before warplda_init makes
 * the context read the record after every launch (debugging; slow).
 * Setting WARPLDA_TRACE_INIT=1 makes warplda_init wait for its stream at each
 * stage boundary and print every stage's wall time to stderr (diagnostics:
 * the waits serialise stages that init otherwise overlaps).
 */
int warplda_sync(warplda_ctx* ctx);

void warplda_destroy(warplda_ctx* ctx);
const char* warplda_last_error(void);

/*
 * warplda_loglik_noalloc -- the joint log-likelihood of warplda_loglik
 * (same definition and FP64 arithmetic) for callers that cannot allocate
 * device memory: code inside a host framework that owns every device
 * allocation (a caching allocator or a fixed arena that forbids raw
 * cudaMalloc), or a serving process with a fixed device-memory budget.  It
 * takes no context, because creating one allocates.  The paper has no
 * counterpart; this is an interface convenience.
 *   D, V, N     documents, vocabulary size, tokens (N < 2^31).
 *   K, alpha, beta   as for warplda_init; K must be at most 16384, else
 *               EINVAL (the scratch below holds that many topic counts).
 *   doc_ptr_dev     device int64[D+1], token offsets of the documents.
 *   z_docmajor_dev  device int32[N], topics in document order.
 *   word_ptr_dev    device int64[V+1], token offsets of the words.
 *   z_wordmajor_dev device int32[N], the same topics grouped by word.
 *               A value outside [0, K) is not counted and makes the
 *               result NaN.  N must equal doc_ptr[D] and word_ptr[V] (the
 *               tokens counted on either side); if it does not, the result
 *               is NaN.  The offsets must otherwise be valid: monotone and
 *               within the z arrays (not checked).
 *   out_dev     device double, receives the log-likelihood.
 *   cuda_stream cudaStream_t or NULL; the call is asynchronous on it.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch is a static device array of about 66 KB that every GPU loading
 * this library holds until the process exits; every call looks up that
 * array's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing).  All calls share the array and each call clears
 * it first, so calls whose kernels overlap on a GPU (different streams,
 * threads) race and must be serialised by the caller.  Cost: every document
 * and word clears and scans K shared-memory counters, O((D + V) K) work
 * besides reading the N topics twice.  Errors: EINVAL (sizes, K above
 * 16384, null pointer), ECUDA.
 */
int warplda_loglik_noalloc(int64_t D, int64_t V, int64_t N, int32_t K, float alpha, float beta,
                           const int64_t* doc_ptr_dev, const int32_t* z_docmajor_dev,
                           const int64_t* word_ptr_dev, const int32_t* z_wordmajor_dev,
                           double* out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* WARPLDA_H */
