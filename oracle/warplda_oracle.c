/*
 * Plain CPU WarpLDA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The CUDA sampler shares no code with it: this
 * file has its own Philox, its own counting, its own proposal draws.
 *
 * What it computes is the WarpLDA sampler of Chen et al. (arXiv 1510.08628):
 * the MCEM E-step target (Eq. 5), sampled with the Metropolis-Hastings chain of
 * Alg. 1 using the two proposals of Eq. 6 and the acceptance rates of Eq. 7,
 * reordered into a document phase and a word phase (Sec. 4.4) and run as in the
 * appendix algorithm (Alg. 2).  It is written to be checked by eye, not to be
 * fast: counts are recomputed from z, words are sorted with qsort, and every
 * floating-point operation is a single FP32 round-to-nearest operation written
 * out in the order of the arithmetic contract below (compile with
 * -ffp-contract=off, no fast-math).
 *
 * Readings taken where the paper is silent or garbled (each repeated where it
 * is used):
 *  R1  the source state of each MH step is the current z (Alg. 1, Eq. 7), not
 *      the previous proposal as the appendix listing literally writes;
 *  R2  the appendix's "C_s + beta_bar V" is C_s + beta_bar (Eq. 7);
 *  R3  beta_w in Eq. 5 is the symmetric beta;
 *  R4  one sweep = document phase, then word phase; initialisation sets every
 *      proposal to z so the first accept step is a no-op;
 *  R5  delayed update (Sec. 4.2): every count used inside a phase is the
 *      histogram of z at the start of that phase, token itself included; c_k
 *      is recomputed once per phase;
 *  R6  proposals are drawn from the post-acceptance z_d / z_w of the segment;
 *  R7  the word proposal's p_A part (prop. to C_wk) is drawn as the j-th
 *      smallest post-acceptance topic of the word, j uniform in [0, L_w): the
 *      same law as the alias table of Alg. 2, independent of storage order;
 *  R8  the word mixture weight is L_w / (L_w + K beta) (Sec. 4.3 footnote, by
 *      symmetry with L_d / (L_d + alpha_bar));
 *  R9  accept iff u < ratio, u = (r >> 8) 2^-24, written division-free as
 *      u * den < num; a proposal equal to the current state is a no-op;
 *  R10 Dice(n) (Alg. 2) = (r * n) >> 32 on a 32-bit Philox4x32-10 output.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11, Sec. 5), key = (seed_lo, seed_hi),
 * counter = (t, iteration, phase << 8 | i, stream), where t is the token's
 * word-major index, phase is 0 (init), 1 (document) or 2 (word), i is the MH
 * step (1..M, 0 at init) and stream is 0 during training.  One block per
 * (token, phase, step): r0 -> accept, r1 -> mixture coin, r2 -> index/topic.
 *
 * Fold-in of new documents against the frozen model (orc_foldin) carries
 * its own readings F1-F4 at its definition.
 *
 * Parity pins (tests/test_oracle_*.py): Philox against Triton's Philox
 * routine; count invariants after each phase; single-token chi-square of the
 * chained MH kernel against the exact Eq. 5 conditional; K = 1 and one-word
 * closed forms; log-likelihood against brute-force log sums; whole-sampler
 * log-likelihood against a plain collapsed Gibbs sampler (Eq. 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Planted mistakes, used only by tests/test_oracle_mutations.py to show that
 * the pins catch them.  ORC_MUTATION = 0 is the oracle. */
#ifndef ORC_MUTATION
#define ORC_MUTATION 0
#endif

enum { ORC_PHASE_INIT = 0, ORC_PHASE_DOC = 1, ORC_PHASE_WORD = 2 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 from its published definition (SC'11, Sec. 5).             */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key schedule (Weyl) */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
#if ORC_MUTATION == 9
    const int rounds = 9;
#else
    const int rounds = 10;
#endif
    for (int r = 0; r < rounds; ++r) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One block of the sampler's stream. */
static void draw_block(uint64_t seed, uint32_t t, uint32_t iter, uint32_t phase,
                       uint32_t step, uint32_t stream, uint32_t r[4])
{
    uint32_t ctr[4] = { t, iter, (phase << 8) | step, stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, r);
}

/* u in [0,1) on 24 bits: exact in FP32 (R9). */
static float u24(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

/* Dice(n) of Alg. 2 by multiply-shift (R10). */
static uint32_t dice(uint32_t r, uint32_t n)
{
#if ORC_MUTATION == 5
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32) % (n > 1 ? n - 1 : 1);
#else
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
#endif
}

/* ------------------------------------------------------------------------ */
/* The two O(1) building blocks of a phase.                                  */
/* ------------------------------------------------------------------------ */

/*
 * One MH accept/reject step (Alg. 1) from current state s to proposal t.
 * Both Eq. 7 rates have the form
 *     min{1, (C_t + g)(c_k[s] + beta_bar) / ((C_s + g)(c_k[t] + beta_bar))}
 * with (C, g) = (C_d, alpha) for pi^word in the document phase and
 * (C, g) = (C_w, beta) for pi^doc in the word phase (R2, R3).  Accept iff
 * u * den < num (R9).  Returns the new state.
 */
int orc_accept(uint32_t r0, int s, int t, int C_s, int C_t, int ck_s, int ck_t,
               float g, float beta_bar)
{
    if (t == s) return s;
    float num, den;
#if ORC_MUTATION == 1
    num = ((float)C_t) * ((float)ck_s + beta_bar);               /* dropped +g */
    den = ((float)C_s + g) * ((float)ck_t + beta_bar);
#elif ORC_MUTATION == 2
    num = ((float)C_t + g) * ((float)ck_t + beta_bar);           /* s/t swapped */
    den = ((float)C_s + g) * ((float)ck_s + beta_bar);
#else
    num = ((float)C_t + g) * ((float)ck_s + beta_bar);
    den = ((float)C_s + g) * ((float)ck_t + beta_bar);
#endif
    return (u24(r0) * den < num) ? t : s;
}

/*
 * Draw from the mixture  q(k) prop. to C_k + g  (Sec. 2.2 "mixture of
 * multinomials", Eq. 6): with probability L / (L + G) take the p_A branch
 * (prop. to C_k), else a uniform topic (p_B, symmetric g).  G = K g:
 * alpha_bar for documents, K beta for words (R8).
 * The p_A branch is given as `pick_a(idx)` = topic at rank idx in [0, L):
 *   documents: the idx-th post-acceptance z of the document, in the
 *              document's own (input CSR) order -- random positioning, Sec. 4.3;
 *   words:     the idx-th smallest post-acceptance z of the word (R7).
 * Both sides pass the array that realises pick_a.
 */
int orc_draw_mixture(uint32_t r1, uint32_t r2, const int* pick_a, int L, int K, float G)
{
    float Lf = (float)L;
#if ORC_MUTATION == 3
    if (u24(r1) * (Lf + G + G) < Lf)                    /* wrong mixture weight */
#else
    if (u24(r1) * (Lf + G) < Lf)
#endif
        return pick_a[dice(r2, (uint32_t)L)];
    return (int)dice(r2, (uint32_t)K);
}

/* ------------------------------------------------------------------------ */
/* Token order.                                                              */
/* ------------------------------------------------------------------------ */

/*
 * Word-major order of the tokens (Sec. 5.2: the data are stored by column,
 * each column sorted by row id).  Tokens are given by document CSR
 * (doc_ptr[D+1], doc_word[N]); the word-major index of the token at doc-major
 * position p is perm[p], word w occupies [word_ptr[w], word_ptr[w+1]), and
 * within a word tokens keep doc-major order (stable counting sort by word).
 * Returns 0, or -1 on a word id outside [0, V).
 */
int orc_word_major(int64_t D, int64_t V, const int64_t* doc_ptr, const int32_t* doc_word,
                   int64_t* word_ptr, int32_t* perm)
{
    int64_t N = doc_ptr[D];
    for (int64_t w = 0; w <= V; ++w) word_ptr[w] = 0;
    for (int64_t p = 0; p < N; ++p) {
        int32_t w = doc_word[p];
        if (w < 0 || (int64_t)w >= V) return -1;
        word_ptr[w + 1] += 1;
    }
    for (int64_t w = 0; w < V; ++w) word_ptr[w + 1] += word_ptr[w];
    int64_t* fill = (int64_t*)malloc((size_t)(V > 0 ? V : 1) * sizeof(int64_t));
    for (int64_t w = 0; w < V; ++w) fill[w] = word_ptr[w];
    for (int64_t p = 0; p < N; ++p) perm[p] = (int32_t)(fill[doc_word[p]]++);
    free(fill);
    return 0;
}

/* Initialisation (Alg. 2): z = Dice(K) per token; every proposal := z (R4). */
void orc_init(int64_t N, int K, int M, uint64_t seed, int32_t* z, int32_t* prop)
{
    for (int64_t t = 0; t < N; ++t) {
        uint32_t r[4];
        draw_block(seed, (uint32_t)t, 0, ORC_PHASE_INIT, 0, 0, r);
        z[t] = (int32_t)dice(r[0], (uint32_t)K);
        for (int i = 0; i < M; ++i) prop[t * M + i] = z[t];
    }
}

/* c_k = histogram of z (Sec. 2.1; recomputed once per phase, R5). */
void orc_topic_counts(int64_t N, int K, const int32_t* z, int32_t* ck)
{
    for (int k = 0; k < K; ++k) ck[k] = 0;
    for (int64_t t = 0; t < N; ++t) ck[z[t]] += 1;
}

/* ------------------------------------------------------------------------ */
/* Document phase (Sec. 4.4; Alg. 2, document loop).                          */
/* ------------------------------------------------------------------------ */

/*
 * One document: c_d from z_d; accept the pending word proposals with
 * pi^word (Eq. 7) against c_d and the phase-start c_k; then draw M new
 * document proposals per token from q^doc (Eq. 6) by random positioning over
 * the post-acceptance z_d.  Tokens are visited in input CSR order; z and
 * proposals live in word-major arrays reached through perm.
 * cd: scratch of K ints, znew: scratch of L_d ints.
 */
static void doc_one(int64_t d, const int64_t* doc_ptr, const int32_t* perm, int K, int M,
                    float alpha, float alpha_bar, float beta_bar, uint64_t seed, uint32_t iter,
                    int32_t* z, int32_t* prop, const int32_t* ck, int32_t* cd, int32_t* znew)
{
    int64_t b = doc_ptr[d];
    int L = (int)(doc_ptr[d + 1] - b);
    if (L == 0) return;
    for (int k = 0; k < K; ++k) cd[k] = 0;
    for (int j = 0; j < L; ++j) cd[z[perm[b + j]]] += 1;
#if ORC_MUTATION == 7
    cd[z[perm[b + L - 1]]] -= 1;                      /* last token left out */
#endif
    for (int j = 0; j < L; ++j) {
        int32_t t = perm[b + j];
        int s = z[t];
        for (int i = 1; i <= M; ++i) {
            uint32_t r[4];
            draw_block(seed, (uint32_t)t, iter, ORC_PHASE_DOC, (uint32_t)i, 0, r);
            int tp = prop[(int64_t)t * M + (i - 1)];
#if ORC_MUTATION == 8
            s = orc_accept(r[0], z[t], tp, cd[z[t]], cd[tp], ck[z[t]], ck[tp], alpha, beta_bar);
#else
            s = orc_accept(r[0], s, tp, cd[s], cd[tp], ck[s], ck[tp], alpha, beta_bar);
#endif
        }
        znew[j] = s;
    }
    for (int j = 0; j < L; ++j) {
        int32_t t = perm[b + j];
        for (int i = 1; i <= M; ++i) {
            uint32_t r[4];
            draw_block(seed, (uint32_t)t, iter, ORC_PHASE_DOC, (uint32_t)i, 0, r);
            prop[(int64_t)t * M + (i - 1)] = orc_draw_mixture(r[1], r[2], znew, L, K, alpha_bar);
        }
    }
    for (int j = 0; j < L; ++j) z[perm[b + j]] = znew[j];
}

/* Documents [d0, d1); ck is the phase-start topic count vector (R5). */
void orc_doc_phase(int64_t d0, int64_t d1, const int64_t* doc_ptr, const int32_t* perm,
                   int K, int M, float alpha, float alpha_bar, float beta_bar,
                   uint64_t seed, uint32_t iter, int32_t* z, int32_t* prop, const int32_t* ck)
{
    int64_t maxL = 0;
    for (int64_t d = d0; d < d1; ++d)
        if (doc_ptr[d + 1] - doc_ptr[d] > maxL) maxL = doc_ptr[d + 1] - doc_ptr[d];
#pragma omp parallel
    {
        int32_t* cd = (int32_t*)malloc((size_t)K * sizeof(int32_t));
        int32_t* znew = (int32_t*)malloc((size_t)(maxL > 0 ? maxL : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 64)
        for (int64_t d = d0; d < d1; ++d)
            doc_one(d, doc_ptr, perm, K, M, alpha, alpha_bar, beta_bar, seed, iter, z, prop, ck,
                    cd, znew);
        free(cd);
        free(znew);
    }
}

/* ------------------------------------------------------------------------ */
/* Word phase (Sec. 4.4; Alg. 2, word loop).                                  */
/* ------------------------------------------------------------------------ */

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/*
 * One word: c_w from z_w; accept the pending document proposals with pi^doc
 * (Eq. 7) against c_w and the phase-start c_k; then draw M new word proposals
 * per token from q^word (Eq. 6): with probability L_w / (L_w + K beta) the
 * j-th smallest post-acceptance topic of the word (R7, R8), else uniform.
 * cw: scratch of K ints, znew: scratch of L_w ints.
 */
static void word_one(int64_t w, const int64_t* word_ptr, int K, int M, float beta,
                     float K_beta, float beta_bar, uint64_t seed, uint32_t iter,
                     int32_t* z, int32_t* prop, const int32_t* ck, int32_t* cw, int32_t* znew,
                     int storage)
{
    int64_t b = word_ptr[w];
    int L = (int)(word_ptr[w + 1] - b);
    if (L == 0) return;
    for (int k = 0; k < K; ++k) cw[k] = 0;
    for (int j = 0; j < L; ++j) cw[z[b + j]] += 1;
    for (int j = 0; j < L; ++j) {
        int64_t t = b + j;
        int s = z[t];
        for (int i = 1; i <= M; ++i) {
            uint32_t r[4];
            draw_block(seed, (uint32_t)t, iter, ORC_PHASE_WORD, (uint32_t)i, 0, r);
            int tp = prop[t * M + (i - 1)];
            s = orc_accept(r[0], s, tp, cw[s], cw[tp], ck[s], ck[tp], beta, beta_bar);
        }
        znew[j] = s;
    }
#if ORC_MUTATION == 4
    for (int j = 0; j < L; ++j) znew[j] = z[b + j];   /* pre-acceptance z_w */
#endif
    for (int j = 0; j < L; ++j) z[b + j] = znew[j];
    if (!storage) qsort(znew, (size_t)L, sizeof(int), cmp_int);
    for (int j = 0; j < L; ++j) {
        int64_t t = b + j;
        for (int i = 1; i <= M; ++i) {
            uint32_t r[4];
            draw_block(seed, (uint32_t)t, iter, ORC_PHASE_WORD, (uint32_t)i, 0, r);
            prop[t * M + (i - 1)] = orc_draw_mixture(r[1], r[2], znew, L, K, K_beta);
        }
    }
}

/* Words [w0, w1); ck is the phase-start topic count vector (R5). */
/*
 * Words [w0, w1) with the word proposal rule `storage`: 0 = R7 (the j-th
 * smallest post-acceptance topic); 1 = the paper's literal random
 * positioning (Sec. 4.3) applied to words, the post-acceptance topic of the
 * word's j-th token in storage (word-major) order -- the same law (R7').
 */
void orc_word_phase_rule(int64_t w0, int64_t w1, const int64_t* word_ptr, int K, int M, float beta,
                         float K_beta, float beta_bar, uint64_t seed, uint32_t iter, int32_t* z,
                         int32_t* prop, const int32_t* ck, int storage)
{
    int64_t maxL = 0;
    for (int64_t w = w0; w < w1; ++w)
        if (word_ptr[w + 1] - word_ptr[w] > maxL) maxL = word_ptr[w + 1] - word_ptr[w];
#pragma omp parallel
    {
        int32_t* cw = (int32_t*)malloc((size_t)K * sizeof(int32_t));
        int32_t* znew = (int32_t*)malloc((size_t)(maxL > 0 ? maxL : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t w = w0; w < w1; ++w)
            word_one(w, word_ptr, K, M, beta, K_beta, beta_bar, seed, iter, z, prop, ck, cw, znew,
                     storage);
        free(cw);
        free(znew);
    }
}

void orc_word_phase(int64_t w0, int64_t w1, const int64_t* word_ptr, int K, int M, float beta,
                    float K_beta, float beta_bar, uint64_t seed, uint32_t iter, int32_t* z,
                    int32_t* prop, const int32_t* ck)
{
    orc_word_phase_rule(w0, w1, word_ptr, K, M, beta, K_beta, beta_bar, seed, iter, z, prop, ck, 0);
}

/*
 * n full sweeps starting at iteration iter0 + 1: document phase, c_k, word
 * phase, c_k (R4, R5).  ck must hold the histogram of z on entry and holds it
 * on exit.  alpha_bar = (float)K * alpha, beta_bar = (float)V * beta and
 * K_beta = (float)K * beta are single FP32 products formed by the caller.
 */
void orc_sweeps_rule(int64_t D, int64_t V, const int64_t* doc_ptr, const int32_t* perm,
                     const int64_t* word_ptr, int K, int M, float alpha, float beta,
                     float alpha_bar, float beta_bar, float K_beta, uint64_t seed, uint32_t iter0,
                     int n, int32_t* z, int32_t* prop, int32_t* ck, int storage)
{
    int64_t N = doc_ptr[D];
    for (int s = 1; s <= n; ++s) {
        uint32_t it = iter0 + (uint32_t)s;
        orc_doc_phase(0, D, doc_ptr, perm, K, M, alpha, alpha_bar, beta_bar, seed, it, z, prop, ck);
        orc_topic_counts(N, K, z, ck);
        orc_word_phase_rule(0, V, word_ptr, K, M, beta, K_beta, beta_bar, seed, it, z, prop, ck,
                            storage);
        orc_topic_counts(N, K, z, ck);
    }
}

void orc_sweeps(int64_t D, int64_t V, const int64_t* doc_ptr, const int32_t* perm,
                const int64_t* word_ptr, int K, int M, float alpha, float beta,
                float alpha_bar, float beta_bar, float K_beta, uint64_t seed, uint32_t iter0,
                int n, int32_t* z, int32_t* prop, int32_t* ck)
{
    orc_sweeps_rule(D, V, doc_ptr, perm, word_ptr, K, M, alpha, beta, alpha_bar, beta_bar, K_beta,
                    seed, iter0, n, z, prop, ck, 0);
}

/* ------------------------------------------------------------------------ */
/* Joint log-likelihood (Sec. 6.1), FP64.                                     */
/* ------------------------------------------------------------------------ */

/*
 * log p(W, Z | alpha, beta) = sum_d [lnG(abar) - lnG(abar + L_d)
 *                                    + sum_k (lnG(alpha + C_dk) - lnG(alpha))]
 *                           + sum_k [lnG(bbar) - lnG(bbar + C_k)
 *                                    + sum_w (lnG(beta + C_kw) - lnG(beta))]
 * with symmetric alpha, abar = K alpha, bbar = V beta, all in double from the
 * float hyper-parameters.  Zero counts contribute exactly zero and are skipped.
 */
double orc_loglik(int64_t D, int64_t V, const int64_t* doc_ptr, const int32_t* perm,
                  const int64_t* word_ptr, int K, float alpha_f, float beta_f, const int32_t* z)
{
    double alpha = (double)alpha_f, beta = (double)beta_f;
    double abar = (double)K * alpha, bbar = (double)V * beta;
    double la = lgamma(alpha), lb = lgamma(beta);
    double ll_doc = 0.0, ll_word = 0.0, ll_topic = 0.0;
    int32_t* c = (int32_t*)calloc((size_t)K, sizeof(int32_t));
    int32_t* ck = (int32_t*)calloc((size_t)K, sizeof(int32_t));
    for (int64_t d = 0; d < D; ++d) {
        int64_t b = doc_ptr[d], L = doc_ptr[d + 1] - b;
        ll_doc += lgamma(abar) - lgamma(abar + (double)L);
        for (int64_t j = 0; j < L; ++j) c[z[perm[b + j]]] += 1;
        for (int64_t j = 0; j < L; ++j) {
            int k = z[perm[b + j]];
            if (c[k] > 0) {
                ll_doc += lgamma(alpha + (double)c[k]) - la;
                c[k] = 0;
            }
        }
    }
    for (int64_t w = 0; w < V; ++w) {
        int64_t b = word_ptr[w], L = word_ptr[w + 1] - b;
        for (int64_t j = 0; j < L; ++j) { c[z[b + j]] += 1; ck[z[b + j]] += 1; }
        for (int64_t j = 0; j < L; ++j) {
            int k = z[b + j];
            if (c[k] > 0) {
                ll_word += lgamma(beta + (double)c[k]) - lb;
                c[k] = 0;
            }
        }
    }
    for (int k = 0; k < K; ++k) ll_topic += lgamma(bbar) - lgamma(bbar + (double)ck[k]);
    free(c);
    free(ck);
    return ll_doc + ll_word + ll_topic;
}

/* ------------------------------------------------------------------------ */
/* Test helpers.                                                             */
/* ------------------------------------------------------------------------ */

/*
 * Single-token chains with frozen counts (pin of the MH kernel law).
 * n_chains independent chains, chain c uses token id t = t0 + c.  Each sweep
 * runs the token's document phase (accept the pending word proposals with
 * pi^word against Cd, then draw M doc proposals by positioning over the
 * frozen zd[Ld]) and its word phase (accept the doc proposals with pi^doc
 * against Cw, then draw M word proposals from the frozen sorted zw_sorted[Lw]),
 * through the same orc_accept / orc_draw_mixture used by the phases.  The
 * stationary law is Eq. 5: q(k) prop. to (Cd_k + alpha)(Cw_k + beta)/(ck_k + bbar).
 * s0[c] is the chain's start (proposals start equal to it, R4); after
 * n_sweeps the final state is written to s_out[c].
 */
void orc_token_chains(int K, int M, const int32_t* Cd, const int32_t* Cw, const int32_t* ck,
                      const int32_t* zd, int Ld, const int32_t* zw_sorted, int Lw, float alpha,
                      float beta, float alpha_bar, float beta_bar, float K_beta, uint64_t seed,
                      uint32_t t0, int64_t n_chains, int n_sweeps, const int32_t* s0,
                      int32_t* s_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_chains; ++c) {
        uint32_t t = t0 + (uint32_t)c;
        int s = s0[c];
        int p[16];
        for (int i = 0; i < M; ++i) p[i] = s;
        for (int it = 1; it <= n_sweeps; ++it) {
            uint32_t r[4];
            for (int i = 1; i <= M; ++i) {
                draw_block(seed, t, (uint32_t)it, ORC_PHASE_DOC, (uint32_t)i, 0, r);
                s = orc_accept(r[0], s, p[i - 1], Cd[s], Cd[p[i - 1]], ck[s], ck[p[i - 1]],
                               alpha, beta_bar);
            }
            for (int i = 1; i <= M; ++i) {
                draw_block(seed, t, (uint32_t)it, ORC_PHASE_DOC, (uint32_t)i, 0, r);
                p[i - 1] = orc_draw_mixture(r[1], r[2], zd, Ld, K, alpha_bar);
            }
            for (int i = 1; i <= M; ++i) {
                draw_block(seed, t, (uint32_t)it, ORC_PHASE_WORD, (uint32_t)i, 0, r);
                s = orc_accept(r[0], s, p[i - 1], Cw[s], Cw[p[i - 1]], ck[s], ck[p[i - 1]],
                               beta, beta_bar);
            }
            for (int i = 1; i <= M; ++i) {
                draw_block(seed, t, (uint32_t)it, ORC_PHASE_WORD, (uint32_t)i, 0, r);
                p[i - 1] = orc_draw_mixture(r[1], r[2], zw_sorted, Lw, K, K_beta);
            }
        }
        s_out[c] = s;
    }
}

/*
 * Plain collapsed Gibbs sampler of Eq. 1 (exact O(K) conditional with the
 * token's own assignment removed), used only as the statistical yardstick of
 * the whole-sampler log-likelihood test (Sec. 6.3 compares MCEM with CGS).
 * Visits tokens in document order; its own Philox stream (phase 3).  Counts
 * are built from z on entry.  Double precision.
 */
void orc_cgs_sweeps(int64_t D, int64_t V, const int64_t* doc_ptr, const int32_t* doc_word,
                    const int32_t* perm, int K, float alpha_f, float beta_f, uint64_t seed,
                    uint32_t iter0, int n, int32_t* z)
{
    double alpha = alpha_f, beta = beta_f, bbar = (double)V * beta;
    int64_t N = doc_ptr[D];
    int32_t* cwk = (int32_t*)calloc((size_t)(V * K), sizeof(int32_t));
    int32_t* ck = (int32_t*)calloc((size_t)K, sizeof(int32_t));
    int32_t* cd = (int32_t*)calloc((size_t)K, sizeof(int32_t));
    double* pk = (double*)malloc((size_t)K * sizeof(double));
    for (int64_t p = 0; p < N; ++p) {
        int k = z[perm[p]];
        cwk[(int64_t)doc_word[p] * K + k] += 1;
        ck[k] += 1;
    }
    for (int s = 1; s <= n; ++s) {
        for (int64_t d = 0; d < D; ++d) {
            int64_t b = doc_ptr[d], L = doc_ptr[d + 1] - b;
            for (int k = 0; k < K; ++k) cd[k] = 0;
            for (int64_t j = 0; j < L; ++j) cd[z[perm[b + j]]] += 1;
            for (int64_t j = 0; j < L; ++j) {
                int32_t t = perm[b + j];
                int w = doc_word[b + j], k0 = z[t];
                cd[k0] -= 1; cwk[(int64_t)w * K + k0] -= 1; ck[k0] -= 1;
                double tot = 0.0;
                for (int k = 0; k < K; ++k) {
                    tot += (cd[k] + alpha) * (cwk[(int64_t)w * K + k] + beta) / (ck[k] + bbar);
                    pk[k] = tot;
                }
                uint32_t r[4];
                draw_block(seed, (uint32_t)t, iter0 + (uint32_t)s, 3, 0, 0, r);
                double u = ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6))
                           * (1.0 / 9007199254740992.0) * tot;
                int k1 = 0;
                while (k1 < K - 1 && pk[k1] <= u) ++k1;
                z[t] = k1;
                cd[k1] += 1; cwk[(int64_t)w * K + k1] += 1; ck[k1] += 1;
            }
        }
    }
    free(cwk); free(ck); free(cd); free(pk);
}

/* ------------------------------------------------------------------------ */
/* Fold-in of new documents against a frozen model.                          */
/* ------------------------------------------------------------------------ */

/*
 * The paper trains only; fold-in (inference of theta for unseen documents) is
 * the sampler above with the word side frozen.  Readings:
 *  F1  the frozen model is the trained word-topic counts C_w (dense [V*K])
 *      and c_k; the new documents' tokens enter neither;
 *  F2  a sweep is the document phase (pi^word against the document's own
 *      phase-start c_d and the frozen c_k, then positioning over the
 *      post-acceptance z_d) and the word phase (pi^doc against the frozen
 *      C_w row of the token's word and the frozen c_k, then a word proposal
 *      from the frozen row: with probability L_w / (L_w + K beta), L_w the
 *      frozen row's total, the j-th smallest topic of the frozen word, j
 *      uniform in [0, L_w) (the inverse CDF of the row, R7); else uniform);
 *  F3  random numbers: counter = (position of the token in its document,
 *      iteration, phase << 8 | i, document id), key = the fold-in seed,
 *      phases 3 (init), 4 (document), 5 (word): a document's result depends
 *      only on its words, its id, the seed and the model -- not on the other
 *      documents folded in with it;
 *  F4  output theta_dk = (C_dk + alpha) / (L_d + alpha_bar) from the final z
 *      (Eq. 4), FP32: one add each, then one IEEE division.
 */
enum { ORC_PHASE_FINIT = 3, ORC_PHASE_FDOC = 4, ORC_PHASE_FWORD = 5 };

/* The j-th smallest topic of a frozen word (inverse CDF of its count row,
 * ascending k), by a plain scan: smallest k with C_0 + ... + C_k > j. */
static int frozen_rank_topic(const int32_t* row, int K, int64_t j)
{
    int64_t cum = 0;
    for (int k = 0; k < K; ++k) {
        cum += row[k];
#if ORC_MUTATION == 10
        if (cum >= j) return k;                         /* rank off by one */
#else
        if (cum > j) return k;
#endif
    }
    return K - 1;
}

/* Word proposal from a frozen row (F2): r1 -> coin, r2 -> rank or topic. */
int orc_frozen_word_draw(uint32_t r1, uint32_t r2, const int32_t* row, int K, float K_beta)
{
    int64_t Lw = 0;
    for (int k = 0; k < K; ++k) Lw += row[k];
    float Lf = (float)Lw;
    if (Lw > 0 && u24(r1) * (Lf + K_beta) < Lf)
        return frozen_rank_topic(row, K, (int64_t)dice(r2, (uint32_t)Lw));
    return (int)dice(r2, (uint32_t)K);
}

/*
 * Fold-in of Dn documents (doc CSR doc_ptr[Dn+1], doc_word[Nn]) with ids
 * doc_id[Dn] against the frozen C_w (cw[V*K]) and c_k (ck[K]), `sweeps`
 * sweeps.  Writes the final z in document order (z_out[Nn]) and, if theta_out
 * is not NULL, theta (theta_out[Dn*K], F4).  Word ids must be in [0, V).
 */
void orc_foldin(int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                const int64_t* doc_id, int K, int M, float alpha, float alpha_bar, float beta,
                float K_beta, float beta_bar, const int32_t* cw, const int32_t* ck,
                uint64_t seed, int sweeps, int32_t* z_out, float* theta_out)
{
    int64_t maxL = 1;
    for (int64_t d = 0; d < Dn; ++d)
        if (doc_ptr[d + 1] - doc_ptr[d] > maxL) maxL = doc_ptr[d + 1] - doc_ptr[d];
#pragma omp parallel
    {
        int32_t* cd = (int32_t*)malloc((size_t)K * sizeof(int32_t));
        int32_t* znew = (int32_t*)malloc((size_t)maxL * sizeof(int32_t));
        int32_t* prop = (int32_t*)malloc((size_t)maxL * (size_t)M * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t d = 0; d < Dn; ++d) {
            int64_t b = doc_ptr[d];
            int L = (int)(doc_ptr[d + 1] - b);
            uint32_t id = (uint32_t)doc_id[d];
            int32_t* z = z_out + b;
            uint32_t r[4];
            for (int j = 0; j < L; ++j) {                       /* init (R4) */
                draw_block(seed, (uint32_t)j, 0, ORC_PHASE_FINIT, 0, id, r);
                z[j] = (int32_t)dice(r[0], (uint32_t)K);
                for (int i = 0; i < M; ++i) prop[j * M + i] = z[j];
            }
            for (int it = 1; it <= sweeps; ++it) {
                /* document phase */
                for (int k = 0; k < K; ++k) cd[k] = 0;
                for (int j = 0; j < L; ++j) cd[z[j]] += 1;
                for (int j = 0; j < L; ++j) {
                    int s = z[j];
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FDOC, (uint32_t)i, id, r);
                        int tp = prop[j * M + (i - 1)];
                        s = orc_accept(r[0], s, tp, cd[s], cd[tp], ck[s], ck[tp], alpha, beta_bar);
                    }
                    znew[j] = s;
                }
                for (int j = 0; j < L; ++j)
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FDOC, (uint32_t)i, id, r);
                        prop[j * M + (i - 1)] = orc_draw_mixture(r[1], r[2], znew, L, K, alpha_bar);
                    }
                for (int j = 0; j < L; ++j) z[j] = znew[j];
                /* word phase (frozen C_w, F2) */
                for (int j = 0; j < L; ++j) {
#if ORC_MUTATION == 11
                    const int32_t* row = cw + (int64_t)doc_word[b + (j + 1) % L] * K;   /* neighbour's word */
#else
                    const int32_t* row = cw + (int64_t)doc_word[b + j] * K;
#endif
                    int s = z[j];
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FWORD, (uint32_t)i, id, r);
                        int tp = prop[j * M + (i - 1)];
                        s = orc_accept(r[0], s, tp, row[s], row[tp], ck[s], ck[tp], beta, beta_bar);
                    }
                    z[j] = s;
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FWORD, (uint32_t)i, id, r);
                        prop[j * M + (i - 1)] = orc_frozen_word_draw(r[1], r[2], row, K, K_beta);
                    }
                }
            }
            if (theta_out) {                                    /* F4 */
                for (int k = 0; k < K; ++k) cd[k] = 0;
                for (int j = 0; j < L; ++j) cd[z[j]] += 1;
#if ORC_MUTATION == 12
                float den = (float)L + alpha;                   /* alpha for alpha_bar */
#else
                float den = (float)L + alpha_bar;
#endif
                for (int k = 0; k < K; ++k)
                    theta_out[d * K + k] = ((float)cd[k] + alpha) / den;
            }
        }
        free(cd);
        free(znew);
        free(prop);
    }
}

/*
 * Walker's alias table for a discrete distribution q[K] (Vose's construction,
 * "A linear algorithm for generating random numbers with a given
 * distribution", IEEE TSE 1991): scaled weights p_k = K q_k; columns below 1
 * and at or above 1 go on two stacks in index order; repeatedly the top small
 * column l keeps probability p_l and aliases the top large column g, whose
 * weight becomes (p_g + p_l) - 1.  FP32, every operation one RN operation in
 * this order.  Readings L6: the learned proposal is this table.
 */
void orc_alias_build(const float* q, int K, float* prob, int32_t* alias)
{
    float* p = (float*)malloc((size_t)K * sizeof(float));
    int32_t* small = (int32_t*)malloc((size_t)K * sizeof(int32_t));
    int32_t* large = (int32_t*)malloc((size_t)K * sizeof(int32_t));
    int ns = 0, nl = 0;
    for (int k = 0; k < K; ++k) {
        p[k] = q[k] * (float)K;
        if (p[k] < 1.0f) small[ns++] = k; else large[nl++] = k;
    }
    while (ns > 0 && nl > 0) {
        int l = small[--ns], g = large[--nl];
        prob[l] = p[l];
        alias[l] = g;
        p[g] = (p[g] + p[l]) - 1.0f;
        if (p[g] < 1.0f) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { int g = large[--nl]; prob[g] = 1.0f; alias[g] = g; }
    while (ns > 0) { int l = small[--ns]; prob[l] = 1.0f; alias[l] = l; }
    free(p); free(small); free(large);
}

/* One draw from an alias table: column Dice(K) by r2, kept iff u(r1) < prob. */
int orc_alias_draw(uint32_t r1, uint32_t r2, const float* prob, const int32_t* alias, int K)
{
    int k = (int)dice(r2, (uint32_t)K);
    return u24(r1) < prob[k] ? k : alias[k];
}

/*
 * Fold-in with a learned document proposal (the scope's next row 2; not in
 * the paper).  Readings L6-L7:
 *  L6  q[d*K + k] is the document's proposal distribution (the encoder's
 *      softmax, FP32), drawn through the alias table above;
 *  L7  a sweep is the document phase of orc_foldin with its draw replaced by
 *      M independent draws from the alias table (r1, r2 of the same Philox
 *      blocks), and the word phase of orc_foldin with pi^doc replaced by the
 *      independence-sampler rate of Alg. 1,
 *        min{1, p(t) q(s) / (p(s) q(t))},  p(k) = (C_dk + alpha)(C_wk + beta) / (c_k + beta_bar)
 *      (the Eq. 5 conditional with the word phase's phase-start c_d, the
 *      frozen C_w and c_k), accepted iff u * den < num with
 *        num = (((C_dt + alpha) * (C_wt + beta)) * ckb_s) * q_s,
 *        den = (((C_ds + alpha) * (C_ws + beta)) * ckb_t) * q_t,
 *      ckb_k = c_k + beta_bar, every + and * one FP32 RN operation.
 * Everything else (init, streams, word proposals, theta) is orc_foldin's.
 */
void orc_foldin_learned(int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                        const int64_t* doc_id, int K, int M, float alpha, float beta,
                        float alpha_bar, float K_beta, float beta_bar, const int32_t* cw,
                        const int32_t* ck, const float* q, uint64_t seed, int sweeps,
                        int32_t* z_out, float* theta_out)
{
    int64_t maxL = 1;
    for (int64_t d = 0; d < Dn; ++d)
        if (doc_ptr[d + 1] - doc_ptr[d] > maxL) maxL = doc_ptr[d + 1] - doc_ptr[d];
#pragma omp parallel
    {
        int32_t* cd = (int32_t*)malloc((size_t)K * sizeof(int32_t));
        int32_t* znew = (int32_t*)malloc((size_t)maxL * sizeof(int32_t));
        int32_t* prop = (int32_t*)malloc((size_t)maxL * (size_t)M * sizeof(int32_t));
        float* prob = (float*)malloc((size_t)K * sizeof(float));
        int32_t* alias = (int32_t*)malloc((size_t)K * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t d = 0; d < Dn; ++d) {
            int64_t b = doc_ptr[d];
            int L = (int)(doc_ptr[d + 1] - b);
            uint32_t id = (uint32_t)doc_id[d];
            const float* qd = q + d * K;
            int32_t* z = z_out + b;
            uint32_t r[4];
            orc_alias_build(qd, K, prob, alias);
            for (int j = 0; j < L; ++j) {
                draw_block(seed, (uint32_t)j, 0, ORC_PHASE_FINIT, 0, id, r);
                z[j] = (int32_t)dice(r[0], (uint32_t)K);
                for (int i = 0; i < M; ++i) prop[j * M + i] = z[j];
            }
            for (int it = 1; it <= sweeps; ++it) {
                /* document phase: pi^word, then learned proposals */
                for (int k = 0; k < K; ++k) cd[k] = 0;
                for (int j = 0; j < L; ++j) cd[z[j]] += 1;
                for (int j = 0; j < L; ++j) {
                    int s = z[j];
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FDOC, (uint32_t)i, id, r);
                        int tp = prop[j * M + (i - 1)];
                        s = orc_accept(r[0], s, tp, cd[s], cd[tp], ck[s], ck[tp], alpha, beta_bar);
                    }
                    znew[j] = s;
                }
                for (int j = 0; j < L; ++j) {
                    z[j] = znew[j];
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FDOC, (uint32_t)i, id, r);
                        prop[j * M + (i - 1)] = orc_alias_draw(r[1], r[2], prob, alias, K);
                    }
                }
                /* word phase: independence-sampler rate (L7), frozen word proposals */
                for (int k = 0; k < K; ++k) cd[k] = 0;
                for (int j = 0; j < L; ++j) cd[z[j]] += 1;
                for (int j = 0; j < L; ++j) {
                    const int32_t* row = cw + (int64_t)doc_word[b + j] * K;
                    int s = z[j];
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FWORD, (uint32_t)i, id, r);
                        int t = prop[j * M + (i - 1)];
                        if (t != s) {
#if ORC_MUTATION == 13
                            float num = ((((float)cd[t] + alpha) * ((float)row[t] + beta))
                                         * ((float)ck[s] + beta_bar)) * qd[t];   /* q terms swapped */
                            float den = ((((float)cd[s] + alpha) * ((float)row[s] + beta))
                                         * ((float)ck[t] + beta_bar)) * qd[s];
#else
                            float num = ((((float)cd[t] + alpha) * ((float)row[t] + beta))
                                         * ((float)ck[s] + beta_bar)) * qd[s];
                            float den = ((((float)cd[s] + alpha) * ((float)row[s] + beta))
                                         * ((float)ck[t] + beta_bar)) * qd[t];
#endif
                            if (u24(r[0]) * den < num) s = t;
                        }
                    }
                    znew[j] = s;
                    for (int i = 1; i <= M; ++i) {
                        draw_block(seed, (uint32_t)j, (uint32_t)it, ORC_PHASE_FWORD, (uint32_t)i, id, r);
                        prop[j * M + (i - 1)] = orc_frozen_word_draw(r[1], r[2], row, K, K_beta);
                    }
                }
                for (int j = 0; j < L; ++j) z[j] = znew[j];
            }
            if (theta_out) {
                for (int k = 0; k < K; ++k) cd[k] = 0;
                for (int j = 0; j < L; ++j) cd[z[j]] += 1;
                float den = (float)L + alpha_bar;
                for (int k = 0; k < K; ++k)
                    theta_out[d * K + k] = ((float)cd[k] + alpha) / den;
            }
        }
        free(cd); free(znew); free(prop); free(prob); free(alias);
    }
}

/*
 * Plain collapsed Gibbs fold-in (the yardstick of the fold-in statistics
 * test): the exact O(K) conditional (C_dk^- + alpha)(C_wk + beta)/(c_k + beta_bar)
 * with the frozen C_w and c_k and the token's own assignment removed from
 * c_d; its own Philox stream (phase 6).  Accumulates, over sweeps
 * burn+1..sweeps, the theta of Eq. 4 into theta_sum[Dn*K] (double).
 */
void orc_cgs_foldin(int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word, int K,
                    float alpha_f, float beta_f, float beta_bar_f, const int32_t* cw,
                    const int32_t* ck, uint64_t seed, int sweeps, int burn, double* theta_sum)
{
    double alpha = alpha_f, beta = beta_f, bbar = beta_bar_f;
#pragma omp parallel
    {
        int32_t* cd = (int32_t*)malloc((size_t)K * sizeof(int32_t));
        double* pk = (double*)malloc((size_t)K * sizeof(double));
        int64_t maxL = 1;
        for (int64_t d = 0; d < Dn; ++d)
            if (doc_ptr[d + 1] - doc_ptr[d] > maxL) maxL = doc_ptr[d + 1] - doc_ptr[d];
        int32_t* z = (int32_t*)malloc((size_t)maxL * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t d = 0; d < Dn; ++d) {
            int64_t b = doc_ptr[d];
            int L = (int)(doc_ptr[d + 1] - b);
            uint32_t r[4];
            for (int k = 0; k < K; ++k) cd[k] = 0;
            for (int j = 0; j < L; ++j) {
                draw_block(seed, (uint32_t)j, 0, 6, 0, (uint32_t)d, r);
                z[j] = (int32_t)dice(r[0], (uint32_t)K);
                cd[z[j]] += 1;
            }
            for (int s = 1; s <= sweeps; ++s) {
                for (int j = 0; j < L; ++j) {
                    const int32_t* row = cw + (int64_t)doc_word[b + j] * K;
                    cd[z[j]] -= 1;
                    double tot = 0.0;
                    for (int k = 0; k < K; ++k) {
                        tot += (cd[k] + alpha) * (row[k] + beta) / (ck[k] + bbar);
                        pk[k] = tot;
                    }
                    draw_block(seed, (uint32_t)j, (uint32_t)s, 6, 1, (uint32_t)d, r);
                    double u = ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6))
                               * (1.0 / 9007199254740992.0) * tot;
                    int k1 = 0;
                    while (k1 < K - 1 && pk[k1] <= u) ++k1;
                    z[j] = k1;
                    cd[k1] += 1;
                }
                if (s > burn)
                    for (int k = 0; k < K; ++k)
                        theta_sum[d * K + k] += (cd[k] + alpha) / (L + K * alpha);
            }
        }
        free(cd);
        free(pk);
        free(z);
    }
}

/* Threads the parallel phases will use. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
