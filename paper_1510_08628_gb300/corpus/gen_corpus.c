/*
 * Seeded synthetic LDA corpora (the generative process of Sec. 2.1).
 *
 * Input generator shared by the tests, the oracle checks and the benchmark.
 * It holds none of the sampler's arithmetic: it draws
 *   phi_k ~ Dirichlet(c * V * zipf_s)       (topic-word rows; zipf_s(r) ~ r^-s)
 *   theta_d ~ Dirichlet(a0)                 (integrated out: Polya urn below)
 *   z_dn ~ Mult(theta_d), w_dn ~ Mult(phi_{z_dn})
 * Document lengths are Poisson(mean) or lognormal(mean, sigma), at least 1.
 *
 * The doc-topic draw uses the Polya-urn form of the Dirichlet-multinomial:
 * token n of a document takes a uniformly chosen earlier token's topic with
 * probability n / (n + K_true a0), else a uniform topic -- exactly the law of
 * drawing theta_d ~ Dir(a0) and then z_dn ~ Mult(theta_d), at O(1) per token.
 *
 * Every document and every topic row has its own RNG stream (xoshiro256**
 * seeded through splitmix64 from (seed, tag, index)), so output is identical
 * for any thread count and a document's tokens do not depend on D.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t* r, uint64_t seed, uint64_t tag, uint64_t idx)
{
    uint64_t x = seed ^ (tag * 0xD6E8FEB86659FD93ull) ^ (idx * 0xA0761D6478BD642Full);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r)
{
    uint64_t* s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return out;
}

/* uniform in (0, 1) */
static double rng_u(rng_t* r) { return ((double)(rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static uint64_t rng_below(rng_t* r, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static double rng_normal(rng_t* r)
{
    double u1 = rng_u(r), u2 = rng_u(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* log of a Gamma(a, 1) variate; Marsaglia & Tsang (2000), with the
 * U^(1/a) boost for a < 1 carried in log space so tiny shapes do not
 * underflow. */
static double rng_log_gamma(rng_t* r, double a)
{
    double boost = 0.0;
    if (a < 1.0) {
        boost = log(rng_u(r)) / a;
        a += 1.0;
    }
    double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (;;) {
        double x, v;
        do {
            x = rng_normal(r);
            v = 1.0 + c * x;
        } while (v <= 0.0);
        v = v * v * v;
        double u = rng_u(r);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return log(d * v) + boost;
    }
}

static int64_t rng_poisson(rng_t* r, double lam)
{
    /* product of uniforms (Knuth); used only for modest means */
    double L = exp(-lam), p = 1.0;
    int64_t k = 0;
    do {
        ++k;
        p *= rng_u(r);
    } while (p > L);
    return k - 1;
}

enum { TAG_LEN = 1, TAG_DOC = 2, TAG_PHI = 3, TAG_PERM = 4 };

/*
 * Document lengths for documents [doc_offset, doc_offset + D).
 * kind 0: Poisson(mean); kind 1: lognormal with the given mean and sigma
 * (mu = ln(mean) - sigma^2 / 2), rounded; kind 2: lognormal clipped to
 * [lo, hi].  Zero-length draws become 1.
 */
void gen_lengths(int64_t D, int kind, double mean, double sigma, int64_t lo, int64_t hi,
                 uint64_t seed, int64_t doc_offset, int64_t* len_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t d = 0; d < D; ++d) {
        rng_t r;
        rng_seed(&r, seed, TAG_LEN, (uint64_t)(doc_offset + d));
        int64_t L;
        if (kind == 0) {
            L = rng_poisson(&r, mean);
        } else {
            double mu = log(mean) - 0.5 * sigma * sigma;
            L = (int64_t)llround(exp(mu + sigma * rng_normal(&r)));
            if (kind == 2) {
                if (L < lo) L = lo;
                if (L > hi) L = hi;
            }
        }
        len_out[d] = L < 1 ? 1 : L;
    }
}

/*
 * Topic-word rows phi_k ~ Dir(c V zipf_s), k < K_true, stored as Walker alias
 * tables (prob[K_true * V], alias[K_true * V]).  Rank r (1-based) of the Zipf
 * base maps to word id rank_to_word[r-1], a seeded permutation, so frequent
 * words are spread over the id range.  If phi_out is not NULL the normalised
 * rows are written there too (K_true * V doubles).
 */
void gen_topics(int64_t V, int K_true, double zipf_s, double conc_c, uint64_t seed,
                float* prob, int32_t* alias, int32_t* rank_to_word, double* phi_out)
{
    /* Zipf base and the rank -> word permutation */
    double H = 0.0;
    for (int64_t r = 1; r <= V; ++r) H += pow((double)r, -zipf_s);
    {
        rng_t pr;
        rng_seed(&pr, seed, TAG_PERM, 0);
        for (int64_t i = 0; i < V; ++i) rank_to_word[i] = (int32_t)i;
        for (int64_t i = V - 1; i > 0; --i) {
            int64_t j = (int64_t)rng_below(&pr, (uint64_t)(i + 1));
            int32_t t = rank_to_word[i];
            rank_to_word[i] = rank_to_word[j];
            rank_to_word[j] = t;
        }
    }
#pragma omp parallel
    {
        double* lw = (double*)malloc((size_t)V * sizeof(double));
        double* pw = (double*)malloc((size_t)V * sizeof(double));
        int64_t* small = (int64_t*)malloc((size_t)V * sizeof(int64_t));
        int64_t* large = (int64_t*)malloc((size_t)V * sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < K_true; ++k) {
            rng_t r;
            rng_seed(&r, seed, TAG_PHI, (uint64_t)k);
            double mx = -INFINITY;
            for (int64_t rk = 0; rk < V; ++rk) {
                double a = conc_c * (double)V * pow((double)(rk + 1), -zipf_s) / H;
                double g = rng_log_gamma(&r, a);
                lw[rank_to_word[rk]] = g;
                if (g > mx) mx = g;
            }
            double tot = 0.0;
            for (int64_t w = 0; w < V; ++w) {
                pw[w] = exp(lw[w] - mx);
                tot += pw[w];
            }
            for (int64_t w = 0; w < V; ++w) pw[w] /= tot;
            if (phi_out)
                for (int64_t w = 0; w < V; ++w) phi_out[(int64_t)k * V + w] = pw[w];
            /* Vose's alias method */
            float* pr = prob + (int64_t)k * V;
            int32_t* al = alias + (int64_t)k * V;
            int64_t ns = 0, nl = 0;
            for (int64_t w = 0; w < V; ++w) {
                pw[w] *= (double)V;
                if (pw[w] < 1.0) small[ns++] = w; else large[nl++] = w;
            }
            while (ns > 0 && nl > 0) {
                int64_t s = small[--ns], l = large[--nl];
                pr[s] = (float)pw[s];
                al[s] = (int32_t)l;
                pw[l] = (pw[l] + pw[s]) - 1.0;
                if (pw[l] < 1.0) small[ns++] = l; else large[nl++] = l;
            }
            while (nl > 0) { int64_t l = large[--nl]; pr[l] = 1.0f; al[l] = (int32_t)l; }
            while (ns > 0) { int64_t s = small[--ns]; pr[s] = 1.0f; al[s] = (int32_t)s; }
        }
        free(lw); free(pw); free(small); free(large);
    }
}

/*
 * Truncated topic-word rows for vocabularies where K_true * V dense tables do
 * not fit (ClueWeb-shaped: 5,000 x 10^6): phi_k ~ Dir(c V zipf_s) as above,
 * then every entry below `cut` of the row's mass is dropped and the rest
 * renormalised.  A shape a < 1 draws U first: when ln(U) / a < -60 the
 * entry is below e^-60 times a Gamma(1 + a) variate, far under the cut for
 * any row (the top entries have shapes in the hundreds), so its Gamma part
 * is not drawn.  Pass 1 (fill == 0) writes nnz[k]; pass 2 redraws the same
 * rows and writes, for topic k at [off[k], off[k+1]), the kept word ids and
 * their alias table over the kept entries.  rank_to_word as in gen_topics.
 */
static int64_t sparse_row(int64_t V, double zipf_s, double conc_c, double H, uint64_t seed, int k,
                          double cut, const int32_t* rank_to_word, double* lw, int64_t* keep,
                          double* pw, int64_t* small, int64_t* large, int32_t* words, float* prob,
                          int32_t* alias)
{
    rng_t r;
    rng_seed(&r, seed, TAG_PHI, (uint64_t)k);
    double mx = -INFINITY;
    for (int64_t rk = 0; rk < V; ++rk) {
        double a = conc_c * (double)V * pow((double)(rk + 1), -zipf_s) / H;
        double g;
        if (a < 1.0) {
            double boost = log(rng_u(&r)) / a;
            g = boost < -60.0 ? -INFINITY : rng_log_gamma(&r, a + 1.0) + boost;
        } else {
            g = rng_log_gamma(&r, a);
        }
        lw[rank_to_word[rk]] = g;
        if (g > mx) mx = g;
    }
    double tot = 0.0;
    for (int64_t w = 0; w < V; ++w) tot += exp(lw[w] - mx);
    const double lcut = log(cut * tot) + mx;   /* keep exp(lw - mx) / tot >= cut */
    int64_t n = 0;
    double kept = 0.0;
    for (int64_t w = 0; w < V; ++w)
        if (lw[w] >= lcut) {
            keep[n] = w;
            pw[n] = exp(lw[w] - mx);
            kept += pw[n];
            ++n;
        }
    if (!words) return n;
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        words[i] = (int32_t)keep[i];
        pw[i] = pw[i] / kept * (double)n;
        if (pw[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t sm = small[--ns], l = large[--nl];
        prob[sm] = (float)pw[sm];
        alias[sm] = (int32_t)l;
        pw[l] = (pw[l] + pw[sm]) - 1.0;
        if (pw[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; prob[l] = 1.0f; alias[l] = (int32_t)l; }
    while (ns > 0) { int64_t sm = small[--ns]; prob[sm] = 1.0f; alias[sm] = (int32_t)sm; }
    return n;
}

void gen_topics_sparse(int64_t V, int K_true, double zipf_s, double conc_c, uint64_t seed,
                       double cut, int fill, int32_t* rank_to_word, int64_t* nnz,
                       const int64_t* off, int32_t* words, float* prob, int32_t* alias)
{
    double H = 0.0;
    for (int64_t r = 1; r <= V; ++r) H += pow((double)r, -zipf_s);
    if (!fill) {
        rng_t pr;
        rng_seed(&pr, seed, TAG_PERM, 0);
        for (int64_t i = 0; i < V; ++i) rank_to_word[i] = (int32_t)i;
        for (int64_t i = V - 1; i > 0; --i) {
            int64_t j = (int64_t)rng_below(&pr, (uint64_t)(i + 1));
            int32_t t = rank_to_word[i];
            rank_to_word[i] = rank_to_word[j];
            rank_to_word[j] = t;
        }
    }
#pragma omp parallel
    {
        double* lw = (double*)malloc((size_t)V * sizeof(double));
        double* pw = (double*)malloc((size_t)V * sizeof(double));
        int64_t* keep = (int64_t*)malloc((size_t)V * sizeof(int64_t));
        int64_t* small = (int64_t*)malloc((size_t)V * sizeof(int64_t));
        int64_t* large = (int64_t*)malloc((size_t)V * sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < K_true; ++k) {
            if (!fill)
                nnz[k] = sparse_row(V, zipf_s, conc_c, H, seed, k, cut, rank_to_word, lw, keep, pw, small,
                                    large, NULL, NULL, NULL);
            else
                sparse_row(V, zipf_s, conc_c, H, seed, k, cut, rank_to_word, lw, keep, pw, small, large,
                           words + off[k], prob + off[k], alias + off[k]);
        }
        free(lw); free(pw); free(keep); free(small); free(large);
    }
}

/* gen_words over truncated rows: w = words[off[z] + alias draw over nnz_z]. */
void gen_words_sparse(int64_t D, const int64_t* doc_ptr, int K_true, double a0, const int64_t* off,
                      const int32_t* words, const float* prob, const int32_t* alias, uint64_t seed,
                      int64_t doc_offset, int32_t* doc_word, int32_t* true_z_out)
{
#pragma omp parallel
    {
        int64_t cap = 0;
        int32_t* zs = NULL;
#pragma omp for schedule(dynamic, 256)
        for (int64_t d = 0; d < D; ++d) {
            int64_t b = doc_ptr[d], L = doc_ptr[d + 1] - b;
            if (L > cap) {
                free(zs);
                cap = L;
                zs = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
            }
            rng_t r;
            rng_seed(&r, seed, TAG_DOC, (uint64_t)(doc_offset + d));
            double ka = (double)K_true * a0;
            for (int64_t n = 0; n < L; ++n) {
                int32_t z;
                if (rng_u(&r) * ((double)n + ka) < (double)n)
                    z = zs[rng_below(&r, (uint64_t)n)];
                else
                    z = (int32_t)rng_below(&r, (uint64_t)K_true);
                zs[n] = z;
                int64_t base = off[z], nz = off[z + 1] - base;
                int64_t bin = base + (int64_t)rng_below(&r, (uint64_t)nz);
                int32_t w = (rng_u(&r) < (double)prob[bin]) ? words[bin] : words[base + alias[bin]];
                doc_word[b + n] = w;
                if (true_z_out) true_z_out[b + n] = z;
            }
        }
        free(zs);
    }
}

/*
 * Tokens of documents [doc_offset, doc_offset + D) with the given CSR
 * offsets: z by the Polya urn of Dir(a0) over K_true topics, w ~ phi_z by the
 * alias tables.  true_z_out (optional) receives the generating topics.
 */
void gen_words(int64_t D, const int64_t* doc_ptr, int64_t V, int K_true, double a0,
               const float* prob, const int32_t* alias, uint64_t seed, int64_t doc_offset,
               int32_t* doc_word, int32_t* true_z_out)
{
#pragma omp parallel
    {
        int64_t cap = 0;
        int32_t* zs = NULL;
#pragma omp for schedule(dynamic, 256)
        for (int64_t d = 0; d < D; ++d) {
            int64_t b = doc_ptr[d], L = doc_ptr[d + 1] - b;
            if (L > cap) {
                free(zs);
                cap = L;
                zs = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
            }
            rng_t r;
            rng_seed(&r, seed, TAG_DOC, (uint64_t)(doc_offset + d));
            double ka = (double)K_true * a0;
            for (int64_t n = 0; n < L; ++n) {
                int32_t z;
                if (rng_u(&r) * ((double)n + ka) < (double)n)
                    z = zs[rng_below(&r, (uint64_t)n)];
                else
                    z = (int32_t)rng_below(&r, (uint64_t)K_true);
                zs[n] = z;
                uint64_t bin = rng_below(&r, (uint64_t)V);
                int64_t idx = (int64_t)z * V + (int64_t)bin;
                int32_t w = (rng_u(&r) < (double)prob[idx]) ? (int32_t)bin : alias[idx];
                doc_word[b + n] = w;
                if (true_z_out) true_z_out[b + n] = z;
            }
        }
        free(zs);
    }
}
