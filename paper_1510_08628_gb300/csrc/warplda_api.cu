// C ABI of libwarplda.so (include/warplda.h): device state, the host-side
// token-order build at initialisation (Sec. 5.2 layout: word-major store plus
// the doc-major pointer array perm), work lists, and the per-phase launch
// sequence of the sweep (Sec. 4.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <chrono>
#include <map>
#include <new>
#include <stdexcept>
#include <mutex>

#include "../../include/warplda.h"
#include "wl_kernels.h"

using namespace wl;

namespace {

thread_local std::string g_err;

// Fault injection (see launch_gate in wl_kernels.h): the count of calls that
// saw the variable's current value.
struct InjectState {
    std::string value;
    long count = 0;
};
std::mutex g_inject_mu;
InjectState g_inject_launch, g_inject_alloc;

bool inject_fires(const char* var, InjectState& st) {
    const char* v = std::getenv(var);
    std::lock_guard<std::mutex> lock(g_inject_mu);
    if (!v || !*v) {
        st.value.clear();
        st.count = 0;
        return false;
    }
    if (st.value != v) {
        st.value = v;
        st.count = 0;
    }
    const long k = std::strtol(v, nullptr, 10);
    return k > 0 && ++st.count == k;
}

// Every device and pinned host allocation of the library goes through these.
cudaError_t dev_malloc(void** p, size_t bytes) {
    if (const cudaError_t e = alloc_gate()) return e;
    return cudaMalloc(p, bytes);
}
cudaError_t host_malloc(void** p, size_t bytes) {
    if (const cudaError_t e = alloc_gate()) return e;
    return cudaMallocHost(p, bytes);
}

int64_t r4(int64_t x) { return (x + 3) & ~(int64_t)3; }

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? WARPLDA_ENOMEM : WARPLDA_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define WL_CU(call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

// Host-side exceptions never cross the C ABI: every int-returning entry
// point is a function-try-block ending in this handler, so a failed host
// allocation comes back as ENOMEM (objects being built are freed by their
// ScopeExit guards as the stack unwinds).
#define WL_ABI_CATCH                                                        \
    catch (const std::bad_alloc&) {                                         \
        return fail(WARPLDA_ENOMEM, "host allocation failed");              \
    }                                                                       \
    catch (const std::length_error&) {                                      \
        return fail(WARPLDA_ENOMEM, "host allocation too large");           \
    }                                                                       \
    catch (const std::exception& ex_) {                                     \
        return fail(WARPLDA_EINTERNAL, "host-side failure: %s", ex_.what()); \
    }                                                                       \
    catch (...) {                                                           \
        return fail(WARPLDA_EINTERNAL, "host-side failure");                \
    }

// Runs f when the scope ends unless disarmed: frees an object that is being
// built when its construction is left early, by a return or an exception.
template <class F>
struct ScopeExit {
    F f;
    bool armed = true;
    ~ScopeExit() {
        if (armed) f();
    }
};
template <class F>
ScopeExit<F> on_exit(F f) {
    return ScopeExit<F>{f};
}

enum KernelClass {
    kcDocWarp, kcDocBatch, kcDocHugeHist, kcDocHugeAccept, kcDocHugeDraw,
    kcWordBatch, kcWordMegaHist, kcWordMegaAccept, kcWordMegaHistPost, kcWordMegaDraw,
    kcCountCk, kcFinalize, kcZero, kcDocPipe, kcWordCluster,
    kcFoldBuild, kcFoldDoc, kcFoldWord, kcFoldin,
    kcServe, kcServeNew, kcServeAdmit, kcServeEncoder, kcServeAlias, kcServeRows, kcCount
};
const char* kClassNames[kcCount] = {
    "doc_warp", "doc_batch", "doc_huge_hist", "doc_huge_accept", "doc_huge_draw",
    "word_batch", "word_mega_hist", "word_mega_accept", "word_mega_hist_post", "word_mega_draw",
    "count_ck", "finalize_ck", "zero_rows", "doc_pipe", "word_cluster",
    "foldin_build", "foldin_doc", "foldin_word", "foldin_kernel",
    "serve", "serve_new", "serve_admit", "serve_encoder", "serve_alias", "serve_rows"};
// topics: packed hash entries hold (topic + 1) << 12 in 32 bits
constexpr int kMaxTopics = (1 << 20) - 1;
// tokens of a pipelined document batch (at most 4 * 256 - 3; at most 509
// gives the kernel's 2-tokens-per-thread form)
#ifndef WL_PIPE_TOKENS
#define WL_PIPE_TOKENS 1021
#endif
constexpr int kPipeTokens = WL_PIPE_TOKENS;
static_assert(kPipeTokens >= 1 && kPipeTokens <= 4 * kThreads - 3, "pipelined batch size");
// cluster sizes of the cluster tier: 1, 2, 4, 8, 16 blocks
constexpr int kClusterClasses = 5;
// ranges of the multi-pass tier with dense rows, per SM: enough that the
// last wave of blocks is short (4 per SM left a 1.33-wave tail with three
// resident blocks per SM: 7.7 against 5.8 ms for the PubMed-shaped accept)
#ifndef WL_RANGES_PER_SM
#define WL_RANGES_PER_SM 32
#endif
constexpr int kRangesPerSm = WL_RANGES_PER_SM;
// serving: documents of at least this many tokens are swept by a block
constexpr int kServeBlockMin = 512;
// serving with the learned proposal: requests of at least this many sweeps
// join the step after their admission, shorter ones the step of it
constexpr int kServeDeferMin = 8;
// word-major fold-in: words with at least this many request tokens have
// their frozen row staged in shared memory, the others keep direct loads
#ifndef WL_FOLD_STAGE_MIN
#define WL_FOLD_STAGE_MIN 64
#endif
constexpr int kFoldStageMin = WL_FOLD_STAGE_MIN;
static_assert(kFoldStageMin >= 1, "staging threshold");
// above this K the multi-pass tier's count rows are sparse (global hash)
constexpr int kDenseRowMaxK = 16384;
// work counters: 0-3 batches [class][phase], 4 doc warp tier, 5-8 the
// multi-pass passes (hist, accept, post hist, draw), 9 log-likelihood hist
constexpr int kCounters = 12;
constexpr int kCtrHist = 5, kCtrAccept = 6, kCtrHistPost = 7, kCtrDraw = 8, kCtrLoglik = 9;

struct Rec {
    int cls;
    cudaEvent_t a, b;
};

struct Tier {
    std::vector<int4> batches[2];    // {first segment, end segment, table words, 0}: small, large
    std::vector<int32_t> warp_list;  // segments of the warp tier (documents only)
    std::vector<int4> chunks;        // pieces {row, segment, first position, count}
    std::vector<int32_t> row_len;    // tokens of each long segment (row)
    std::vector<int32_t> range_off;  // range r = pieces [range_off[r], range_off[r+1])
    std::vector<int32_t> region;     // table offset of each batched segment in its batch
    std::vector<int4> ll_batches;    // log-likelihood batches over all non-chunked segments
    // long segments sampled on a thread-block cluster (words only); they keep
    // their rows and pieces above for the log-likelihood, and the multi-pass
    // sampling passes take the pieces s_chunks / ranges s_range_off of the
    // other long segments
    std::vector<int32_t> cluster_list;   // grouped by cluster size: class c holds
    std::vector<int32_t> cluster_cls;    // cluster_list[cluster_cls[c] .. cluster_cls[c+1])
    std::vector<int4> s_chunks;
    std::vector<int32_t> s_range_off;
    int64_t cluster_tokens = 0, s_row_tokens = 0;
    int32_t* d_cluster_list = nullptr;
    int4* d_s_chunks = nullptr;
    int32_t* d_s_range_off = nullptr;
    int64_t nrows = 0, row_tokens = 0, large_tokens = 0, warp_tokens = 0;
    int4* d_batches[2] = {nullptr, nullptr};
    int32_t* d_warp_list = nullptr;
    int4* d_chunks = nullptr;
    int32_t* d_range_off = nullptr;
    int32_t* d_region = nullptr;
    int4* d_ll_batches = nullptr;
};

}  // namespace

struct warplda_ctx {
    int64_t D = 0, V = 0, N = 0;
    int K = 0, M = 0;
    float alpha = 0, beta = 0, abar = 0, bbar = 0, kbeta = 0;
    uint64_t seed = 0;
    uint32_t k0 = 0, k1 = 0;
    uint32_t iter = 0;
    int doc_done = 0;
    cudaStream_t st = nullptr;
    int dev = 0, sms = 0;
    int bmax[2] = {0, 0}, region[2] = {0, 0}, chunk = 0, stage_ck = 0, kbits = 0;
    // tokens per thread of the small batch class, per phase [doc, word]: 4
    // for documents with hash tables (more resident blocks for the
    // latency-bound gather and probe loops), else 8
    int tpt0[2] = {8, 8};
    int dbmax[2] = {0, 0};
    int dregion[2] = {0, 0};   // table budget of the document batches [class]
    // document batches of the small class run in the pipelined kernel
    // (wl_docpipe.cu): by default with hash tables, or as tuning says
    bool doc_pipe = true;
    int4* d_pipe_desc = nullptr;
    int grid_pipe = 1;
    // words sampled on a thread-block cluster: cluster size, tokens per block
    // (slice capacity), dynamic shared memory per block
    int cluster_C = 0, cluster_T = 0, cluster_smem = 0;
    // plain-proposal fold-in: word-major phases (default) or one warp per
    // document for all sweeps (tuning foldin_kernel = 1)
    bool foldin_word_major = true;
    // warplda_foldin's device scratch, kept between calls and grown on
    // demand (slot i = the call's i-th buffer)
    struct Scratch {
        void* p = nullptr;
        size_t bytes = 0;
    };
    std::vector<Scratch> fold_ws;
    bool dense = true;   // 16-bit dense count tables (K <= kDenseMaxK), else hash tables
    int warp_tpl = 16;   // tokens per lane of the document warp tier
    int grid_doc_warp = 1;
    int32_t *z = nullptr, *prop = nullptr, *perm = nullptr, *doc_off = nullptr, *word_off = nullptr;
    int32_t* sperm = nullptr;     // document batches' tokens in word-major order
    uint32_t* sinfo = nullptr;    // their (slot << 16 | position in batch)
    int32_t *ck = nullptr, *counters = nullptr, *rows = nullptr, *scratch = nullptr;
    float* ckb = nullptr;
    double* d_ll = nullptr;
    int32_t* d_bad = nullptr;
    int32_t* d_fault = nullptr;   // index-check record of the kernels
    bool sync_check = false;      // WARPLDA_SYNC_CHECK=1: read the record after every launch
    int word_storage = 0;         // word proposals by storage-order positioning
    int32_t *rows_doc = nullptr, *rows_pre = nullptr, *rows_post = nullptr;
    int64_t rows_words = 0;
    // K above a shared-memory row: long segments count into sparse hash rows
    // in global memory ([0] documents, [1] words)
    bool sparse = false;
    int ck_delta = 0;   // kernels apply c_k deltas in global memory (sparse mode)
    int64_t* d_soff[2] = {nullptr, nullptr};
    unsigned long long* sslots[2] = {nullptr, nullptr};
    int64_t sn[2] = {0, 0};
    Tier docs, words;
    std::vector<int64_t> word_ptr_h;
    int grid_batch[2][2] = {{1, 1}, {1, 1}};   // [doc 0 / word 1][class]
    int grid_hist = 1, grid_acc_doc = 1, grid_acc_word = 1, grid_draw = 1, grid_topic = 1;
    // frozen model of fold-in, taken after sweep model_iter: C_w ([V, K]),
    // each word's topics ascending ([N]) and (float)c_k + beta_bar
    int32_t* model_cw = nullptr;
    int32_t* model_zs = nullptr;
    float* model_ckb = nullptr;
    int64_t model_iter = -1;
    bool prof = false;
    std::vector<Rec> recs;
    int64_t device_bytes = 0;
    std::vector<void*> allocs;
    // fold-in encoder (learned document proposal)
    struct Encoder {
        int log2F = 0, H = 0, Kp = 0, B = 256, step = 0;
        float *W1 = nullptr, *b1 = nullptr, *W2t = nullptr, *b2 = nullptr;   // FP32 masters
        float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2;               // Adam moments
        uint16_t *W1b, *W2tb, *W2nb;                                          // BF16 copies
        float *gW1, *gb1, *gW2t, *gb2;                                        // gradients
        float *h_pre, *logits, *dH;
        float* gwork = nullptr;      // split-K partial tiles of the three GEMMs
        int64_t gwork_floats = 0;
        uint16_t *hb, *hbT, *dl, *dlT;
        int32_t *cnt, *ids, *docword = nullptr;
        double* loss;
        bool ready = false;
    } enc;
};

namespace {

template <typename T>
int dalloc(warplda_ctx* c, T** p, int64_t n, const char* what) {
    size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    cudaError_t e = dev_malloc((void**)p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    c->allocs.push_back(*p);
    c->device_bytes += (int64_t)bytes;
    e = cudaMemsetAsync(*p, 0, bytes, c->st);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return WARPLDA_OK;
}

void free_all(warplda_ctx* c) {
    for (auto& r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->recs.clear();
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    for (auto& w : c->fold_ws)
        if (w.p) cudaFree(w.p);
    c->fold_ws.clear();
}

// Table words of a segment of L tokens: dense ceil(K/2) words (two 16-bit
// counts each), or a hash of the smallest power of two above min(2L, K)
// (Sec. 5.4); empty segments need none.
int table_words(int L, int K, bool dense) {
    if (L <= 0) return 0;
    if (dense) return (K + 1) / 2;
    return (int)pow2_above((uint32_t)std::min(2 * L, K));
}

// Split segments [0, S) with offsets off[] into the kernel tiers: segments
// with 1..warp_max tokens go to the warp tier (warp_max = 0: none); small
// segments to block batches of the 8-tokens-per-thread kernel (at most
// bmax[0] tokens, segs0 segments, region[0] table words per batch), large
// ones to batches of the 16-tokens-per-thread kernel (bmax[1], region[1]);
// longer segments get a count row, and their tokens are cut into ranges of
// about equal size (ranges_target of them), each a list of pieces of at
// most `chunk` tokens of one segment.  A batch is a run of
// consecutive segments of one class (empty segments join the open batch);
// each batched segment records its table offset within the batch.  The
// log-likelihood batches cover every segment that is not chunked, with the
// paper's table rule.
// The tier lists of segments [s0, s1): the greedy batching below, closed at
// s1.  Rows of long segments are numbered from 0 within the part.
struct TierPart {
    std::vector<int4> batches[2], ll_batches, longs, s_longs;
    std::vector<int32_t> warp_list, row_len;
    std::vector<int2> cl_words;   // {tokens, segment} of the cluster tier
    int64_t nrows = 0, row_tokens = 0, large_tokens = 0, warp_tokens = 0, cluster_tokens = 0, s_row_tokens = 0;
};

void scan_tier(const std::vector<int32_t>& off, int64_t s0, int64_t s1, int K, bool dense, int warp_max,
               const int bmax[2], const int region[2], const int segs_max[2], int64_t cluster_max,
               int32_t* seg_region, TierPart* t) {
    int cur0 = -1, cls = -1, ntok = 0, nseg = 0, nw = 0;
    auto close = [&](int end) {
        if (cur0 >= 0 && end > cur0) t->batches[cls].push_back(make_int4(cur0, end, nw, 0));
        cur0 = -1;
        ntok = nseg = nw = 0;
    };
    int l0 = -1, lt = 0, ls = 0, lw = 0;   // open log-likelihood batch
    auto lclose = [&](int end) {
        if (l0 >= 0 && end > l0) t->ll_batches.push_back(make_int4(l0, end, lw, 0));
        l0 = -1;
        lt = ls = lw = 0;
    };
    for (int64_t s = s0; s < s1; ++s) {
        const int L = off[s + 1] - off[s];
        if (L == 0) {
            if (cur0 >= 0 && nseg + 1 <= segs_max[cls]) {
                seg_region[s] = nw;
                nseg += 1;
            } else {
                close((int)s);
            }
            if (l0 >= 0 && ls + 1 <= kSegsMax) ls += 1; else lclose((int)s);
            continue;
        }
        const int w = table_words(L, K, dense);
        int c = -1;
        if (L <= warp_max) c = 2;
        else if (L <= bmax[0] && w <= region[0]) c = 0;
        else if (L <= bmax[1] && w <= region[1]) c = 1;
        if (c < 0) {
            close((int)s);
            lclose((int)s);
            const int row = (int)t->nrows++;
            t->row_tokens += L;
            t->row_len.push_back(L);
            t->longs.push_back(make_int4(row, (int)s, off[s], L));
            if (cluster_max > 0 && L <= cluster_max) {
                t->cl_words.push_back(make_int2(L, (int)s));
                t->cluster_tokens += L;
            } else {
                t->s_longs.push_back(make_int4(row, (int)s, off[s], L));
                t->s_row_tokens += L;
            }
            continue;
        }
        // log-likelihood batches (paper's table rule)
        {
            uint32_t w2 = 0, cap2 = 0;
            table_shape((uint32_t)L, (uint32_t)K, &w2, &cap2);
            if (l0 >= 0 && (lt + L > kMaxBatchTokens || ls + 1 > kSegsMax || lw + (int)w2 > 8192))
                lclose((int)s);
            if (l0 < 0) l0 = (int)s;
            lt += L;
            ls += 1;
            lw += (int)w2;
        }
        if (c == 2) {
            close((int)s);
            t->warp_list.push_back((int32_t)s);
            t->warp_tokens += L;
            continue;
        }
        if (c == 1) t->large_tokens += L;
        if (cur0 >= 0 && (c != cls || ntok + L > bmax[c] || nseg + 1 > segs_max[c] || nw + w > region[c]))
            close((int)s);
        if (cur0 < 0) {
            cur0 = (int)s;
            cls = c;
        }
        seg_region[s] = nw;
        ntok += L;
        nseg += 1;
        nw += w;
    }
    close((int)s1);
    lclose((int)s1);
}

// Segments per part of the tier scan.  Parts are scanned on host threads;
// a batch never spans two parts, so the lists depend on this size only, not
// on the number of host cores.
constexpr int64_t kTierPart = 1 << 20;

void build_tier(const std::vector<int32_t>& off, int64_t S, int K, bool dense, int warp_max,
                const int bmax[2], const int region[2], int chunk, int ranges_target, Tier* t,
                int segs0 = kSegsMax, int64_t cluster_max = 0, int64_t cluster_slice = 1) {
    const int segs_max[2] = {segs0, kSegsMax};
    for (auto& b : t->batches) b.clear();
    t->warp_list.clear();
    t->chunks.clear();
    t->row_len.clear();
    t->range_off.clear();
    t->ll_batches.clear();
    t->cluster_list.clear();
    t->s_chunks.clear();
    t->s_range_off.clear();
    t->cluster_tokens = t->s_row_tokens = 0;
    t->region.assign((size_t)std::max<int64_t>(S, 1), 0);
    t->nrows = t->row_tokens = t->large_tokens = t->warp_tokens = 0;
    const int64_t nparts = std::max<int64_t>(1, (S + kTierPart - 1) / kTierPart);
    std::vector<TierPart> parts((size_t)nparts);
    auto scan = [&](int64_t i) {
        scan_tier(off, i * kTierPart, std::min(S, (i + 1) * kTierPart), K, dense, warp_max, bmax, region, segs_max,
                  cluster_max, t->region.data(), &parts[(size_t)i]);
    };
    {
        // parts taken from a counter by up to 15 helper threads and this one
        // (which alone does the work if no thread can be started)
        std::atomic<int64_t> next{0};
        auto work = [&] {
            for (int64_t i; (i = next.fetch_add(1)) < nparts;) scan(i);
        };
        std::vector<std::thread> th;
        const int helpers = (int)std::min<int64_t>(nparts - 1, (int64_t)std::min(15u, std::thread::hardware_concurrency()));
        try {
            for (int k = 0; k < helpers; ++k) th.emplace_back(work);
        } catch (...) {
        }
        work();
        for (auto& x : th) x.join();
    }
    // the parts in segment order; rows renumbered
    std::vector<int4> s_longs;   // long segments of the multi-pass sampling passes
    std::vector<int2> cl_words;  // {tokens, segment} of the cluster tier
    std::vector<int4> longs;     // {row, segment, first position, length}
    for (auto& p : parts) {
        const int base = (int)t->nrows;
        for (int k = 0; k < 2; ++k) t->batches[k].insert(t->batches[k].end(), p.batches[k].begin(), p.batches[k].end());
        t->ll_batches.insert(t->ll_batches.end(), p.ll_batches.begin(), p.ll_batches.end());
        t->warp_list.insert(t->warp_list.end(), p.warp_list.begin(), p.warp_list.end());
        t->row_len.insert(t->row_len.end(), p.row_len.begin(), p.row_len.end());
        for (int4 h : p.longs) longs.push_back(make_int4(h.x + base, h.y, h.z, h.w));
        for (int4 h : p.s_longs) s_longs.push_back(make_int4(h.x + base, h.y, h.z, h.w));
        cl_words.insert(cl_words.end(), p.cl_words.begin(), p.cl_words.end());
        t->nrows += p.nrows;
        t->row_tokens += p.row_tokens;
        t->large_tokens += p.large_tokens;
        t->warp_tokens += p.warp_tokens;
        t->cluster_tokens += p.cluster_tokens;
        t->s_row_tokens += p.s_row_tokens;
    }
    // ranges of about equal size over the long segments' tokens, each a list
    // of pieces of at most `chunk` tokens of one segment
    auto make_ranges = [&](const std::vector<int4>& ls, int64_t tokens, std::vector<int4>* chunks,
                           std::vector<int32_t>* range_off) {
        if (tokens <= 0) return;
        const int64_t R = std::max<int64_t>(1, std::min<int64_t>(ranges_target, (tokens + 4095) / 4096));
        const int64_t per = (tokens + R - 1) / R;
        int64_t fill = 0;
        range_off->push_back(0);
        for (const int4& h : ls) {
            int p = h.z, left = h.w;
            while (left > 0) {
                const int take = (int)std::min<int64_t>(std::min<int64_t>(left, per - fill), chunk);
                chunks->push_back(make_int4(h.x, h.y, p, take));
                p += take;
                left -= take;
                fill += take;
                if (fill == per) {
                    range_off->push_back((int32_t)chunks->size());
                    fill = 0;
                }
            }
        }
        if (fill > 0) range_off->push_back((int32_t)chunks->size());
    };
    make_ranges(longs, t->row_tokens, &t->chunks, &t->range_off);
    make_ranges(s_longs, t->s_row_tokens, &t->s_chunks, &t->s_range_off);
    // cluster-tier words by cluster size: class c (size 2^c) takes the words
    // whose slices fit with 2^c blocks but not with 2^(c-1)
    t->cluster_cls.assign(kClusterClasses + 1, 0);
    if (!cl_words.empty()) {
        std::vector<std::vector<int32_t>> by(kClusterClasses);
        for (const int2& w : cl_words) {
            int c = 0;
            while (c + 1 < kClusterClasses && (int64_t)(1 << c) * cluster_slice < w.x) ++c;
            by[c].push_back(w.y);
        }
        for (int c = 0; c < kClusterClasses; ++c) {
            t->cluster_cls[c] = (int32_t)t->cluster_list.size();
            t->cluster_list.insert(t->cluster_list.end(), by[c].begin(), by[c].end());
        }
    }
    t->cluster_cls[kClusterClasses] = (int32_t)t->cluster_list.size();
}

// Reads the index-check record of the kernels (synchronises); a non-zero
// record means a kernel met a bad index and skipped the access.
int check_record(warplda_ctx* c, const char* where) {
    int32_t f[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(f, c->d_fault, sizeof(f), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        // a fault of an earlier launch surfaces here: name the call that read
        // the record (with WARPLDA_SYNC_CHECK=1, the launch just made)
        char what[96];
        std::snprintf(what, sizeof(what), "read check record after %s", where);
        return cuda_fail(e, what);
    }
    if (f[0] == 0 && f[3] == 0) return WARPLDA_OK;
    WL_CU(cudaMemsetAsync(c->d_fault, 0, sizeof(f), c->st), "clear check record");
    if (f[0] == 0) return fail(WARPLDA_ETIMEDOUT, "a tensor-core wait ran out (reported at %s)", where);
    static const char* kSites[] = {"?", "doc batch", "word batch", "multi-pass hist",
                                   "multi-pass accept", "multi-pass draw", "doc warp", "loglik",
                                   "fold-in", "word cluster"};
    const char* site = (f[0] >= 1 && f[0] <= 9) ? kSites[f[0]] : "?";
    return fail(WARPLDA_ECUDA, "index check failed (reported at %s): first in the %s kernel, checks 0x%x",
                where, site, (unsigned)f[2]);
}

int launch_rec(warplda_ctx* c, int cls, cudaError_t (*fn)(warplda_ctx*, void*), void* arg) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        WL_CU(cudaEventCreate(&a), "cudaEventCreate");
        WL_CU(cudaEventCreate(&b), "cudaEventCreate");
        WL_CU(cudaEventRecord(a, c->st), "cudaEventRecord");
    }
    cudaError_t e = fn(c, arg);
    if (e != cudaSuccess) return cuda_fail(e, kClassNames[cls]);
    if (c->prof) {
        WL_CU(cudaEventRecord(b, c->st), "cudaEventRecord");
        c->recs.push_back(Rec{cls, a, b});
    }
    if (c->sync_check) {
        // debugging mode (WARPLDA_SYNC_CHECK=1): every launch is followed by a
        // look at the index-check record
        const int rc = check_record(c, kClassNames[cls]);
        if (rc) return rc;
    }
    return WARPLDA_OK;
}

// A launch outside the sweep (fold-in, serving), timed like launch_rec on
// the stream it is queued on.
template <class F>
int launch_timed(warplda_ctx* c, int cls, F&& fn, cudaStream_t on = nullptr) {
    if (!on) on = c->st;
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        WL_CU(cudaEventCreate(&a), "cudaEventCreate");
        WL_CU(cudaEventCreate(&b), "cudaEventCreate");
        WL_CU(cudaEventRecord(a, on), "cudaEventRecord");
    }
    const cudaError_t e = fn();
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        return cuda_fail(e, kClassNames[cls]);
    }
    if (c->prof) {
        WL_CU(cudaEventRecord(b, on), "cudaEventRecord");
        c->recs.push_back(Rec{cls, a, b});
    }
    return WARPLDA_OK;
}

PhaseArgs phase_args(warplda_ctx* c, bool doc, uint32_t iter) {
    PhaseArgs a;
    a.z = c->z;
    a.prop = c->prop;
    a.perm = c->perm;
    a.sperm = c->sperm;
    a.sinfo = c->sinfo;
    a.seg_off = doc ? c->doc_off : c->word_off;
    a.ckb = c->ckb;
    a.K = c->K;
    a.M = c->M;
    a.g = doc ? c->alpha : c->beta;
    a.G = doc ? c->abar : c->kbeta;
    a.iter = iter;
    a.rk = round_keys(c->seed);
    a.ck = c->ck;
    a.word_storage = c->word_storage;
    a.stage_ck = c->stage_ck;
    a.ck_delta = c->ck_delta;
    a.N = c->N;
    a.nseg_total = doc ? c->D : c->V;
    a.fault = c->d_fault;
    return a;
}

struct PhaseCall {
    PhaseArgs a;
    bool doc;
    int cls;
};

// Work of the multi-pass passes: the sampling pieces (long segments not on a
// cluster), or with `all` every long segment's pieces (log-likelihood).
HugeWork huge_work(warplda_ctx* c, const Tier& T, int counter, bool all = false) {
    HugeWork w;
    w.pieces = all ? T.d_chunks : T.d_s_chunks;
    w.range_off = all ? T.d_range_off : T.d_s_range_off;
    w.nranges = (int)(all ? T.range_off.size() : T.s_range_off.size()) - 1;
    w.npieces = (int)(all ? T.chunks.size() : T.s_chunks.size());
    w.nrows = (int)T.nrows;
    w.guide_bits = huge_guide_bits(c->K);
    w.counter = c->counters + counter;
    return w;
}

int run_phase(warplda_ctx* c, bool doc) {
    const uint32_t it = c->iter + 1;
    PhaseCall pc{phase_args(c, doc, it), doc, 0};
    Tier& T = doc ? c->docs : c->words;
    const int nch = (int)T.s_chunks.size();
    int rc;
    if (nch > 0 && c->sparse) {
        rc = launch_rec(c, kcZero, [](warplda_ctx* cc, void* p) {
            const int k = ((PhaseCall*)p)->doc ? 0 : 1;
            return cudaMemsetAsync(cc->sslots[k], 0, (size_t)cc->sn[k] * 8, cc->st);
        }, &pc);
        if (rc) return rc;
        rc = launch_rec(c, doc ? kcDocHugeHist : kcWordMegaHist, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            const int k = q->doc ? 0 : 1;
            return launch_sparse_hist(q->doc, q->a, huge_work(cc, q->doc ? cc->docs : cc->words, kCtrHist),
                                      SparseRows{cc->d_soff[k], cc->sslots[k]}, cc->grid_hist, cc->st);
        }, &pc);
        if (rc) return rc;
    } else if (nch > 0) {
        rc = launch_rec(c, kcZero, [](warplda_ctx* cc, void* p) {
            const bool d = ((PhaseCall*)p)->doc;
            return d ? launch_zero(cc->rows_doc, r4(cc->docs.nrows * (int64_t)cc->K), cc->st)
                     : launch_zero(cc->rows_pre, 2 * r4(cc->words.nrows * (int64_t)cc->K), cc->st);
        }, &pc);
        if (rc) return rc;
        rc = launch_rec(c, doc ? kcDocHugeHist : kcWordMegaHist, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            return launch_huge_hist(q->doc, q->a, huge_work(cc, q->doc ? cc->docs : cc->words, kCtrHist),
                                    q->doc ? cc->rows_doc : cc->rows_pre, cc->grid_hist, cc->st);
        }, &pc);
        if (rc) return rc;
    }
    if (doc && !T.warp_list.empty()) {
        rc = launch_rec(c, kcDocWarp, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            return launch_doc_warp(cc->warp_tpl, cc->dense, q->a, cc->docs.d_warp_list,
                                   (int)cc->docs.warp_list.size(), cc->counters + 4,
                                   cc->grid_doc_warp, cc->st);
        }, &pc);
        if (rc) return rc;
    }
    for (int cls = 1; cls >= 0; --cls) {
        if (T.batches[cls].empty()) continue;
        pc.cls = cls;
        rc = launch_rec(c, doc ? (cls == 0 && c->doc_pipe ? kcDocPipe : kcDocBatch) : kcWordBatch,
                        [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            Tier& TT = q->doc ? cc->docs : cc->words;
            const int k = q->cls;
            if (q->doc && k == 0 && cc->doc_pipe)
                return launch_doc_pipe(cc->dense, cc->tpt0[0], q->a, cc->d_pipe_desc, (int)TT.batches[0].size(),
                                       cc->counters, TT.d_region, cc->dregion[0], cc->grid_pipe, cc->st);
            return launch_batch_phase(q->doc, cc->dense, k ? 16 : cc->tpt0[q->doc ? 0 : 1], q->a, TT.d_batches[k],
                                      (int)TT.batches[k].size(),
                                      cc->counters + 2 * k + (q->doc ? 0 : 1), TT.d_region,
                                      q->doc ? cc->dregion[k] : cc->region[k], cc->kbits,
                                      cc->grid_batch[q->doc ? 0 : 1][k], cc->st);
        }, &pc);
        if (rc) return rc;
    }
    for (int cls = 0; !doc && cls < kClusterClasses && !T.cluster_list.empty(); ++cls) {
        if (T.cluster_cls[cls + 1] == T.cluster_cls[cls]) continue;
        pc.cls = cls;
        rc = launch_rec(c, kcWordCluster, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            const Tier& W = cc->words;
            const int b0 = W.cluster_cls[q->cls], b1 = W.cluster_cls[q->cls + 1];
            return launch_cluster_word(q->a, W.d_cluster_list + b0, b1 - b0, 1 << q->cls, cc->cluster_T,
                                       cc->cluster_smem, cc->st);
        }, &pc);
        if (rc) return rc;
    }
    if (nch > 0) {
        rc = launch_rec(c, doc ? kcDocHugeAccept : kcWordMegaAccept, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            const HugeWork w = huge_work(cc, q->doc ? cc->docs : cc->words, kCtrAccept);
            const int grid = q->doc ? cc->grid_acc_doc : cc->grid_acc_word;
            if (cc->sparse) {
                const int k = q->doc ? 0 : 1;
                return launch_sparse_accept(q->doc, q->a, w, SparseRows{cc->d_soff[k], cc->sslots[k]},
                                            grid, cc->st);
            }
            return launch_huge_accept(q->doc, q->a, w, q->doc ? cc->rows_doc : cc->rows_pre, grid, cc->st);
        }, &pc);
        if (rc) return rc;
        if (!doc && !c->word_storage) {
            // the word draw takes its ranks from the post-acceptance counts
            rc = launch_rec(c, kcWordMegaHistPost, [](warplda_ctx* cc, void* p) {
                PhaseCall* q = (PhaseCall*)p;
                return launch_huge_hist(false, q->a, huge_work(cc, cc->words, kCtrHistPost),
                                        cc->rows_post, cc->grid_hist, cc->st);
            }, &pc);
            if (rc) return rc;
        }
        rc = launch_rec(c, doc ? kcDocHugeDraw : kcWordMegaDraw, [](warplda_ctx* cc, void* p) {
            PhaseCall* q = (PhaseCall*)p;
            return launch_huge_draw(q->doc, q->a, huge_work(cc, q->doc ? cc->docs : cc->words, kCtrDraw),
                                    q->doc ? cc->rows_doc : cc->rows_post, cc->grid_draw, cc->st);
        }, &pc);
        if (rc) return rc;
    }
    // c_k of the new assignments (per-block partials, one global pass;
    // Sec. 5.4), then the FP32 operands of the next phase
    if (!c->stage_ck && !c->ck_delta) {
        rc = launch_rec(c, kcCountCk, [](warplda_ctx* cc, void*) {
            return launch_topic_hist(cc->z, cc->N, cc->ck, cc->K, cc->grid_topic, cc->st);
        }, nullptr);
        if (rc) return rc;
    }
    rc = launch_rec(c, kcFinalize, [](warplda_ctx* cc, void*) {
        return launch_finalize_ck(cc->ck, cc->ckb, cc->K, cc->bbar, cc->counters, kCounters, cc->st);
    }, nullptr);
    if (rc) return rc;
    if (doc) {
        c->doc_done = 1;
    } else {
        c->doc_done = 0;
        c->iter = it;
    }
    return WARPLDA_OK;
}

int launches_per_phase(const warplda_ctx* c, bool doc) {
    const Tier& T = doc ? c->docs : c->words;
    int cl = 0;
    for (int k = 0; !doc && k < kClusterClasses && !T.cluster_list.empty(); ++k)
        cl += T.cluster_cls[k + 1] > T.cluster_cls[k] ? 1 : 0;
    return (T.s_chunks.empty() ? 0 : ((doc || c->word_storage) ? 4 : 5)) + cl +
           (T.batches[0].empty() ? 0 : 1) +
           (T.batches[1].empty() ? 0 : 1) + (T.warp_list.empty() ? 0 : 1) + ((c->stage_ck || c->ck_delta) ? 1 : 2);
}

int recount(warplda_ctx* c) {
    WL_CU(launch_topic_hist(c->z, c->N, c->ck, c->K, c->grid_topic, c->st), "topic histogram");
    WL_CU(launch_finalize_ck(c->ck, c->ckb, c->K, c->bbar, c->counters, kCounters, c->st), "finalize c_k");
    return WARPLDA_OK;
}

}  // namespace

int wl::record_error(int code, const char* msg) { return fail(code, "%s", msg); }

cudaError_t wl::launch_gate() {
    return inject_fires("WARPLDA_FAIL_LAUNCH", g_inject_launch) ? cudaErrorLaunchOutOfResources : cudaSuccess;
}
cudaError_t wl::alloc_gate() {
    return inject_fires("WARPLDA_FAIL_ALLOC", g_inject_alloc) ? cudaErrorMemoryAllocation : cudaSuccess;
}

// Device buffers of one fold-in call, freed on every return path.
// Buffers of one warplda_foldin call from the context's scratch: the call's
// i-th request takes slot i, which is reallocated (a quarter larger) only
// when too small, so repeated calls of similar size allocate nothing.
struct FoldScratch {
    warplda_ctx* c;
    size_t next = 0;
    template <typename T>
    cudaError_t get(T** out, int64_t n) {
        const size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
        if (next >= c->fold_ws.size()) c->fold_ws.resize(next + 1);
        auto& w = c->fold_ws[next++];
        if (w.bytes < bytes) {
            if (w.p) cudaFree(w.p);
            w.p = nullptr;
            w.bytes = 0;
            const size_t want = bytes + bytes / 4;
            const cudaError_t e = dev_malloc(&w.p, want);
            if (e != cudaSuccess) return e;
            w.bytes = want;
        }
        *out = static_cast<T*>(w.p);
        return cudaSuccess;
    }
};

struct FoldBuffers {
    std::vector<void*> p;
    template <typename T>
    cudaError_t get(T** out, int64_t n) {
        cudaError_t e = dev_malloc((void**)out, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) p.push_back(*out);
        return e;
    }
    ~FoldBuffers() {
        for (void* q : p) cudaFree(q);
    }
};

namespace {

int64_t enc_F(const warplda_ctx* c) { return (int64_t)1 << c->enc.log2F; }

// Forward pass of one batch (rows of b), logits into enc.logits; with
// dl_targets the softmax also writes the loss, dlogits and gb2 (targets
// given rows, or theta of the context's own assignments when tgt is null);
// q_out receives the proposal rows.
int enc_forward(warplda_ctx* c, const EncBatch& b, float* q_out, bool grads, const float* tgt) {
    auto& e = c->enc;
    WL_CU(launch_enc_l1_fwd(b, e.B, e.W1b, e.b1, e.H, e.log2F, e.h_pre, e.hb, e.hbT, c->st), "encoder layer 1");
    // the GEMM's status flag reuses the check record's last word
    WL_CU(launch_gemm_bf16(e.hb, e.W2tb, e.logits, e.b2, e.B, e.Kp, e.H, c->d_fault + 3, c->st, e.gwork,
                           e.gwork_floats),
          "encoder layer 2");
    WL_CU(launch_enc_softmax(b, e.B, e.logits, c->K, e.Kp, q_out, tgt, c->z, c->perm, c->alpha, c->abar,
                             grads ? e.dl : nullptr, e.dlT, e.gb2, e.loss, e.cnt, c->st), "encoder softmax");
    return WARPLDA_OK;
}

int enc_backward(warplda_ctx* c, const EncBatch& b) {
    auto& e = c->enc;
    WL_CU(launch_gemm_bf16(e.dl, e.W2nb, e.dH, nullptr, e.B, e.H, e.Kp, c->d_fault + 3, c->st, e.gwork,
                           e.gwork_floats),
          "encoder dH");
    WL_CU(launch_gemm_bf16(e.dlT, e.hbT, e.gW2t, nullptr, e.Kp, e.H, e.B, c->d_fault + 3, c->st, e.gwork,
                           e.gwork_floats),
          "encoder dW2");
    WL_CU(launch_enc_l1_bwd(b, e.B, e.dH, e.h_pre, e.H, e.log2F, e.gW1, e.gb1, c->st), "encoder layer 1 backward");
    return WARPLDA_OK;
}

int enc_zero_grads(warplda_ctx* c) {
    auto& e = c->enc;
    WL_CU(cudaMemsetAsync(e.gW1, 0, (size_t)enc_F(c) * e.H * 4, c->st), "zero gradients");
    WL_CU(cudaMemsetAsync(e.gb1, 0, (size_t)e.H * 4, c->st), "zero gradients");
    WL_CU(cudaMemsetAsync(e.gb2, 0, (size_t)e.Kp * 4, c->st), "zero gradients");
    return WARPLDA_OK;
}

int enc_adam_step(warplda_ctx* c, float lr) {
    auto& e = c->enc;
    e.step += 1;
    WL_CU(launch_enc_adam(e.W1, e.mW1, e.vW1, e.gW1, enc_F(c) * e.H, lr, e.step, e.W1b, c->st), "Adam W1");
    WL_CU(launch_enc_adam(e.b1, e.mb1, e.vb1, e.gb1, e.H, lr, e.step, nullptr, c->st), "Adam b1");
    WL_CU(launch_enc_adam(e.W2t, e.mW2, e.vW2, e.gW2t, (int64_t)e.Kp * e.H, lr, e.step, nullptr, c->st), "Adam W2");
    WL_CU(launch_enc_adam(e.b2, e.mb2, e.vb2, e.gb2, e.Kp, lr, e.step, nullptr, c->st), "Adam b2");
    WL_CU(launch_enc_w2_copies(e.W2t, e.Kp, e.H, e.W2tb, e.W2nb, c->st), "W2 copies");
    return WARPLDA_OK;
}

// Reads the GEMM status word (synchronises).
int enc_status(warplda_ctx* c) {
    int32_t h = 0;
    WL_CU(cudaMemcpyAsync(&h, c->d_fault + 3, 4, cudaMemcpyDeviceToHost, c->st), "read GEMM status");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    if (h) {
        WL_CU(cudaMemsetAsync(c->d_fault + 3, 0, 4, c->st), "clear GEMM status");
        return fail(WARPLDA_ETIMEDOUT, "encoder GEMM: a tensor-core wait ran out");
    }
    return WARPLDA_OK;
}

// Device copies of a host document CSR for encoder / fold-in calls.
struct HostDocs {
    int32_t *off = nullptr, *words = nullptr, *ids = nullptr;
};

int upload_docs(warplda_ctx* c, FoldBuffers& buf, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                HostDocs* out) {
    const int64_t Nn = doc_ptr[Dn];
    std::vector<int32_t> off((size_t)Dn + 1), ids((size_t)std::max<int64_t>(Dn, 1));
    for (int64_t d = 0; d <= Dn; ++d) off[d] = (int32_t)doc_ptr[d];
    for (int64_t d = 0; d < Dn; ++d) ids[d] = (int32_t)d;
    WL_CU(buf.get(&out->off, Dn + 1), "alloc offsets");
    WL_CU(buf.get(&out->words, Nn + 1), "alloc words");
    WL_CU(buf.get(&out->ids, Dn + 1), "alloc ids");
    WL_CU(cudaMemcpyAsync(out->off, off.data(), (size_t)(Dn + 1) * 4, cudaMemcpyHostToDevice, c->st), "upload offsets");
    if (Nn > 0)
        WL_CU(cudaMemcpyAsync(out->words, doc_word, (size_t)Nn * 4, cudaMemcpyHostToDevice, c->st), "upload words");
    if (Dn > 0)
        WL_CU(cudaMemcpyAsync(out->ids, ids.data(), (size_t)Dn * 4, cudaMemcpyHostToDevice, c->st), "upload ids");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");   // the host vectors go out of scope
    return WARPLDA_OK;
}

// First position of a word id outside [0, V), or -1.  The scan is a
// branch-free OR over blocks of ids (one unsigned compare each, which the
// compiler vectorises); the position is searched only in a bad block.
int64_t first_bad_word(const int32_t* w, int64_t n, int64_t V) {
    const uint32_t v = (uint32_t)std::min<int64_t>(V, 0x7FFFFFFF);
    constexpr int64_t kBlock = 4096;
    for (int64_t b = 0; b < n; b += kBlock) {
        const int64_t e = std::min(n, b + kBlock);
        uint32_t bad = 0;
        for (int64_t p = b; p < e; ++p) bad |= (uint32_t)((uint32_t)w[p] >= v);
        if (bad)
            for (int64_t p = b; p < e; ++p)
                if ((uint32_t)w[p] >= v) return p;
    }
    return -1;
}

int check_docs(const warplda_ctx* c, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word) {
    if (Dn < 0 || !doc_ptr || doc_ptr[0] != 0) return fail(WARPLDA_EINVAL, "bad document CSR");
    for (int64_t d = 0; d < Dn; ++d)
        if (doc_ptr[d + 1] < doc_ptr[d]) return fail(WARPLDA_EINVAL, "doc_ptr decreases at %lld", (long long)d);
    const int64_t Nn = doc_ptr[Dn];
    if (Nn > (int64_t)0x7FFFFFF0) return fail(WARPLDA_EINVAL, "too many tokens");
    if (Nn > 0 && !doc_word) return fail(WARPLDA_EINVAL, "null doc_word");
    const int64_t p = first_bad_word(doc_word, Nn, c->V);
    if (p >= 0) return fail(WARPLDA_EINVAL, "word id %d at %lld outside [0, V)", doc_word[p], (long long)p);
    return WARPLDA_OK;
}

// Proposal rows q[Dn, K] of host documents (device output).
int enc_proposal_dev(warplda_ctx* c, int64_t Dn, const HostDocs& hd, float* q_dev) {
    auto& e = c->enc;
    for (int64_t b0 = 0; b0 < Dn; b0 += e.B) {
        EncBatch b{hd.ids + b0, hd.off, hd.words, (int)std::min<int64_t>(e.B, Dn - b0)};
        int rc = enc_forward(c, b, q_dev + b0 * c->K, false, nullptr);
        if (rc) return rc;
    }
    return enc_status(c);
}

// Builds the fold-in model of the current state if it is stale.
int ensure_model(warplda_ctx* c) {
    if (c->model_iter == (int64_t)c->iter) return WARPLDA_OK;
    const int K = c->K;
    int rc;
    if (!c->model_cw && (rc = dalloc(c, &c->model_cw, c->V * (int64_t)K, "alloc fold-in model"))) return rc;
    if (!c->model_zs && (rc = dalloc(c, &c->model_zs, c->N + 4, "alloc fold-in topics"))) return rc;
    if (!c->model_ckb && (rc = dalloc(c, &c->model_ckb, K, "alloc fold-in c_k"))) return rc;
    WL_CU(launch_model_build(c->z, c->word_off, c->V, K, c->model_cw, c->model_zs, c->d_fault, 4 * c->sms,
                             c->st), "build fold-in model");
    WL_CU(cudaMemcpyAsync(c->model_ckb, c->ckb, (size_t)K * sizeof(float), cudaMemcpyDeviceToDevice, c->st),
          "copy c_k");
    c->model_iter = c->iter;
    return WARPLDA_OK;
}

}  // namespace


// ---------------------------------------------------------------------------
// Serving: continuous batching of fold-in requests.
// ---------------------------------------------------------------------------
struct warplda_server {
    warplda_ctx* c = nullptr;
    int nslots = 0, sweeps = 0, proposal = 0, max_tokens = 0, tab_words = 0, grid = 1;
    int64_t pool_tokens = 0;
    uint64_t seed = 0;
    int4* d_info = nullptr;
    int32_t *d_active = nullptr, *d_z = nullptr, *d_prop = nullptr, *d_words = nullptr, *d_counter = nullptr;
    float *d_fin_theta = nullptr, *d_q = nullptr;
    int32_t* d_fin_slot = nullptr;
    int2* d_atab = nullptr;         // learned proposal: each slot's alias table
    int32_t* d_staged = nullptr;   // words of requests admitted since the last step
    int4* d_req = nullptr;          // their {slot, pool offset, L, id}
    int32_t* d_src = nullptr;       // their offsets in the staged words
    int64_t staged_cap = 0;
    float* h_theta = nullptr;       // pinned: finished rows of the last step
    int32_t* h_fin_slot = nullptr;
    int32_t* h_stage = nullptr;     // pinned upload staging: words, then requests, sources, active list
    int64_t h_stage_cap = 0;
    // learned proposal: admission scratch for up to nslots new requests
    float* d_aq = nullptr;
    int2* d_aatab = nullptr;
    int n_fin_staged = 0;
    cudaEvent_t tick = nullptr;
    // learned proposal: the admission work (encoder, alias tables, rows) of
    // a step, and with few sweeps per request its new requests' first sweep,
    // run on a second stream while the step's sweep of the running requests
    // runs
    cudaStream_t side = nullptr;
    cudaEvent_t uploaded = nullptr, admitted = nullptr;
    struct Slot {
        bool used = false;
        int64_t id = 0;
        int32_t off = 0, L = 0, done = 0;
    };
    std::vector<Slot> slots;
    std::vector<int32_t> free_slots;
    std::map<int64_t, int64_t> free_ranges;   // pool start -> length
    // admitted since the last step
    std::vector<int32_t> new_words, new_src;
    std::vector<int4> new_req;
    std::vector<int64_t> new_ptr{0};
    std::vector<void*> allocs;
};

namespace {

// First fit in the token pool; -1 if no free range is long enough.
int64_t pool_take(warplda_server* s, int64_t n) {
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second < n) continue;
        const int64_t start = it->first, len = it->second;
        s->free_ranges.erase(it);
        if (len > n) s->free_ranges[start + n] = len - n;
        return start;
    }
    return -1;
}

void pool_give(warplda_server* s, int64_t start, int64_t n) {
    if (n <= 0) return;
    auto it = s->free_ranges.emplace(start, n).first;
    auto nx = std::next(it);
    if (nx != s->free_ranges.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_ranges.erase(nx);
    }
    if (it != s->free_ranges.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_ranges.erase(it);
        }
    }
}

template <typename T>
int salloc(warplda_server* s, T** p, int64_t n) {
    cudaError_t e = dev_malloc((void**)p, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "alloc server");
    s->allocs.push_back(*p);
    return WARPLDA_OK;
}

void server_free(warplda_server* s) {
    for (void* p : s->allocs) cudaFree(p);
    s->allocs.clear();
    if (s->h_theta) cudaFreeHost(s->h_theta);
    if (s->h_fin_slot) cudaFreeHost(s->h_fin_slot);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->tick) cudaEventDestroy(s->tick);
    if (s->uploaded) cudaEventDestroy(s->uploaded);
    if (s->admitted) cudaEventDestroy(s->admitted);
    if (s->side) cudaStreamDestroy(s->side);
}

FoldArgs server_args(warplda_server* s) {
    warplda_ctx* c = s->c;
    FoldArgs f{};
    f.Cw = c->model_cw;
    f.Zs = c->model_zs;
    f.word_off = c->word_off;
    f.ckb = c->model_ckb;
    f.counter = s->d_counter;
    f.fault = c->d_fault;
    f.K = c->K;
    f.M = c->M;
    f.V = (int)c->V;
    f.sweeps = s->sweeps;
    f.Lmax = s->max_tokens;
    f.alpha = c->alpha;
    f.abar = c->abar;
    f.beta = c->beta;
    f.kbeta = c->kbeta;
    f.rk = round_keys(s->seed);
    return f;
}

// Pinned staging of at least n ints.
int stage_room(warplda_server* s, int64_t n) {
    if (n <= s->h_stage_cap) return WARPLDA_OK;
    if (s->h_stage) cudaFreeHost(s->h_stage);
    s->h_stage = nullptr;
    const int64_t cap = std::max<int64_t>(n, 2 * s->h_stage_cap);
    if (host_malloc((void**)&s->h_stage, (size_t)cap * 4) != cudaSuccess) {
        s->h_stage_cap = 0;
        return fail(WARPLDA_ENOMEM, "pinned staging");
    }
    s->h_stage_cap = cap;
    return WARPLDA_OK;
}

// Uploads the requests admitted since the last step (one copy from pinned
// staging, one admission kernel) and, with the learned proposal, makes their
// proposal rows and alias tables -- all queued on the stream, no host wait.
// The staging also carries the step's active list (written at `act_off`).
int server_admit(warplda_server* s, const std::vector<int32_t>& active, int64_t* act_off, int64_t* sl_off) {
    warplda_ctx* c = s->c;
    const int n = (int)s->new_req.size();
    const int64_t nw = (int64_t)s->new_words.size();
    // layout: words | req (4 ints each) | src | offsets (n+1) | ids | slots | active
    // (the int4 descriptors start 16-byte aligned)
    const int64_t o_req = r4(nw), o_src = o_req + 4 * (int64_t)n, o_off = o_src + n, o_ids = o_off + n + 1,
                  o_sl = o_ids + n, o_act = o_sl + n, total = o_act + (int64_t)active.size();
    int rc = stage_room(s, total + 4);
    if (rc) return rc;
    if (total + 4 > s->staged_cap) {
        int64_t cap = std::max<int64_t>(total + 4, 2 * s->staged_cap);
        int32_t* p = nullptr;
        WL_CU(dev_malloc((void**)&p, (size_t)cap * 4), "alloc staging");
        s->allocs.push_back(p);
        s->d_staged = p;
        s->staged_cap = cap;
    }
    int32_t* h = s->h_stage;
    if (nw) std::memcpy(h, s->new_words.data(), (size_t)nw * 4);
    if (n) std::memcpy(h + o_req, s->new_req.data(), (size_t)n * sizeof(int4));
    for (int i = 0; i < n; ++i) {
        h[o_src + i] = s->new_src[i];
        h[o_ids + i] = i;
        h[o_sl + i] = s->new_req[i].x;
    }
    for (int i = 0; i <= n; ++i) h[o_off + i] = (int32_t)s->new_ptr[i];
    if (!active.empty()) std::memcpy(h + o_act, active.data(), active.size() * 4);
    WL_CU(cudaMemcpyAsync(s->d_staged, h, (size_t)total * 4, cudaMemcpyHostToDevice, c->st), "upload requests");
    *act_off = o_act;
    *sl_off = o_sl;
    const int32_t* d = s->d_staged;
    if (n > 0) {
        rc = launch_timed(c, kcServeAdmit, [&] {
            return launch_serve_admit(d, reinterpret_cast<const int4*>(d + o_req), d + o_src, n, s->nslots,
                                      s->pool_tokens, s->d_words, s->d_info, c->st);
        });
        if (rc) return rc;
    }
    if (n > 0 && s->proposal == WARPLDA_PROPOSAL_LEARNED) {
        // on the side stream, once the upload is done; the caller queues the
        // new requests' first sweep behind it there and makes the main stream
        // wait for `admitted` after the running requests' sweep is queued
        const int K = c->K;
        auto& e = c->enc;
        WL_CU(cudaEventRecord(s->uploaded, c->st), "record upload");
        WL_CU(cudaStreamWaitEvent(s->side, s->uploaded, 0), "wait upload");
        cudaStream_t main_st = c->st;
        c->st = s->side;   // enc_forward queues on the context's stream
        for (int b0 = 0; b0 < n && !rc; b0 += e.B) {
            EncBatch b{d + o_ids + b0, d + o_off, d, std::min(e.B, n - b0)};
            cudaEvent_t ea = nullptr, eb = nullptr;
            if (c->prof) {
                if (cudaEventCreate(&ea) != cudaSuccess) ea = nullptr;
                if (ea && cudaEventCreate(&eb) != cudaSuccess) {
                    cudaEventDestroy(ea);
                    ea = eb = nullptr;
                }
                if (ea) cudaEventRecord(ea, c->st);
            }
            rc = enc_forward(c, b, s->d_aq + (int64_t)b0 * K, false, nullptr);
            if (ea) {
                cudaEventRecord(eb, c->st);
                c->recs.push_back(Rec{kcServeEncoder, ea, eb});
            }
        }
        c->st = main_st;
        if (rc) return rc;
        if ((rc = launch_timed(c, kcServeAlias, [&] { return launch_enc_alias(s->d_aq, n, K, s->d_aatab, s->side); },
                               s->side)))
            return rc;
        rc = launch_timed(c, kcServeRows, [&] {
            const cudaError_t e1 = launch_serve_rows(s->d_aq, d + o_sl, n, K, s->nslots, s->d_q, s->side);
            return e1 != cudaSuccess ? e1 : launch_serve_rows(s->d_aatab, d + o_sl, n, 2 * K, s->nslots, s->d_atab, s->side);
        }, s->side);
        if (rc) return rc;
    }
    s->new_words.clear();
    s->new_src.clear();
    s->new_req.clear();
    s->new_ptr.assign(1, 0);
    return WARPLDA_OK;
}

// WARPLDA_TRACE_INIT=1: warplda_init waits for the stream at each stage
// boundary and prints the stage's wall time to stderr (diagnostics; the
// waits serialise what init otherwise overlaps).
struct InitTrace {
    bool on = false;
    cudaStream_t st = nullptr;
    std::chrono::steady_clock::time_point t0, last;
    void start(cudaStream_t s) {
        const char* v = std::getenv("WARPLDA_TRACE_INIT");
        on = v && v[0] == '1';
        st = s;
        t0 = last = std::chrono::steady_clock::now();
    }
    void mark(const char* stage) {
        if (!on) return;
        cudaStreamSynchronize(st);
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "warplda_init %-34s %9.2f ms  (at %9.2f ms)\n", stage,
                     std::chrono::duration<double, std::milli>(now - last).count(),
                     std::chrono::duration<double, std::milli>(now - t0).count());
        last = now;
    }
};

}  // namespace

extern "C" {

const char* warplda_last_error(void) { return g_err.c_str(); }

int warplda_init(warplda_ctx** out, int64_t D, int64_t V, int64_t N, const int64_t* doc_ptr,
                 const int32_t* doc_word, int32_t K, float alpha, float beta, int32_t M,
                 uint64_t seed, void* cuda_stream, const warplda_tuning* tuning) try {
    if (!out) return fail(WARPLDA_EINVAL, "out is NULL");
    *out = nullptr;
    InitTrace trace;
    trace.start((cudaStream_t)cuda_stream);
    if (D < 0 || V < 1) return fail(WARPLDA_EINVAL, "need D >= 0 and V >= 1");
    if (N < 0 || N > (int64_t)0x7FFFFFF0) return fail(WARPLDA_EINVAL, "N must be in [0, 2^31 - 16]");
    if (V > (int64_t)0x7FFFFFF0 || D > (int64_t)0x7FFFFFF0) return fail(WARPLDA_EINVAL, "D, V too large");
    if (K < 1 || K > kMaxTopics) return fail(WARPLDA_EINVAL, "K must be in [1, %d]", kMaxTopics);
    if (M < 1 || M > 4) return fail(WARPLDA_EINVAL, "M must be in [1, 4]");
    if (!(alpha > 0.0f) || !std::isfinite(alpha)) return fail(WARPLDA_EINVAL, "alpha must be > 0");
    if (!(beta > 0.0f) || !std::isfinite(beta)) return fail(WARPLDA_EINVAL, "beta must be > 0");
    if (!doc_ptr || (N > 0 && !doc_word)) return fail(WARPLDA_EINVAL, "null corpus pointer");
    if (doc_ptr[0] != 0 || doc_ptr[D] != N) return fail(WARPLDA_EINVAL, "doc_ptr must run from 0 to N");
    for (int64_t d = 0; d < D; ++d)
        if (doc_ptr[d + 1] < doc_ptr[d]) return fail(WARPLDA_EINVAL, "doc_ptr decreases at %lld", (long long)d);
    trace.mark("argument and CSR checks");
    warplda_ctx* c = new warplda_ctx();
    auto undo = on_exit([&] {
        free_all(c);
        delete c;
    });
    c->D = D; c->V = V; c->N = N; c->K = K; c->M = M;
    c->alpha = alpha; c->beta = beta;
    c->abar = (float)K * alpha;   // one FP32 product each
    c->bbar = (float)V * beta;
    c->kbeta = (float)K * beta;
    c->seed = seed;
    c->k0 = (uint32_t)seed;
    c->k1 = (uint32_t)(seed >> 32);
    c->st = (cudaStream_t)cuda_stream;
    {
        const char* sc = std::getenv("WARPLDA_SYNC_CHECK");
        c->sync_check = sc && sc[0] == '1';
    }
    c->dense = K <= kDenseMaxK;
    // dense tables: c_k is staged in shared memory and kept by per-block
    // deltas; larger K: a histogram pass after each phase rebuilds c_k
    c->stage_ck = c->dense ? 1 : 0;
    while ((1 << c->kbits) < K) ++c->kbits;
    // block batches: up to 2045 tokens with 8 tokens per thread, up to 4093
    // with 16; the table budget of a batch is region_budget words (defaults
    // 4096 and 8192)
    const int bmax = (tuning && tuning->batch_max_tokens > 0) ? tuning->batch_max_tokens : kMaxBatchTokens;
    c->chunk = (tuning && tuning->huge_chunk > 0) ? tuning->huge_chunk : (1 << 30);
    const int rb = (tuning && tuning->region_budget > 0) ? ((tuning->region_budget + 3) & ~3) : 0;
    c->bmax[0] = std::min(bmax, kThreads * 8 - 3);
    c->bmax[1] = std::min(bmax, std::min(kMaxBatchTokens, kThreads * 16 - 3));
    c->tpt0[0] = (K > kDenseMaxK) ? 4 : 8;
    c->tpt0[1] = 8;
    c->dbmax[0] = std::min(bmax, kThreads * c->tpt0[0] - 3);
    c->dbmax[1] = c->bmax[1];
    c->region[0] = rb ? rb : 8192;
    c->region[1] = rb ? rb : 8192;
    // the pipelined document kernel takes batches of up to 1021 tokens and
    // 128 documents; their hash tables need at most 4 words per token
    if (tuning && tuning->cluster_max_tokens < -1) {
        return fail(WARPLDA_EINVAL, "cluster_max_tokens must be -1, 0 or positive");
    }
    if (tuning && (tuning->doc_batch_kernel < 0 || tuning->doc_batch_kernel > 2)) {
        return fail(WARPLDA_EINVAL, "doc_batch_kernel must be 0, 1 or 2");
    }
    if (tuning && (tuning->foldin_kernel < 0 || tuning->foldin_kernel > 2)) {
        return fail(WARPLDA_EINVAL, "foldin_kernel must be 0, 1 or 2");
    }
    c->foldin_word_major = !tuning || tuning->foldin_kernel != 1;
    {
        // measured: pipelined batches of 1021 tokens beat the block kernel
        // with hash tables and K up to 16384; with dense tables the block
        // kernel's 2045-token batches share more gather sectors, and with
        // sparse rows (c_k in L2) its grouped operand loads, and it wins
        const int dk = tuning ? tuning->doc_batch_kernel : 0;
        c->doc_pipe = dk == 2 || (dk == 0 && !c->dense && K <= kDenseRowMaxK);
    }
    if (c->doc_pipe) {
        c->dbmax[0] = std::min(bmax, kPipeTokens);
        c->tpt0[0] = c->dbmax[0] + 3 <= 2 * kThreads ? 2 : 4;
    }
    c->dregion[0] = rb ? rb : (c->doc_pipe ? (c->tpt0[0] == 2 ? 2048 : 4096) : 8192);
    c->dregion[1] = c->region[1];
    // documents of up to 32 * warp_tpl tokens go to the warp tier; the
    // block tier takes the rest (its small class is not used for documents)
    c->warp_tpl = c->dense ? 16 : 8;
    // the warp tier is off unless asked for: all documents in one kernel keep
    // the doc-order sweep over the word columns that makes the perm gather
    // hit L2 (Sec. 5.2)
    int warp_max = 0;
    if (tuning && (tuning->word_positioning < 0 || tuning->word_positioning > 1)) {
        return fail(WARPLDA_EINVAL, "word_positioning must be 0 or 1");
    }
    c->word_storage = (tuning && tuning->word_positioning == 1) ? 1 : 0;
    c->sparse = K > kDenseRowMaxK;
    if (c->sparse) c->word_storage = 1;   // ranks need sorted rows; sparse rows use positioning
    // with 10^5..10^6 topics the deltas' global atomics rarely collide and
    // touch only the tokens that change; the histogram pass touches all
    c->ck_delta = c->sparse ? 1 : 0;
    if (tuning && tuning->doc_warp_max > 0)
        warp_max = std::min(std::min(32 * c->warp_tpl, bmax), (int)tuning->doc_warp_max);

    auto bail = [](int rc) { return rc; };   // `undo` frees the context
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));

    // token arrays first: the word-major order is built on the device in them
    int rc;
    if ((rc = dalloc(c, &c->z, N + 4, "alloc z"))) return bail(rc);
    if ((rc = dalloc(c, &c->sperm, N + 4, "alloc sorted perm"))) return bail(rc);
    if ((rc = dalloc(c, &c->sinfo, N + 4, "alloc sorted info"))) return bail(rc);
    if ((rc = dalloc(c, &c->prop, (N + 4) * M, "alloc proposals"))) return bail(rc);
    if ((rc = dalloc(c, &c->perm, N + 4, "alloc perm"))) return bail(rc);
    if ((rc = dalloc(c, &c->doc_off, D + 1, "alloc doc offsets"))) return bail(rc);
    if ((rc = dalloc(c, &c->word_off, V + 1, "alloc word offsets"))) return bail(rc);
    if ((rc = dalloc(c, &c->d_bad, 2, "alloc flag"))) return bail(rc);
    trace.mark("token array allocation");
    // word ids go where pass 0 of the word sort reads them, so that the last
    // pass leaves the positions in prop (z and prop are rewritten at the end)
    const bool odd = token_sort_passes(V) % 2 == 1;
    int32_t* ka = odd ? c->sperm : c->z;
    int32_t* va = odd ? reinterpret_cast<int32_t*>(c->sinfo) : c->prop;
    int32_t* kb = odd ? c->z : c->sperm;
    int32_t* vb = odd ? c->prop : reinterpret_cast<int32_t*>(c->sinfo);
    std::vector<int32_t> doc_off(D + 1), word_off(V + 1);
    for (int64_t d = 0; d <= D; ++d) doc_off[d] = (int32_t)doc_ptr[d];
    // dense rows live in shared memory: a few ranges per block slot, each
    // long enough that its row load is a small part of it.
    // Sparse rows live in global memory: ranges of ~4K tokens taken in
    // order keep the rows that the resident blocks touch at once few enough
    // to stay in L2.
    const int ranges_target = c->sparse ? (1 << 30) : kRangesPerSm * c->sms;
    // word-major order (Sec. 5.2): the word ids are checked, then a stable
    // sort of the tokens by word leaves the doc-major positions in prop and
    // the sorted ids in z; each word's first index gives the word offsets
    int32_t* pos = nullptr;
    {
        std::vector<int32_t> wstart((size_t)V, -1);
        const int32_t init_bad[2] = {0x7FFFFFFF, 0x7FFFFFFF};
        int32_t bad[2];
        int32_t* scratch = nullptr;
        int32_t* keys = nullptr;
        if (N > 0 && (e = cudaMemcpyAsync(ka, doc_word, (size_t)N * 4, cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
            return bail(cuda_fail(e, "upload word ids"));
        trace.mark("upload of the word ids");
        if ((e = cudaMemcpyAsync(c->d_bad, init_bad, sizeof(init_bad), cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
            return bail(cuda_fail(e, "upload flag"));
        e = launch_word_check(ka, N, (int32_t)V, c->d_bad, c->st);
        // the sort's tile counters (~N/16 words) live in perm, which is only
        // written from the sorted positions afterwards; tiny corpora allocate
        const bool own_scratch = token_sort_scratch(N) > N + 4;
        if (!own_scratch) scratch = c->perm;
        else if (e == cudaSuccess) e = dev_malloc((void**)&scratch, (size_t)token_sort_scratch(N) * 4);
        if (e == cudaSuccess) e = launch_token_sort(ka, va, kb, vb, N, (int32_t)V, scratch, &pos, &keys, c->st);
        if (e == cudaSuccess && N > 0 && (pos != c->prop || keys != c->z)) e = cudaErrorInvalidValue;   // by the parity above
        trace.mark("word check and word sort");
        if (e == cudaSuccess) e = launch_word_starts(keys, N, (int32_t)V, c->word_off, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(wstart.data(), c->word_off, (size_t)V * 4, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, c->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->st);
        // the document tier needs only the document offsets: the host builds
        // it while the word ids upload and sort
        if (e == cudaSuccess)
            build_tier(doc_off, D, K, c->dense, warp_max, c->dbmax, c->dregion, c->chunk, ranges_target, &c->docs,
                       c->doc_pipe ? kDocSegs : kSegsMax);
        trace.mark("word starts; document tier (host)");
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (own_scratch && scratch) cudaFree(scratch);
        if (e != cudaSuccess) return bail(cuda_fail(e, "token order sort"));
        if (bad[0] != 0x7FFFFFFF)
            return bail(fail(WARPLDA_EINVAL, "word id %d at %lld outside [0, V)", doc_word[bad[0]], (long long)bad[0]));
        // words without tokens start where the next word does
        c->word_ptr_h.assign(V + 1, N);
        for (int64_t w = V - 1; w >= 0; --w) c->word_ptr_h[w] = wstart[w] >= 0 ? wstart[w] : c->word_ptr_h[w + 1];
    }
    for (int64_t w = 0; w <= V; ++w) word_off[w] = (int32_t)c->word_ptr_h[w];
    // with tuning cluster_max_tokens, words too long for a block batch but
    // within a cluster's shared memory (or the cap) are sampled on a
    // thread-block cluster (up to 16 blocks where the device allows, else 8).
    // Off by default: measured slower than the multi-pass tier on the
    // PubMed- and NYTimes-shaped workloads (8.4 vs 7.3 ms and 1.1 vs 0.7 ms
    // per sweep for the same words)
    int64_t cluster_max = 0;
    {
        const int ct = tuning ? tuning->cluster_max_tokens : 0;
        int optin = 0;
        if (!c->sparse && ct != 0 &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev) == cudaSuccess) {
            const int smem = (optin - 1024) & ~15;   // room for the kernel's static shared memory
            for (int C : {16, 8}) {
                if (cluster_size_supported(K, M, c->stage_ck, C, smem) >= 1) {
                    c->cluster_C = C;
                    c->cluster_smem = smem;
                    c->cluster_T = cluster_slice_capacity(K, M, c->stage_ck, smem);
                    break;
                }
            }
            if (c->cluster_C > 0 && c->cluster_T > 0) {
                cluster_max = (int64_t)c->cluster_C * c->cluster_T;
                if (ct > 0) cluster_max = std::min<int64_t>(cluster_max, ct);
            }
        }
    }
    build_tier(word_off, V, K, c->dense, 0, c->bmax, c->region, c->chunk, ranges_target, &c->words, kSegsMax,
               cluster_max, std::max(1, c->cluster_T));

    trace.mark("word tier (host)");
    if ((rc = dalloc(c, &c->ck, K, "alloc c_k"))) return bail(rc);
    if ((rc = dalloc(c, &c->ckb, K, "alloc c_k float"))) return bail(rc);
    if ((rc = dalloc(c, &c->counters, kCounters, "alloc counters"))) return bail(rc);
    if ((rc = dalloc(c, &c->d_ll, 1, "alloc loglik"))) return bail(rc);
    if ((rc = dalloc(c, &c->d_fault, 4, "alloc check record"))) return bail(rc);
    // count rows of the multi-pass tier; each row set starts 16-byte aligned
    // and is zeroed in whole int4 units
    const int64_t rd = c->sparse ? 0 : r4(c->docs.nrows * (int64_t)K);
    const int64_t rw = c->sparse ? 0 : r4(c->words.nrows * (int64_t)K);
    c->rows_words = rd + 2 * rw + 4;
    if ((rc = dalloc(c, &c->rows, c->rows_words, "alloc count rows"))) return bail(rc);
    c->rows_doc = c->rows;
    c->rows_pre = c->rows + rd;
    c->rows_post = c->rows_pre + rw;
    if (c->sparse) {
        for (int k = 0; k < 2; ++k) {
            const Tier& T = k ? c->words : c->docs;
            std::vector<int64_t> off(T.row_len.size() + 1, 0);
            for (size_t r = 0; r < T.row_len.size(); ++r)
                off[r + 1] = off[r] + (int64_t)pow2_above((uint32_t)std::min(2 * T.row_len[r], K));
            c->sn[k] = off.back();
            if ((rc = dalloc(c, &c->d_soff[k], (int64_t)off.size(), "alloc sparse rows"))) return bail(rc);
            if ((rc = dalloc(c, &c->sslots[k], c->sn[k] + 2, "alloc sparse rows"))) return bail(rc);
            if ((e = cudaMemcpyAsync(c->d_soff[k], off.data(), off.size() * 8, cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload sparse rows"));
            if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess)   // `off` goes out of scope
                return bail(cuda_fail(e, "synchronize"));
        }
    }
    for (Tier* t : {&c->docs, &c->words}) {
        for (int k = 0; k < 2; ++k) {
            if ((rc = dalloc(c, &t->d_batches[k], (int64_t)t->batches[k].size(), "alloc batches"))) return bail(rc);
            if (!t->batches[k].empty())
                if ((e = cudaMemcpyAsync(t->d_batches[k], t->batches[k].data(), t->batches[k].size() * sizeof(int4),
                                         cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                    return bail(cuda_fail(e, "upload batches"));
        }
        if ((rc = dalloc(c, &t->d_warp_list, (int64_t)t->warp_list.size(), "alloc warp list"))) return bail(rc);
        if (!t->warp_list.empty())
            if ((e = cudaMemcpyAsync(t->d_warp_list, t->warp_list.data(), t->warp_list.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload warp list"));
        if ((rc = dalloc(c, &t->d_ll_batches, (int64_t)t->ll_batches.size(), "alloc ll batches"))) return bail(rc);
        if (!t->ll_batches.empty())
            if ((e = cudaMemcpyAsync(t->d_ll_batches, t->ll_batches.data(), t->ll_batches.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload ll batches"));
        if ((rc = dalloc(c, &t->d_region, (int64_t)t->region.size(), "alloc table offsets"))) return bail(rc);
        if ((e = cudaMemcpyAsync(t->d_region, t->region.data(), t->region.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
            return bail(cuda_fail(e, "upload table offsets"));
        if ((rc = dalloc(c, &t->d_chunks, (int64_t)t->chunks.size(), "alloc chunks"))) return bail(rc);
        if (!t->chunks.empty())
            if ((e = cudaMemcpyAsync(t->d_chunks, t->chunks.data(), t->chunks.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload chunks"));
        if ((rc = dalloc(c, &t->d_range_off, (int64_t)t->range_off.size(), "alloc ranges"))) return bail(rc);
        if (!t->range_off.empty())
            if ((e = cudaMemcpyAsync(t->d_range_off, t->range_off.data(), t->range_off.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload ranges"));
        if ((rc = dalloc(c, &t->d_s_chunks, (int64_t)t->s_chunks.size(), "alloc chunks"))) return bail(rc);
        if (!t->s_chunks.empty())
            if ((e = cudaMemcpyAsync(t->d_s_chunks, t->s_chunks.data(), t->s_chunks.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload chunks"));
        if ((rc = dalloc(c, &t->d_s_range_off, (int64_t)t->s_range_off.size(), "alloc ranges"))) return bail(rc);
        if (!t->s_range_off.empty())
            if ((e = cudaMemcpyAsync(t->d_s_range_off, t->s_range_off.data(), t->s_range_off.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload ranges"));
        if ((rc = dalloc(c, &t->d_cluster_list, (int64_t)t->cluster_list.size(), "alloc cluster words"))) return bail(rc);
        if (!t->cluster_list.empty())
            if ((e = cudaMemcpyAsync(t->d_cluster_list, t->cluster_list.data(), t->cluster_list.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
                return bail(cuda_fail(e, "upload cluster words"));
    }
    {
        // descriptors of the pipelined document batches: {first document,
        // documents | table words << 16, first token, tokens}
        const auto& B = c->docs.batches[0];
        std::vector<int4> desc(B.size());
        for (size_t i = 0; i < B.size(); ++i)
            desc[i] = make_int4(B[i].x, (B[i].y - B[i].x) | (B[i].z << 16), doc_off[B[i].x],
                                doc_off[B[i].y] - doc_off[B[i].x]);
        if ((rc = dalloc(c, &c->d_pipe_desc, (int64_t)desc.size(), "alloc batch descriptors"))) return bail(rc);
        if (!desc.empty()) {
            if ((e = cudaMemcpyAsync(c->d_pipe_desc, desc.data(), desc.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(c->st)) != cudaSuccess)   // `desc` goes out of scope
                return bail(cuda_fail(e, "upload batch descriptors"));
        }
    }
    trace.mark("count rows, tier uploads, descriptors");
    if ((e = cudaMemcpyAsync(c->doc_off, doc_off.data(), (D + 1) * 4, cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
        return bail(cuda_fail(e, "upload doc offsets"));
    if ((e = cudaMemcpyAsync(c->word_off, word_off.data(), (V + 1) * 4, cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
        return bail(cuda_fail(e, "upload word offsets"));
    // perm from the sorted positions, then each document batch's tokens in
    // word-major order
    {
        e = launch_perm(pos, N, c->perm, c->st);
        // padding past N is zero, as every array's tail is
        trace.mark("perm");
        if (e == cudaSuccess) e = cudaMemsetAsync(c->perm + N, 0, 4 * 4, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->sperm, 0, ((size_t)N + 4) * 4, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->sinfo, 0, ((size_t)N + 4) * 4, c->st);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            e = launch_batch_lists(c->docs.d_batches[k], (int)c->docs.batches[k].size(), c->dbmax[k], c->doc_off,
                                   c->perm, pos, N,
                                   c->sperm, c->sinfo, c->d_bad + 1, c->st);
        int32_t bad2 = 0x7FFFFFFF;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad2, c->d_bad + 1, 4, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "token order build"));
        if (bad2 != 0x7FFFFFFF) return bail(fail(WARPLDA_EINVAL, "document batch %d malformed", bad2));
        trace.mark("document batches' word-major lists");
    }

    // grids: persistent blocks, as many as fit
    auto fit = [&](int per_sm) { return std::max(1, per_sm) * c->sms; };
    for (int w = 0; w < 2; ++w)
        for (int k = 0; k < 2; ++k) {
            const int64_t nb = (int64_t)(w ? c->words : c->docs).batches[k].size();
            const int rw = w ? c->region[k] : c->dregion[k];
            if (w == 0 && k == 0 && c->doc_pipe) {
                const int per_sm = docpipe_blocks_per_sm(K, c->dense ? 1 : 0, rw, c->tpt0[0], M);
                if (per_sm < 1)
                    return bail(fail(WARPLDA_EINVAL, "document batch kernel does not fit (region_budget too large?)"));
                c->grid_pipe = (int)std::min<int64_t>(fit(per_sm), std::max<int64_t>(1, nb));
                continue;
            }
            const int per_sm = batch_blocks_per_sm(K, c->stage_ck, rw, k ? 16 : c->tpt0[w], w, M, c->dense);
            if (per_sm < 1)
                return bail(fail(WARPLDA_EINVAL, "batch kernel does not fit (region_budget too large?)"));
            c->grid_batch[w][k] = (int)std::min<int64_t>(fit(per_sm), std::max<int64_t>(1, nb));
        }
    {
        const int per_sm = docwarp_blocks_per_sm(K, c->stage_ck, c->warp_tpl, M, c->dense);
        if (per_sm < 1) return bail(fail(WARPLDA_EINVAL, "document warp kernel does not fit"));
        const int64_t need = ((int64_t)c->docs.warp_list.size() + kWarps - 1) / kWarps;
        c->grid_doc_warp = (int)std::min<int64_t>(fit(per_sm), std::max<int64_t>(1, need));
    }
    if (c->sparse) {
        // no shared-memory rows: blocks of 256 threads, as many as fit
        c->grid_hist = c->grid_acc_doc = c->grid_acc_word = c->grid_draw = fit(8);
    } else {
        c->grid_hist = fit(huge_blocks_per_sm(K, c->stage_ck, 0, false, M));
        c->grid_acc_doc = fit(huge_blocks_per_sm(K, c->stage_ck, 1, true, M));
        c->grid_acc_word = fit(huge_blocks_per_sm(K, c->stage_ck, 1, false, M));
        c->grid_draw = fit(huge_blocks_per_sm(K, c->stage_ck, 2, false, M));
    }
    c->grid_topic = (int)std::min<int64_t>(fit(topic_hist_blocks_per_sm(K)), std::max<int64_t>(1, (N + 8191) / 8192));

    // z = Dice(K), proposals = z (Alg. 2); c_k = histogram of z.  The sort
    // left its values in z and prop: their padding past N is cleared
    if ((e = cudaMemsetAsync(c->z + N, 0, 4 * 4, c->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->prop + N * M, 0, (size_t)4 * M * 4, c->st)) != cudaSuccess)
        return bail(cuda_fail(e, "clear padding"));
    if ((e = launch_init_z(c->z, c->prop, N, K, M, c->seed, c->st)) != cudaSuccess)
        return bail(cuda_fail(e, "init z"));
    if ((rc = recount(c))) return bail(rc);
    if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return bail(cuda_fail(e, "init"));
    trace.mark("grids, initial z and c_k");
    undo.armed = false;
    *out = c;
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_sweep(warplda_ctx* c, int32_t n) try {
    if (!c || n < 0) return fail(WARPLDA_EINVAL, "bad context or n");
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        int rc = run_phase(c, true);
        if (rc) return rc;
        rc = run_phase(c, false);
        if (rc) return rc;
    }
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_phase(warplda_ctx* c, int32_t phase) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (phase == WARPLDA_PHASE_DOC) {
        if (c->doc_done) return fail(WARPLDA_ESTATE, "document phase already run");
        return run_phase(c, true);
    }
    if (phase == WARPLDA_PHASE_WORD) {
        if (!c->doc_done) return fail(WARPLDA_ESTATE, "word phase before document phase");
        return run_phase(c, false);
    }
    return fail(WARPLDA_EINVAL, "unknown phase %d", phase);
} WL_ABI_CATCH

static int ensure_scratch(warplda_ctx* c) {
    if (c->scratch) return WARPLDA_OK;
    return dalloc(c, &c->scratch, c->N + 4, "alloc export scratch");
}

int warplda_counts_dev(warplda_ctx* c, int32_t* z_dev, int32_t* ck_dev) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (z_dev) WL_CU(launch_gather_docmajor(c->z, c->perm, c->N, z_dev, c->st), "gather z");
    if (ck_dev) WL_CU(cudaMemcpyAsync(ck_dev, c->ck, (size_t)c->K * 4, cudaMemcpyDeviceToDevice, c->st), "copy c_k");
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_counts(warplda_ctx* c, int32_t* z_docmajor, int32_t* ck) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (z_docmajor && c->N > 0) {
        // pinned host buffer: the gather writes into it through its device
        // alias (no device scratch, no separate copy); otherwise gather on
        // the device and copy
        cudaPointerAttributes pa{};
        const cudaError_t pe = cudaPointerGetAttributes(&pa, z_docmajor);
        if (pe != cudaSuccess) cudaGetLastError();   // clear the query's own error only
        const bool pinned = pe == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
        if (pinned) {
            WL_CU(launch_gather_docmajor(c->z, c->perm, c->N, static_cast<int32_t*>(pa.devicePointer), c->st),
                  "gather z");
        } else {
            int rc = ensure_scratch(c);
            if (rc) return rc;
            WL_CU(launch_gather_docmajor(c->z, c->perm, c->N, c->scratch, c->st), "gather z");
            WL_CU(cudaMemcpyAsync(z_docmajor, c->scratch, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->st),
                  "copy z");
        }
    }
    if (ck) WL_CU(cudaMemcpyAsync(ck, c->ck, (size_t)c->K * 4, cudaMemcpyDeviceToHost, c->st), "copy c_k");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return check_record(c, "counts");
} WL_ABI_CATCH

int warplda_get_state(warplda_ctx* c, int32_t* z, int32_t* prop, int32_t* ck, uint32_t* sweeps) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (z && c->N) WL_CU(cudaMemcpyAsync(z, c->z, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->st), "copy z");
    if (prop && c->N) WL_CU(cudaMemcpyAsync(prop, c->prop, (size_t)c->N * c->M * 4, cudaMemcpyDeviceToHost, c->st), "copy proposals");
    if (ck) WL_CU(cudaMemcpyAsync(ck, c->ck, (size_t)c->K * 4, cudaMemcpyDeviceToHost, c->st), "copy c_k");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    if (sweeps) *sweeps = c->iter;
    return check_record(c, "state");
} WL_ABI_CATCH

int warplda_set_state(warplda_ctx* c, const int32_t* z, const int32_t* prop, uint32_t sweeps) try {
    if (!c || (c->N > 0 && (!z || !prop))) return fail(WARPLDA_EINVAL, "null argument");
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (c->N) {
        WL_CU(cudaMemcpyAsync(c->z, z, (size_t)c->N * 4, cudaMemcpyHostToDevice, c->st), "upload z");
        WL_CU(cudaMemcpyAsync(c->prop, prop, (size_t)c->N * c->M * 4, cudaMemcpyHostToDevice, c->st), "upload proposals");
    }
    WL_CU(cudaMemsetAsync(c->d_bad, 0, 4, c->st), "memset");
    WL_CU(launch_check_range(c->z, c->N, c->K, c->d_bad, c->st), "range check");
    WL_CU(launch_check_range(c->prop, c->N * c->M, c->K, c->d_bad, c->st), "range check");
    int32_t bad = 0;
    WL_CU(cudaMemcpyAsync(&bad, c->d_bad, 4, cudaMemcpyDeviceToHost, c->st), "copy flag");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    if (bad) {
        // leave a valid state behind: re-initialise
        WL_CU(launch_init_z(c->z, c->prop, c->N, c->K, c->M, c->seed, c->st), "init z");
        int rc = recount(c);
        if (rc) return rc;
        c->iter = 0;
        WL_CU(cudaStreamSynchronize(c->st), "synchronize");
        return fail(WARPLDA_EINVAL, "%d values outside [0, K); state re-initialised", bad);
    }
    int rc = recount(c);
    if (rc) return rc;
    c->iter = sweeps;
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_doc_batches(warplda_ctx* c, int64_t* n_batches, int32_t* batches, int32_t* sperm,
                        uint32_t* sinfo) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (n_batches) *n_batches = (int64_t)(c->docs.batches[0].size() + c->docs.batches[1].size());
    if (batches) {
        size_t o = 0;
        for (int k = 0; k < 2; ++k) {
            const auto& b = c->docs.batches[k];
            if (!b.empty()) std::memcpy(batches + o, b.data(), b.size() * sizeof(int4));
            o += 4 * b.size();
        }
    }
    if (c->N > 0 && sperm)
        WL_CU(cudaMemcpyAsync(sperm, c->sperm, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->st), "copy lists");
    if (c->N > 0 && sinfo)
        WL_CU(cudaMemcpyAsync(sinfo, c->sinfo, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->st), "copy lists");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_token_order(warplda_ctx* c, int64_t* word_ptr, int32_t* perm) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (word_ptr) std::memcpy(word_ptr, c->word_ptr_h.data(), (size_t)(c->V + 1) * 8);
    if (perm && c->N) {
        WL_CU(cudaMemcpyAsync(perm, c->perm, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->st), "copy perm");
        WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    }
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_loglik(warplda_ctx* c, double* out) try {
    if (!c || !out) return fail(WARPLDA_EINVAL, "null argument");
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    WL_CU(cudaMemsetAsync(c->d_ll, 0, sizeof(double), c->st), "memset");
    const double a = c->alpha, b = c->beta;
    const double abar = (double)c->K * a, bbar = (double)c->V * b;
    for (int doc = 1; doc >= 0; --doc) {
        Tier& T = doc ? c->docs : c->words;
        PhaseArgs pa = phase_args(c, doc, c->iter);
        int32_t* rows = doc ? c->rows_doc : c->rows_pre;
        if (!T.chunks.empty() && c->sparse) {
            const int k = doc ? 0 : 1;
            WL_CU(cudaMemsetAsync(c->sslots[k], 0, (size_t)c->sn[k] * 8, c->st), "zero rows");
            WL_CU(cudaMemsetAsync(c->counters + kCtrLoglik, 0, sizeof(int32_t), c->st), "reset counter");
            WL_CU(launch_sparse_hist(doc, pa, huge_work(c, T, kCtrLoglik, true), SparseRows{c->d_soff[k], c->sslots[k]},
                                     c->grid_hist, c->st), "loglik rows");
            WL_CU(cudaMemsetAsync(c->counters + kCtrLoglik, 0, sizeof(int32_t), c->st), "reset counter");
            WL_CU(launch_sparse_loglik(c->sslots[k], c->sn[k], doc ? a : b, c->d_ll, c->st), "loglik rows");
        } else if (!T.chunks.empty()) {
            WL_CU(launch_zero(rows, r4(T.nrows * (int64_t)c->K), c->st), "zero rows");
            WL_CU(cudaMemsetAsync(c->counters + kCtrLoglik, 0, sizeof(int32_t), c->st), "reset counter");
            WL_CU(launch_huge_hist(doc, pa, huge_work(c, T, kCtrLoglik, true), rows, c->grid_hist, c->st),
                  "loglik rows");
            WL_CU(launch_loglik_rows(rows, T.nrows, c->K, doc ? a : b, c->d_ll, c->st), "loglik rows");
        }
        WL_CU(launch_loglik_batches(doc, c->z, c->perm, doc ? c->doc_off : c->word_off,
                                    T.d_ll_batches, (int)T.ll_batches.size(), c->K, doc ? a : b,
                                    8192, c->N, doc ? c->D : c->V, c->d_fault, c->d_ll, c->sms * 2,
                                    c->st), "loglik batches");
    }
    WL_CU(launch_loglik_lengths(c->doc_off, c->D, abar, c->d_ll, c->st), "loglik lengths");
    WL_CU(launch_loglik_topics(c->ck, c->K, bbar, c->d_ll, c->st), "loglik topics");
    WL_CU(cudaMemcpyAsync(out, c->d_ll, sizeof(double), cudaMemcpyDeviceToHost, c->st), "copy loglik");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return check_record(c, "loglik");
} WL_ABI_CATCH

struct CkptHeader {
    char magic[8];
    int64_t D, V, N;
    int32_t K, M;
    float alpha, beta;
    uint64_t seed;
    uint32_t iter, pad;
};

int warplda_save(warplda_ctx* c, const char* path) try {
    if (!c || !path) return fail(WARPLDA_EINVAL, "null argument");
    std::vector<int32_t> z((size_t)c->N), p((size_t)c->N * c->M);
    uint32_t it = 0;
    int rc = warplda_get_state(c, z.data(), p.data(), nullptr, &it);
    if (rc) return rc;
    CkptHeader h{};
    std::memcpy(h.magic, "WARPLDA1", 8);
    h.D = c->D; h.V = c->V; h.N = c->N; h.K = c->K; h.M = c->M;
    h.alpha = c->alpha; h.beta = c->beta; h.seed = c->seed; h.iter = it;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(WARPLDA_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
              std::fwrite(z.data(), 4, z.size(), f) == z.size() &&
              std::fwrite(p.data(), 4, p.size(), f) == p.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? WARPLDA_OK : fail(WARPLDA_EIO, "write to %s failed", path);
} WL_ABI_CATCH

int warplda_load(warplda_ctx* c, const char* path) try {
    if (!c || !path) return fail(WARPLDA_EINVAL, "null argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(WARPLDA_EIO, "cannot open %s", path);
    CkptHeader h{};
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "WARPLDA1", 8) != 0) {
        std::fclose(f);
        return fail(WARPLDA_EIO, "%s is not a checkpoint", path);
    }
    if (h.D != c->D || h.V != c->V || h.N != c->N || h.K != c->K || h.M != c->M ||
        h.alpha != c->alpha || h.beta != c->beta || h.seed != c->seed) {
        std::fclose(f);
        return fail(WARPLDA_EINVAL, "checkpoint does not match this context");
    }
    std::vector<int32_t> z((size_t)c->N), p((size_t)c->N * c->M);
    bool ok = std::fread(z.data(), 4, z.size(), f) == z.size() &&
              std::fread(p.data(), 4, p.size(), f) == p.size();
    std::fclose(f);
    if (!ok) return fail(WARPLDA_EIO, "%s is truncated", path);
    return warplda_set_state(c, z.data(), p.data(), h.iter);
} WL_ABI_CATCH

int warplda_get_info(warplda_ctx* c, warplda_info* o) try {
    if (!c || !o) return fail(WARPLDA_EINVAL, "null argument");
    std::memset(o, 0, sizeof(*o));
    o->D = c->D; o->V = c->V; o->N = c->N; o->K = c->K; o->M = c->M;
    o->launches_per_sweep = launches_per_phase(c, true) + launches_per_phase(c, false);
    o->batch_max_tokens = std::max(c->bmax[0], c->bmax[1]);
    o->doc_batches = (int64_t)(c->docs.batches[0].size() + c->docs.batches[1].size() +
                               c->docs.warp_list.size());
    o->word_batches = (int64_t)(c->words.batches[0].size() + c->words.batches[1].size());
    o->huge_docs = c->docs.nrows;
    o->huge_doc_tokens = c->docs.row_tokens;
    o->mega_words = c->words.nrows - (int64_t)c->words.cluster_list.size();
    o->mega_word_tokens = c->words.s_row_tokens;
    o->cluster_words = (int64_t)c->words.cluster_list.size();
    o->cluster_word_tokens = c->words.cluster_tokens;
    o->device_bytes = c->device_bytes;
    // the small document class: every batched token outside the large
    // class and the warp tier
    o->pipe_doc_tokens = c->doc_pipe ? c->N - c->docs.row_tokens - c->docs.large_tokens - c->docs.warp_tokens : 0;
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_profile(warplda_ctx* c, int32_t enable) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    for (auto& r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->recs.clear();
    c->prof = enable != 0;
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_kernel_times(warplda_ctx* c, int32_t cap, const char** names, int64_t* launches,
                         double* total_ms) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    double ms[kcCount] = {0};
    int64_t n[kcCount] = {0};
    for (auto& r : c->recs) {
        float t = 0;
        WL_CU(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
        ms[r.cls] += t;
        n[r.cls] += 1;
    }
    int k = 0;
    for (int i = 0; i < kcCount; ++i) {
        if (n[i] == 0) continue;
        if (k < cap) {
            if (names) names[k] = kClassNames[i];
            if (launches) launches[k] = n[i];
            if (total_ms) total_ms[k] = ms[i];
        }
        ++k;
    }
    return k;
} WL_ABI_CATCH

int warplda_foldin(warplda_ctx* c, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                   const int64_t* doc_ids, int32_t sweeps, uint64_t seed, int32_t proposal,
                   float* theta_out, int32_t* z_out) try {
    if (!c || !doc_ptr || Dn < 0 || sweeps < 0) return fail(WARPLDA_EINVAL, "bad fold-in arguments");
    if (proposal != WARPLDA_PROPOSAL_PLAIN && proposal != WARPLDA_PROPOSAL_LEARNED)
        return fail(WARPLDA_EINVAL, "unknown proposal %d", proposal);
    if (c->K > kDenseRowMaxK) return fail(WARPLDA_EINVAL, "fold-in keeps a dense [V, K] model: K must be <= %d", kDenseRowMaxK);
    if (proposal == WARPLDA_PROPOSAL_LEARNED && !c->enc.ready)
        return fail(WARPLDA_ESTATE, "the learned proposal needs an initialised encoder");
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    if (Dn > (int64_t)0x7FFFFFF0) return fail(WARPLDA_EINVAL, "too many documents");
    if (doc_ptr[0] != 0) return fail(WARPLDA_EINVAL, "doc_ptr[0] must be 0");
    const int K = c->K, M = c->M;
    const int Lcap = K <= kDenseMaxK ? 65535 : (1 << kHashCountBits) - 1;
    int64_t Lmax = 0;
    for (int64_t d = 0; d < Dn; ++d) {
        const int64_t L = doc_ptr[d + 1] - doc_ptr[d];
        if (L < 0) return fail(WARPLDA_EINVAL, "doc_ptr decreases at %lld", (long long)d);
        Lmax = std::max(Lmax, L);
    }
    if (Lmax > Lcap) return fail(WARPLDA_EINVAL, "a fold-in document has more than %d tokens", Lcap);
    const int64_t Nn = doc_ptr[Dn];
    if (Nn > (int64_t)0x7FFFFFF0) return fail(WARPLDA_EINVAL, "too many fold-in tokens");
    if (Nn > 0 && !doc_word) return fail(WARPLDA_EINVAL, "null doc_word");
    {
        const int64_t p = first_bad_word(doc_word, Nn, c->V);
        if (p >= 0) return fail(WARPLDA_EINVAL, "word id %d at %lld outside [0, V)", doc_word[p], (long long)p);
    }
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");

    // the frozen model: C_w prefix rows and c_k of the current state
    {
        int rc = ensure_model(c);
        if (rc) return rc;
    }

    // documents longest first, so that the long ones start early
    std::vector<int32_t> order((size_t)Dn), off((size_t)Dn + 1);
    std::vector<int64_t> ids((size_t)Dn);
    for (int64_t d = 0; d < Dn; ++d) {
        order[d] = (int32_t)d;
        ids[d] = doc_ids ? doc_ids[d] : d;
    }
    for (int64_t d = 0; d <= Dn; ++d) off[d] = (int32_t)doc_ptr[d];
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return off[a + 1] - off[a] > off[b + 1] - off[b];
    });

    FoldScratch buf{c};
    FoldArgs f{};
    int32_t *d_z, *d_prop, *d_words, *d_off, *d_order, *d_counter;
    int64_t* d_ids;
    float* d_theta = nullptr;
    WL_CU(buf.get(&d_z, Nn + 1), "alloc fold-in z");
    WL_CU(buf.get(&d_prop, (Nn + 1) * M), "alloc fold-in proposals");
    WL_CU(buf.get(&d_words, Nn + 1), "alloc fold-in words");
    WL_CU(buf.get(&d_off, Dn + 1), "alloc fold-in offsets");
    WL_CU(buf.get(&d_order, Dn + 1), "alloc fold-in order");
    WL_CU(buf.get(&d_ids, Dn + 1), "alloc fold-in ids");
    WL_CU(buf.get(&d_counter, 1), "alloc fold-in counter");
    if (theta_out) WL_CU(buf.get(&d_theta, Dn * (int64_t)K + 1), "alloc fold-in theta");
    if (Nn > 0)
        WL_CU(cudaMemcpyAsync(d_words, doc_word, (size_t)Nn * 4, cudaMemcpyHostToDevice, c->st), "upload words");
    WL_CU(cudaMemcpyAsync(d_off, off.data(), (size_t)(Dn + 1) * 4, cudaMemcpyHostToDevice, c->st), "upload offsets");
    if (Dn > 0) {
        WL_CU(cudaMemcpyAsync(d_order, order.data(), (size_t)Dn * 4, cudaMemcpyHostToDevice, c->st), "upload order");
        WL_CU(cudaMemcpyAsync(d_ids, ids.data(), (size_t)Dn * 8, cudaMemcpyHostToDevice, c->st), "upload ids");
    }
    WL_CU(cudaMemsetAsync(d_counter, 0, 4, c->st), "reset counter");
    f.z = d_z;
    f.prop = d_prop;
    f.words = d_words;
    f.doc_off = d_off;
    f.order = d_order;
    f.ids = d_ids;
    f.Cw = c->model_cw;
    f.Zs = c->model_zs;
    f.word_off = c->word_off;
    f.ckb = c->model_ckb;
    f.theta = d_theta;
    f.counter = d_counter;
    f.fault = c->d_fault;
    f.Dn = (int)Dn;
    f.K = K;
    f.M = M;
    f.V = (int)c->V;
    f.sweeps = sweeps;
    f.Lmax = (int)Lmax;
    f.alpha = c->alpha;
    f.abar = c->abar;
    f.beta = c->beta;
    f.kbeta = c->kbeta;
    f.rk = round_keys(seed);
    if (proposal == WARPLDA_PROPOSAL_LEARNED && Dn > 0) {
        // the encoder's proposal rows and their alias tables
        HostDocs hd;
        float* q;
        int2* atab;
        int32_t* ident;
        std::vector<int32_t> idv((size_t)Dn);
        for (int64_t d = 0; d < Dn; ++d) idv[d] = (int32_t)d;
        WL_CU(buf.get(&ident, Dn), "alloc ids");
        WL_CU(buf.get(&q, Dn * (int64_t)K), "alloc proposals");
        WL_CU(buf.get(&atab, Dn * (int64_t)K), "alloc alias tables");
        WL_CU(cudaMemcpyAsync(ident, idv.data(), (size_t)Dn * 4, cudaMemcpyHostToDevice, c->st), "upload ids");
        hd.off = d_off;
        hd.words = d_words;
        hd.ids = ident;
        int rc2 = enc_proposal_dev(c, Dn, hd, q);   // synchronises
        if (rc2) return rc2;
        WL_CU(launch_enc_alias(q, Dn, K, atab, c->st), "alias tables");
        f.q = q;
        f.atab = atab;
    }
    const int tab_words = foldin_table_words(K, (int)Lmax);
    const int warps = foldin_warps(tab_words);
    if (proposal == WARPLDA_PROPOSAL_PLAIN && c->foldin_word_major && Dn > 0) {
        // word-major phases: the requests' tokens grouped by word once, then
        // per sweep a document-phase and a word-phase launch
        const int64_t V = c->V;
        const bool stage = K <= kFoldStageMaxK;
        const int stage_min = stage ? kFoldStageMin : 0x7FFFFFFF;
        int32_t *cnt, *hc, *lc, *pc, *cur, *tmp, *npieces, *counters;
        int4 *rec, *pieces;
        WL_CU(buf.get(&cnt, V + 1), "alloc fold-in word counts");
        WL_CU(buf.get(&hc, V + 1), "alloc fold-in word offsets");
        WL_CU(buf.get(&lc, V + 1), "alloc fold-in word offsets");
        WL_CU(buf.get(&pc, V + 1), "alloc fold-in piece offsets");
        WL_CU(buf.get(&cur, V + 1), "alloc fold-in cursors");
        WL_CU(buf.get(&tmp, scan_scratch_words(V + 1)), "alloc fold-in scan scratch");
        WL_CU(buf.get(&rec, Nn), "alloc fold-in records");
        WL_CU(buf.get(&pieces, fold_pieces_bound(Nn, stage_min)), "alloc fold-in pieces");
        WL_CU(buf.get(&npieces, 1), "alloc fold-in piece count");
        WL_CU(buf.get(&counters, (int64_t)sweeps + 2), "alloc fold-in counters");
        WL_CU(cudaMemsetAsync(counters, 0, ((size_t)sweeps + 2) * 4, c->st), "reset counters");
        FoldWords fw{};
        fw.rec = rec;
        fw.pieces = pieces;
        fw.npieces = npieces;
        fw.Nn = Nn;
        fw.pstride = stage ? ((K + 1 + 3) & ~3) : 0;
        fw.per = ((K + 31) / 32) | 1;
        int rc = launch_timed(c, kcFoldBuild, [&] {
            return launch_fold_words_build(f, Nn, stage_min, cnt, hc, lc, pc, cur, tmp, rec, pieces, npieces,
                                           4 * c->sms, c->st);
        });
        if (rc) return rc;
        const int dper = fold_doc_blocks_per_sm(K, M, tab_words);
        const int wper = fold_word_blocks_per_sm(M, fw);
        if (dper < 1 || wper < 1) return fail(WARPLDA_EINVAL, "fold-in tables do not fit in shared memory");
        const int dgrid = (int)std::min<int64_t>((int64_t)dper * c->sms, (Dn + warps - 1) / warps + 1);
        const int wgrid = wper * c->sms;
        auto doc_launch = [&](int it, int mode) {
            return launch_timed(c, kcFoldDoc, [&] {
                return launch_fold_doc(f, tab_words, it, mode, counters + it - 1, dgrid, c->st);
            });
        };
        if (sweeps == 0) {
            if ((rc = doc_launch(1, 1 | 4))) return rc;
        } else {
            for (int it = 1; it <= sweeps; ++it) {
                if ((rc = doc_launch(it, (it == 1 ? 1 : 0) | 2))) return rc;
                rc = launch_timed(c, kcFoldWord, [&] { return launch_fold_word(f, fw, it, wgrid, c->st); });
                if (rc) return rc;
            }
            if (theta_out && (rc = doc_launch(sweeps + 1, 4))) return rc;
        }
    } else {
        const int per_sm = foldin_blocks_per_sm(K, M, tab_words);
        if (per_sm < 1) return fail(WARPLDA_EINVAL, "fold-in tables do not fit in shared memory");
        const int grid = (int)std::min<int64_t>((int64_t)per_sm * c->sms, (Dn + warps - 1) / warps + 1);
        const int rc = launch_timed(c, kcFoldin, [&] { return launch_foldin(f, tab_words, grid, c->st); });
        if (rc) return rc;
    }
    if (z_out && Nn > 0)
        WL_CU(cudaMemcpyAsync(z_out, d_z, (size_t)Nn * 4, cudaMemcpyDeviceToHost, c->st), "copy z");
    if (theta_out && Dn > 0)
        WL_CU(cudaMemcpyAsync(theta_out, d_theta, (size_t)Dn * K * 4, cudaMemcpyDeviceToHost, c->st), "copy theta");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return check_record(c, "fold-in");
} WL_ABI_CATCH

int warplda_word_counts(warplda_ctx* c, int32_t* cw) try {
    if (!c || !cw) return fail(WARPLDA_EINVAL, "null argument");
    if (c->K > kDenseRowMaxK) return fail(WARPLDA_EINVAL, "dense C_w needs K <= %d", kDenseRowMaxK);
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    int rc = ensure_model(c);
    if (rc) return rc;
    WL_CU(cudaMemcpyAsync(cw, c->model_cw, (size_t)c->V * c->K * 4, cudaMemcpyDeviceToHost, c->st), "copy C_w");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return check_record(c, "word counts");
} WL_ABI_CATCH

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static float unit_uniform(uint64_t* x) { return (float)((splitmix64(x) >> 40) * (1.0 / 16777216.0)); }

int warplda_encoder_init(warplda_ctx* c, int32_t log2_features, int32_t hidden, int32_t batch_rows,
                         uint64_t seed) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    auto& e = c->enc;
    if (e.ready) return fail(WARPLDA_ESTATE, "the encoder is already initialised");
    if (c->K > kDenseRowMaxK) return fail(WARPLDA_EINVAL, "the encoder needs K <= %d", kDenseRowMaxK);
    if (log2_features < 6 || log2_features > 20) return fail(WARPLDA_EINVAL, "log2_features must be in [6, 20]");
    if (hidden < 128 || hidden > 2048 || hidden % 128) return fail(WARPLDA_EINVAL, "hidden must be a multiple of 128 in [128, 2048]");
    if (batch_rows < 128 || batch_rows > 2048 || batch_rows % 128)
        return fail(WARPLDA_EINVAL, "batch_rows must be a multiple of 128 in [128, 2048]");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    e.log2F = log2_features;
    e.H = hidden;
    e.B = batch_rows;
    e.Kp = (c->K + 127) / 128 * 128;
    const int64_t F = enc_F(c), H = e.H, Kp = e.Kp, B = e.B;
    int rc;
#define WL_A(ptr, n) if ((rc = dalloc(c, &(ptr), (n), "alloc encoder"))) return rc
    WL_A(e.W1, F * H); WL_A(e.b1, H); WL_A(e.W2t, Kp * H); WL_A(e.b2, Kp);
    WL_A(e.mW1, F * H); WL_A(e.vW1, F * H); WL_A(e.mb1, H); WL_A(e.vb1, H);
    WL_A(e.mW2, Kp * H); WL_A(e.vW2, Kp * H); WL_A(e.mb2, Kp); WL_A(e.vb2, Kp);
    WL_A(e.W1b, F * H); WL_A(e.W2tb, Kp * H); WL_A(e.W2nb, Kp * H);
    WL_A(e.gW1, F * H); WL_A(e.gb1, H); WL_A(e.gW2t, Kp * H); WL_A(e.gb2, Kp);
    WL_A(e.h_pre, B * H); WL_A(e.logits, B * Kp); WL_A(e.dH, B * H);
    WL_A(e.hb, B * H); WL_A(e.hbT, B * H); WL_A(e.dl, B * Kp); WL_A(e.dlT, B * Kp);
    WL_A(e.cnt, B * (int64_t)c->K); WL_A(e.loss, 1); WL_A(e.ids, std::max<int64_t>(c->D, 1));
    e.gwork_floats = std::max({gemm_splits((int)B, (int)Kp, (int)H, INT64_MAX) * B * Kp,
                               gemm_splits((int)B, (int)H, (int)Kp, INT64_MAX) * B * H,
                               gemm_splits((int)Kp, (int)H, (int)B, INT64_MAX) * Kp * H});
    WL_A(e.gwork, e.gwork_floats);
#undef WL_A
    // W1 ~ U(-1, 1); W2 ~ U(-a, a), a = sqrt(6 / (H + K)) (Glorot); biases 0
    std::vector<float> w1((size_t)(F * H)), w2((size_t)(Kp * H), 0.0f);
    uint64_t st = seed;
    for (auto& v : w1) v = 2.0f * unit_uniform(&st) - 1.0f;
    const float a = std::sqrt(6.0f / (float)(H + c->K));
    for (int64_t k = 0; k < c->K; ++k)
        for (int64_t j = 0; j < H; ++j) w2[k * H + j] = a * (2.0f * unit_uniform(&st) - 1.0f);
    WL_CU(cudaMemcpyAsync(e.W1, w1.data(), w1.size() * 4, cudaMemcpyHostToDevice, c->st), "upload W1");
    WL_CU(cudaMemcpyAsync(e.W2t, w2.data(), w2.size() * 4, cudaMemcpyHostToDevice, c->st), "upload W2");
    WL_CU(cudaMemsetAsync(e.b1, 0, H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.b2, 0, Kp * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.mW1, 0, F * H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.vW1, 0, F * H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.mb1, 0, H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.vb1, 0, H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.mW2, 0, Kp * H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.vW2, 0, Kp * H * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.mb2, 0, Kp * 4, c->st), "zero");
    WL_CU(cudaMemsetAsync(e.vb2, 0, Kp * 4, c->st), "zero");
    WL_CU(launch_enc_to_bf16(e.W1, F * H, e.W1b, c->st), "W1 copy");
    WL_CU(launch_enc_w2_copies(e.W2t, (int)Kp, (int)H, e.W2tb, e.W2nb, c->st), "W2 copies");
    WL_CU(cudaMemsetAsync(c->d_fault + 3, 0, 4, c->st), "clear GEMM status");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    e.step = 0;
    e.ready = true;
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_encoder_weights(warplda_ctx* c, int32_t set, float* W1, float* b1, float* W2, float* b2) try {
    if (!c || !W1 || !b1 || !W2 || !b2) return fail(WARPLDA_EINVAL, "null argument");
    auto& e = c->enc;
    if (!e.ready) return fail(WARPLDA_ESTATE, "the encoder is not initialised");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    const int64_t F = enc_F(c), H = e.H, Kp = e.Kp, K = c->K;
    std::vector<float> w2t((size_t)(Kp * H), 0.0f);
    if (set) {
        for (int64_t j = 0; j < H; ++j)
            for (int64_t k = 0; k < K; ++k) w2t[k * H + j] = W2[j * K + k];
        WL_CU(cudaMemcpyAsync(e.W1, W1, (size_t)(F * H) * 4, cudaMemcpyHostToDevice, c->st), "upload W1");
        WL_CU(cudaMemcpyAsync(e.b1, b1, (size_t)H * 4, cudaMemcpyHostToDevice, c->st), "upload b1");
        WL_CU(cudaMemcpyAsync(e.W2t, w2t.data(), w2t.size() * 4, cudaMemcpyHostToDevice, c->st), "upload W2");
        WL_CU(cudaMemsetAsync(e.b2, 0, (size_t)Kp * 4, c->st), "zero b2");
        WL_CU(cudaMemcpyAsync(e.b2, b2, (size_t)K * 4, cudaMemcpyHostToDevice, c->st), "upload b2");
        WL_CU(launch_enc_to_bf16(e.W1, F * H, e.W1b, c->st), "W1 copy");
        WL_CU(launch_enc_w2_copies(e.W2t, (int)Kp, (int)H, e.W2tb, e.W2nb, c->st), "W2 copies");
        WL_CU(cudaStreamSynchronize(c->st), "synchronize");
        return WARPLDA_OK;
    }
    WL_CU(cudaMemcpyAsync(W1, e.W1, (size_t)(F * H) * 4, cudaMemcpyDeviceToHost, c->st), "copy W1");
    WL_CU(cudaMemcpyAsync(b1, e.b1, (size_t)H * 4, cudaMemcpyDeviceToHost, c->st), "copy b1");
    WL_CU(cudaMemcpyAsync(w2t.data(), e.W2t, w2t.size() * 4, cudaMemcpyDeviceToHost, c->st), "copy W2");
    WL_CU(cudaMemcpyAsync(b2, e.b2, (size_t)K * 4, cudaMemcpyDeviceToHost, c->st), "copy b2");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    for (int64_t j = 0; j < H; ++j)
        for (int64_t k = 0; k < K; ++k) W2[j * K + k] = w2t[k * H + j];
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_encoder_grad(warplda_ctx* c, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                         const float* theta, double* loss, float* gW1, float* gb1, float* gW2, float* gb2) try {
    if (!c || !theta || !loss || !gW1 || !gb1 || !gW2 || !gb2) return fail(WARPLDA_EINVAL, "null argument");
    auto& e = c->enc;
    if (!e.ready) return fail(WARPLDA_ESTATE, "the encoder is not initialised");
    if (Dn < 1 || Dn > e.B) return fail(WARPLDA_EINVAL, "Dn must be in [1, batch_rows]");
    int rc = check_docs(c, Dn, doc_ptr, doc_word);
    if (rc) return rc;
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    FoldBuffers buf;
    HostDocs hd;
    if ((rc = upload_docs(c, buf, Dn, doc_ptr, doc_word, &hd))) return rc;
    const int64_t F = enc_F(c), H = e.H, Kp = e.Kp, K = c->K;
    float* tg;
    WL_CU(buf.get(&tg, Dn * K), "alloc targets");
    WL_CU(cudaMemcpyAsync(tg, theta, (size_t)(Dn * K) * 4, cudaMemcpyHostToDevice, c->st), "upload targets");
    if ((rc = enc_zero_grads(c))) return rc;
    WL_CU(cudaMemsetAsync(e.loss, 0, 8, c->st), "zero loss");
    EncBatch b{hd.ids, hd.off, hd.words, (int)Dn};
    if ((rc = enc_forward(c, b, nullptr, true, tg))) return rc;
    if ((rc = enc_backward(c, b))) return rc;
    if ((rc = enc_status(c))) return rc;
    std::vector<float> g2((size_t)(Kp * H));
    WL_CU(cudaMemcpyAsync(loss, e.loss, 8, cudaMemcpyDeviceToHost, c->st), "copy loss");
    WL_CU(cudaMemcpyAsync(gW1, e.gW1, (size_t)(F * H) * 4, cudaMemcpyDeviceToHost, c->st), "copy gW1");
    WL_CU(cudaMemcpyAsync(gb1, e.gb1, (size_t)H * 4, cudaMemcpyDeviceToHost, c->st), "copy gb1");
    WL_CU(cudaMemcpyAsync(g2.data(), e.gW2t, g2.size() * 4, cudaMemcpyDeviceToHost, c->st), "copy gW2");
    WL_CU(cudaMemcpyAsync(gb2, e.gb2, (size_t)K * 4, cudaMemcpyDeviceToHost, c->st), "copy gb2");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    for (int64_t j = 0; j < H; ++j)
        for (int64_t k = 0; k < K; ++k) gW2[j * K + k] = g2[k * H + j];
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_encoder_train(warplda_ctx* c, int32_t epochs, float lr, uint64_t seed, double* epoch_loss) try {
    if (!c || epochs < 0 || !(lr > 0.0f)) return fail(WARPLDA_EINVAL, "bad training arguments");
    auto& e = c->enc;
    if (!e.ready) return fail(WARPLDA_ESTATE, "the encoder is not initialised");
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    int rc;
    if (!e.docword) {
        if ((rc = dalloc(c, &e.docword, c->N + 4, "alloc document words"))) return rc;
        WL_CU(launch_enc_docword(c->perm, c->word_off, c->N, c->V, e.docword, c->st), "document words");
    }
    std::vector<int32_t> docs;
    std::vector<int32_t> off((size_t)c->D + 1);
    WL_CU(cudaMemcpyAsync(off.data(), c->doc_off, (size_t)(c->D + 1) * 4, cudaMemcpyDeviceToHost, c->st), "copy offsets");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    for (int64_t d = 0; d < c->D; ++d)
        if (off[d + 1] > off[d]) docs.push_back((int32_t)d);
    const int64_t nd = (int64_t)docs.size();
    uint64_t rs = seed;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = nd - 1; i > 0; --i) std::swap(docs[i], docs[splitmix64(&rs) % (uint64_t)(i + 1)]);
        if (nd > 0)
            WL_CU(cudaMemcpyAsync(e.ids, docs.data(), (size_t)nd * 4, cudaMemcpyHostToDevice, c->st), "upload order");
        WL_CU(cudaMemsetAsync(e.loss, 0, 8, c->st), "zero loss");
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 < nd; b0 += e.B, ++nb) {
            EncBatch b{e.ids + b0, c->doc_off, e.docword, (int)std::min<int64_t>(e.B, nd - b0)};
            if ((rc = enc_zero_grads(c))) return rc;
            if ((rc = enc_forward(c, b, nullptr, true, nullptr))) return rc;
            if ((rc = enc_backward(c, b))) return rc;
            if ((rc = enc_adam_step(c, lr))) return rc;
        }
        double l = 0.0;
        WL_CU(cudaMemcpyAsync(&l, e.loss, 8, cudaMemcpyDeviceToHost, c->st), "copy loss");
        if ((rc = enc_status(c))) return rc;   // synchronises (the order upload reads `docs`)
        if (epoch_loss) epoch_loss[ep] = nb ? l / (double)nb : 0.0;
    }
    return check_record(c, "encoder training");
} WL_ABI_CATCH

int warplda_encoder_proposal(warplda_ctx* c, int64_t Dn, const int64_t* doc_ptr, const int32_t* doc_word,
                             float* q_out) try {
    if (!c || !q_out) return fail(WARPLDA_EINVAL, "null argument");
    if (!c->enc.ready) return fail(WARPLDA_ESTATE, "the encoder is not initialised");
    int rc = check_docs(c, Dn, doc_ptr, doc_word);
    if (rc) return rc;
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    FoldBuffers buf;
    HostDocs hd;
    if ((rc = upload_docs(c, buf, Dn, doc_ptr, doc_word, &hd))) return rc;
    float* q;
    WL_CU(buf.get(&q, Dn * (int64_t)c->K), "alloc proposals");
    if ((rc = enc_proposal_dev(c, Dn, hd, q))) return rc;
    if (Dn > 0)
        WL_CU(cudaMemcpyAsync(q_out, q, (size_t)Dn * c->K * 4, cudaMemcpyDeviceToHost, c->st), "copy proposals");
    WL_CU(cudaStreamSynchronize(c->st), "synchronize");
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, const float* bias_dev,
                      int32_t M, int32_t N, int32_t K, void* cuda_stream) try {
    if (!A_dev || !B_dev || !C_dev) return fail(WARPLDA_EINVAL, "null matrix pointer");
    if (M < 0 || N < 0 || K < 0 || M % 128 || N % 128 || K % 64)
        return fail(WARPLDA_EINVAL, "GEMM needs M, N multiples of 128 and K a multiple of 64");
    if (((uintptr_t)A_dev | (uintptr_t)B_dev | (uintptr_t)C_dev) & 15)
        return fail(WARPLDA_EINVAL, "GEMM operands must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int32_t* status = nullptr;
    float* work = nullptr;
    // the split-K workspace the encoder would use for this shape
    const int64_t wf = M > 0 && N > 0 && K > 0 ? (int64_t)gemm_splits(M, N, K, INT64_MAX) * M * N : 0;
    WL_CU(dev_malloc((void**)&status, sizeof(int32_t)), "alloc GEMM status");
    cudaError_t e = wf > (int64_t)M * N ? dev_malloc((void**)&work, (size_t)wf * 4) : cudaSuccess;
    if (e != cudaSuccess) {
        cudaFree(status);
        return cuda_fail(e, "alloc GEMM workspace");
    }
    int32_t h = 0;
    e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_gemm_bf16((const uint16_t*)A_dev, (const uint16_t*)B_dev, C_dev, bias_dev, M, N, K, status, st,
                             work, work ? wf : 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(status);
    if (work) cudaFree(work);
    if (e != cudaSuccess) return cuda_fail(e, "GEMM");
    if (h) return fail(WARPLDA_ETIMEDOUT, "GEMM: a tensor-core wait ran out");
    return WARPLDA_OK;
} WL_ABI_CATCH


int warplda_server_create(warplda_ctx* c, int32_t slots, int64_t pool_tokens, int32_t max_doc_tokens,
                          int32_t sweeps, uint64_t seed, int32_t proposal, warplda_server** out) try {
    if (!c || !out) return fail(WARPLDA_EINVAL, "null argument");
    *out = nullptr;
    if (slots < 1 || slots > (1 << 20) || pool_tokens < 1 || pool_tokens > (int64_t)0x7FFFFFF0 || sweeps < 1 ||
        max_doc_tokens < 1)
        return fail(WARPLDA_EINVAL, "bad server sizes");
    const int Lcap = c->K <= kDenseMaxK ? 65535 : (1 << kHashCountBits) - 1;
    if (max_doc_tokens > Lcap) return fail(WARPLDA_EINVAL, "max_doc_tokens above %d", Lcap);
    if (proposal != WARPLDA_PROPOSAL_PLAIN && proposal != WARPLDA_PROPOSAL_LEARNED)
        return fail(WARPLDA_EINVAL, "unknown proposal %d", proposal);
    if (proposal == WARPLDA_PROPOSAL_LEARNED && !c->enc.ready)
        return fail(WARPLDA_ESTATE, "the learned proposal needs an initialised encoder");
    if (c->K > kDenseRowMaxK) return fail(WARPLDA_EINVAL, "serving keeps a dense [V, K] model: K must be <= %d", kDenseRowMaxK);
    if (c->doc_done) return fail(WARPLDA_ESTATE, "a word phase is pending");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    int rc = ensure_model(c);
    if (rc) return rc;
    auto* s = new warplda_server();
    auto undo = on_exit([&] {
        server_free(s);
        delete s;
    });
    s->c = c;
    s->nslots = slots;
    s->pool_tokens = pool_tokens;
    s->max_tokens = max_doc_tokens;
    s->sweeps = sweeps;
    s->seed = seed;
    s->proposal = proposal;
    const int K = c->K, M = c->M;
    auto bail = [](int code) { return code; };   // `undo` frees the server
    if ((rc = salloc(s, &s->d_info, slots)) || (rc = salloc(s, &s->d_active, slots)) ||
        (rc = salloc(s, &s->d_z, pool_tokens + 4)) || (rc = salloc(s, &s->d_prop, (pool_tokens + 4) * M)) ||
        (rc = salloc(s, &s->d_words, pool_tokens + 4)) || (rc = salloc(s, &s->d_counter, 8)) ||
        (rc = salloc(s, &s->d_fin_theta, (int64_t)slots * K)) || (rc = salloc(s, &s->d_fin_slot, slots)) ||
        (rc = salloc(s, &s->d_req, slots)) || (rc = salloc(s, &s->d_src, slots)))
        return bail(rc);
    if (proposal == WARPLDA_PROPOSAL_LEARNED &&
        ((rc = salloc(s, &s->d_q, (int64_t)slots * K)) || (rc = salloc(s, &s->d_atab, (int64_t)slots * K)) ||
         (rc = salloc(s, &s->d_aq, (int64_t)slots * K)) || (rc = salloc(s, &s->d_aatab, (int64_t)slots * K))))
        return bail(rc);
    if (host_malloc((void**)&s->h_theta, (size_t)slots * K * 4) != cudaSuccess ||
        host_malloc((void**)&s->h_fin_slot, (size_t)slots * 4) != cudaSuccess)
        return bail(fail(WARPLDA_ENOMEM, "pinned staging"));
    if (cudaEventCreateWithFlags(&s->tick, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(WARPLDA_ECUDA, "event"));
    if (proposal == WARPLDA_PROPOSAL_LEARNED &&
        (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->admitted, cudaEventDisableTiming) != cudaSuccess))
        return bail(fail(WARPLDA_ECUDA, "side stream"));
    s->slots.resize(slots);
    for (int i = slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->free_ranges[0] = pool_tokens;
    s->tab_words = foldin_table_words(K, max_doc_tokens);
    const int per_sm = foldin_blocks_per_sm(K, M, s->tab_words);
    if (per_sm < 1) return bail(fail(WARPLDA_EINVAL, "serving tables do not fit in shared memory"));
    s->grid = per_sm * c->sms;
    undo.armed = false;
    *out = s;
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_server_submit(warplda_server* s, int64_t id, int32_t L, const int32_t* words) try {
    if (!s || L < 0 || (L > 0 && !words)) return fail(WARPLDA_EINVAL, "bad request");
    warplda_ctx* c = s->c;
    if (L > s->max_tokens) return fail(WARPLDA_EINVAL, "request longer than max_doc_tokens");
    for (int32_t j = 0; j < L; ++j)
        if (words[j] < 0 || (int64_t)words[j] >= c->V) return fail(WARPLDA_EINVAL, "word id outside [0, V)");
    if (s->free_slots.empty()) return WARPLDA_EBUSY;
    const int64_t off = pool_take(s, std::max(L, 1));
    if (off < 0) return WARPLDA_EBUSY;   // admission by memory
    const int32_t sl = s->free_slots.back();
    s->free_slots.pop_back();
    auto& S = s->slots[sl];
    S.used = true;
    S.id = id;
    S.off = (int32_t)off;
    S.L = L;
    S.done = 0;
    // staged on the host; the next step uploads every new request at once
    s->new_src.push_back((int32_t)s->new_words.size());
    s->new_words.insert(s->new_words.end(), words, words + L);
    s->new_ptr.push_back((int64_t)s->new_words.size());
    s->new_req.push_back(make_int4(sl, (int)off, L, (int)(uint32_t)id));
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_server_step(warplda_server* s, int32_t* active_out) try {
    if (!s) return fail(WARPLDA_EINVAL, "null server");
    warplda_ctx* c = s->c;
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    if (s->n_fin_staged > 0) return fail(WARPLDA_ESTATE, "poll the previous step's results first");
    // the pinned staging is reused: the previous step's upload must be done
    WL_CU(cudaEventSynchronize(s->tick), "previous step");
    // requests staged since the last step: with the plain proposal they join
    // this step's sweep.  With the learned one their encoder forward and
    // alias tables run on the side stream beside the running requests'
    // sweep, and then either their first sweep follows there (few sweeps per
    // request: a step of delay would be a large part of the latency) or
    // they join the next step (many sweeps: one more step costs little,
    // while a first sweep behind the encoder would lengthen every step)
    const bool learned = s->proposal == WARPLDA_PROPOSAL_LEARNED;
    const bool defer = learned && s->sweeps >= kServeDeferMin;
    std::vector<int32_t> active, fresh;
    if (learned)
        for (const int4& r : s->new_req) fresh.push_back(r.x);
    std::vector<char> is_fresh((size_t)s->nslots, 0);
    for (int32_t i : fresh) is_fresh[i] = 1;
    int nfin = 0;
    for (int i = 0; i < s->nslots; ++i) {
        const auto& S = s->slots[i];
        if (!S.used || S.done >= s->sweeps) continue;
        if (is_fresh[i]) {
            if (!defer && S.done + 1 >= s->sweeps) ++nfin;
            continue;
        }
        active.push_back(i);
        if (S.done + 1 >= s->sweeps) ++nfin;
    }
    if (active_out) *active_out = (int32_t)(active.size() + fresh.size());
    if (active.empty() && fresh.empty()) return WARPLDA_OK;
    // a step lasts as long as its longest document: documents of at least
    // kServeBlockMin tokens are swept by a whole block each.  Upload order:
    // running short, running long, new short, new long.
    const bool blocks = foldin_warps(s->tab_words) >= 4;
    std::vector<int32_t> lists[4];
    for (int32_t i : active) lists[blocks && s->slots[i].L >= kServeBlockMin ? 1 : 0].push_back(i);
    if (!defer)
        for (int32_t i : fresh) lists[blocks && s->slots[i].L >= kServeBlockMin ? 3 : 2].push_back(i);
    std::vector<int32_t> upload;
    for (const auto& l : lists) upload.insert(upload.end(), l.begin(), l.end());
    // counters: short-document work [0] (running) and [2] (new), long
    // [3] and [4], and the shared count of finished rows [1]; zeroed
    // before the side stream is released
    WL_CU(cudaMemsetAsync(s->d_counter, 0, 32, c->st), "reset counters");
    int64_t act_off = 0, sl_off = 0;
    int rc = server_admit(s, upload, &act_off, &sl_off);
    if (rc) return rc;
    FoldArgs f = server_args(s);
    ServeSlots sl{};
    sl.info = s->d_info;
    sl.nslots = s->nslots;
    sl.pool_tokens = s->pool_tokens;
    sl.z = s->d_z;
    sl.prop = s->d_prop;
    sl.words = s->d_words;
    sl.fin_theta = s->d_fin_theta;
    sl.fin_slot = s->d_fin_slot;
    sl.fin_count = s->d_counter + 1;
    sl.q = s->d_q;
    sl.atab = s->d_atab;
    const int warps = foldin_warps(s->tab_words);
    // one launch over a short and a long list starting at `off` in the upload
    auto serve = [&](int which, int64_t off, cudaStream_t st) -> int {
        const int ns = (int)lists[which].size(), nl = (int)lists[which + 1].size();
        if (ns + nl == 0) return WARPLDA_OK;
        FoldArgs fa = f;
        fa.counter = s->d_counter + (which == 0 ? 0 : 2);
        ServeSlots a = sl;
        a.active = s->d_staged + off;
        a.nactive = ns;
        a.long_active = s->d_staged + off + ns;
        a.nlong = nl;
        a.long_counter = s->d_counter + (which == 0 ? 3 : 4);
        a.long_blocks = nl > 0 ? (int)std::min<int64_t>(nl, std::max(1, s->grid / 2)) : 0;
        const int short_blocks = ns > 0 ? (int)std::min<int64_t>(s->grid, ((int64_t)ns + warps - 1) / warps) : 0;
        return launch_timed(c, which == 0 ? kcServe : kcServeNew,
                            [&] { return launch_serve(fa, a, s->tab_words, a.long_blocks + short_blocks, st); }, st);
    };
    if ((rc = serve(0, act_off, c->st))) return rc;
    if (!fresh.empty()) {
        if ((rc = serve(2, act_off + (int64_t)(lists[0].size() + lists[1].size()), s->side))) return rc;
        WL_CU(cudaEventRecord(s->admitted, s->side), "record admission");
        WL_CU(cudaStreamWaitEvent(c->st, s->admitted, 0), "wait admission");
    }
    for (int32_t i : active) s->slots[i].done += 1;
    if (!defer)
        for (int32_t i : fresh) s->slots[i].done += 1;
    if (nfin > 0) {
        WL_CU(cudaMemcpyAsync(s->h_fin_slot, s->d_fin_slot, (size_t)nfin * 4, cudaMemcpyDeviceToHost, c->st), "copy finished");
        WL_CU(cudaMemcpyAsync(s->h_theta, s->d_fin_theta, (size_t)nfin * c->K * 4, cudaMemcpyDeviceToHost, c->st),
              "copy finished");
    }
    s->n_fin_staged = nfin;
    WL_CU(cudaEventRecord(s->tick, c->st), "record tick");
    return WARPLDA_OK;
} WL_ABI_CATCH

int warplda_server_poll(warplda_server* s, int32_t max_results, int64_t* ids, float* theta, int32_t* n_out,
                        int32_t timeout_ms) try {
    if (!s || !n_out || max_results < 0 || (max_results > 0 && (!ids || !theta)))
        return fail(WARPLDA_EINVAL, "bad poll arguments");
    *n_out = 0;
    warplda_ctx* c = s->c;
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    // bounded wait for the last step
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(s->tick);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "serve step");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (ms > timeout_ms) return fail(WARPLDA_ETIMEDOUT, "a serving step did not finish within %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    int rc = check_record(c, "serving");
    if (rc) return rc;
    const int K = c->K, n = s->n_fin_staged;
    if (n > max_results) return fail(WARPLDA_EINVAL, "max_results below the %d finished requests", n);
    for (int i = 0; i < n; ++i) {
        const int32_t sl = s->h_fin_slot[i];
        if (sl < 0 || sl >= s->nslots || !s->slots[sl].used) return fail(WARPLDA_ECUDA, "bad finished slot");
        auto& S = s->slots[sl];
        ids[i] = S.id;
        std::memcpy(theta + (int64_t)i * K, s->h_theta + (int64_t)i * K, (size_t)K * 4);
        pool_give(s, S.off, std::max(S.L, 1));
        S.used = false;
        s->free_slots.push_back(sl);
    }
    s->n_fin_staged = 0;
    *n_out = n;
    return WARPLDA_OK;
} WL_ABI_CATCH

void warplda_server_destroy(warplda_server* s) {
    if (!s) return;
    cudaSetDevice(s->c->dev);
    cudaStreamSynchronize(s->c->st);
    server_free(s);
    delete s;
}

int warplda_sync(warplda_ctx* c) try {
    if (!c) return fail(WARPLDA_EINVAL, "null context");
    WL_CU(cudaSetDevice(c->dev), "cudaSetDevice");
    return check_record(c, "sync");
} WL_ABI_CATCH

void warplda_destroy(warplda_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
}

}  // extern "C"
