"""Count invariants, special cases and log-likelihood pins of the oracle.

* Counts (Sec. 2.1): after every phase z and all proposals lie in [0, K),
  c_k is the histogram of z and sums to N, and every token's new assignment is
  its old one or one of the proposals it had pending (an MH step moves only
  to a proposal, Alg. 1).
* K = 1: every assignment is topic 0 and the log-likelihood has the closed
  form of Sec. 6.1 with C_dk = L_d, C_kw = L_w, C_k = N.
* One-word vocabulary: c_w = c_k and beta_bar = beta, so pi^doc = 1 (Eq. 7)
  and the word phase accepts every pending document proposal.
* Log-likelihood (Sec. 6.1): lnG(a + n) - lnG(a) = sum_{i<n} ln(a + i), summed
  here exactly with math.fsum from the counts of z.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1510_08628_gb300 import corpus


def _small(seed=2, K=7, M=2, lens=None, V=60):
    lens = lens if lens is not None else [5, 1, 17, 3, 40, 2, 9, 9, 11]
    c = corpus.from_lengths(lens, V=V, seed=seed)
    return c, oracle.Oracle(c.doc_ptr, c.doc_word, V, K, 0.3, 0.05, M, seed=seed + 9)


def _check_phase_moves(o, before_z, before_p):
    assert o.z.min() >= 0 and o.z.max() < o.K
    assert o.prop.min() >= 0 and o.prop.max() < o.K
    allowed = np.concatenate([before_z[:, None], before_p.reshape(-1, o.M)], axis=1)
    assert np.all((allowed == o.z[:, None]).any(axis=1))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_counts_and_moves_each_phase(M):
    c, o = _small(M=M)
    for it in range(1, 6):
        z0, p0 = o.z.copy(), o.prop.copy()
        o.doc_phase(it)
        _check_phase_moves(o, z0, p0)
        o.recount()
        assert o.ck.sum() == o.N
        assert np.array_equal(o.ck, np.bincount(o.z, minlength=o.K))
        z0, p0 = o.z.copy(), o.prop.copy()
        o.word_phase(it)
        _check_phase_moves(o, z0, p0)
        o.recount()
        assert np.array_equal(o.ck, np.bincount(o.z, minlength=o.K))
        o.iteration = it
    # per-document and per-word counts sum to the segment lengths
    zd = o.z_docmajor()
    for d in range(o.D):
        b, e = o.doc_ptr[d], o.doc_ptr[d + 1]
        assert np.bincount(zd[b:e], minlength=o.K).sum() == e - b


def test_init_sets_proposals_to_z():
    c, o = _small(M=3)
    assert np.array_equal(o.prop.reshape(-1, 3), np.repeat(o.z[:, None], 3, axis=1))


def test_word_major_order_is_stable_sort():
    c, o = _small()
    order = np.argsort(c.doc_word, kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    assert np.array_equal(o.perm[: o.N], inv)
    assert np.array_equal(np.diff(o.word_ptr), np.bincount(c.doc_word, minlength=c.V))


def _ll_bruteforce(o):
    alpha, beta = float(o.alpha), float(o.beta)
    abar, bbar = o.K * alpha, o.V * beta
    terms = []
    zd = o.z_docmajor()
    for d in range(o.D):
        b, e = o.doc_ptr[d], o.doc_ptr[d + 1]
        L = int(e - b)
        terms += [-math.log(abar + i) for i in range(L)]
        for cnt in np.bincount(zd[b:e], minlength=o.K):
            terms += [math.log(alpha + i) for i in range(int(cnt))]
    for w in range(o.V):
        seg = o.z[o.word_ptr[w]:o.word_ptr[w + 1]]
        for cnt in np.bincount(seg, minlength=o.K):
            terms += [math.log(beta + i) for i in range(int(cnt))]
    for ck in np.bincount(o.z[: o.N], minlength=o.K):
        terms += [-math.log(bbar + i) for i in range(int(ck))]
    return math.fsum(terms)


def test_loglik_matches_log_sums():
    c, o = _small(K=5, M=1)
    for _ in range(3):
        o.sweep(1)
        got, want = o.loglik(), _ll_bruteforce(o)
        assert abs(got - want) <= 1e-9 * abs(want)


def test_k1_closed_form():
    c, o = _small(K=1, M=2)
    o.sweep(4)
    assert np.all(o.z[: o.N] == 0) and np.all(o.prop == 0)
    a, b = float(o.alpha), float(o.beta)
    L_d = np.diff(o.doc_ptr)
    L_w = np.diff(o.word_ptr)
    want = sum(math.lgamma(a) - math.lgamma(a + L) + math.lgamma(a + L) - math.lgamma(a)
               for L in L_d)
    want += math.lgamma(o.V * b) - math.lgamma(o.V * b + o.N)
    want += sum(math.lgamma(b + L) - math.lgamma(b) for L in L_w if L > 0)
    assert abs(o.loglik() - want) <= 1e-10 * abs(want)


def test_one_word_vocabulary_accepts_every_doc_proposal():
    lens = [4, 6, 3, 8]
    doc_ptr = np.zeros(len(lens) + 1, dtype=np.int64)
    doc_ptr[1:] = np.cumsum(lens)
    doc_word = np.zeros(int(doc_ptr[-1]), dtype=np.int32)
    o = oracle.Oracle(doc_ptr, doc_word, 1, 9, 0.2, 0.07, 2, seed=5)
    o.sweep(2)
    o.doc_phase(3)            # fresh doc proposals pending
    o.recount()
    p = o.prop.reshape(-1, 2).copy()
    o.word_phase(3)
    assert np.array_equal(o.z[: o.N], p[:, 1])


def test_empty_documents_and_words_are_skipped():
    lens = [3, 0, 5, 0, 0, 2]
    doc_ptr = np.zeros(len(lens) + 1, dtype=np.int64)
    doc_ptr[1:] = np.cumsum(lens)
    doc_word = np.array([0, 4, 4, 1, 1, 4, 0, 0, 4, 1], dtype=np.int32)   # words 2, 3 empty
    o = oracle.Oracle(doc_ptr, doc_word, 5, 4, 0.5, 0.1, 2, seed=8)
    o.sweep(3)
    assert np.array_equal(o.ck, np.bincount(o.z[: o.N], minlength=4))
    assert np.isfinite(o.loglik())


def test_results_do_not_depend_on_thread_count():
    """The oracle's OpenMP loops over documents and words give the same state
    with 1 and with several threads: every random number is keyed by the
    token, and documents (words) of one phase touch disjoint tokens."""
    c, _ = corpus.generate("tiny", seed=3)
    prev = oracle.num_threads()
    try:
        out = []
        for n in (1, max(2, prev)):
            oracle.set_threads(n)
            o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 16, 3.125, 0.01, 2, 11)
            o.sweep(3)
            out.append((o.z.copy(), o.prop.copy(), o.ck.copy()))
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b)
    finally:
        oracle.set_threads(prev)
