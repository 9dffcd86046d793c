"""Whole-sampler pin: the oracle's WarpLDA reaches the log-likelihood of a plain
collapsed Gibbs sampler (Eq. 1), as Sec. 6.3 reports for MCEM against CGS, and
M = 2 converges no slower per iteration than M = 1 (Sec. 6.3, impact of M).

Corpus: the first 400 documents of the ``tiny`` workload (K = 16, alpha = 50/K,
beta = 0.01), four seeds each.  Tolerance on the final mean log-likelihood:
max(3 standard errors, 0.5% of |LL|).
"""
import numpy as np
import pytest

import oracle
from paper_1510_08628_gb300 import corpus

ITERS = 500
SEEDS = [100, 101, 102, 103]


@pytest.fixture(scope="module")
def runs():
    c, wl = corpus.generate("tiny", seed=1, D=400)
    lib = oracle.load()
    out = {"w1": [], "w2": [], "cgs": [], "w1_early": [], "w2_early": []}
    for s in SEEDS:
        o1 = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 16, wl.alpha, 0.01, 1, seed=s)
        o2 = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 16, wl.alpha, 0.01, 2, seed=s)
        oc = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 16, wl.alpha, 0.01, 1, seed=s)
        o1.sweep(60)
        o2.sweep(60)
        out["w1_early"].append(o1.loglik())
        out["w2_early"].append(o2.loglik())
        o1.sweep(ITERS - 60)
        o2.sweep(ITERS - 60)
        lib.orc_cgs_sweeps(oc.D, oc.V, oc.doc_ptr, oc.doc_word, oc.perm, 16, oc.alpha, oc.beta,
                           s, 0, ITERS, oc.z)
        out["w1"].append(o1.loglik())
        out["w2"].append(o2.loglik())
        out["cgs"].append(oc.loglik())
    return {k: np.array(v) for k, v in out.items()}


@pytest.mark.slow
def test_warplda_reaches_cgs_loglik(runs):
    a, b = runs["w1"], runs["cgs"]
    se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    tol = max(3 * se, 0.005 * abs(b.mean()))
    assert abs(a.mean() - b.mean()) <= tol, (a, b)


@pytest.mark.slow
def test_more_mh_steps_converge_no_slower(runs):
    a, b = runs["w1_early"], runs["w2_early"]
    se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    assert b.mean() >= a.mean() - 3 * se, (a, b)


def test_topic_recovery_against_the_generator():
    """Soft check: after 150 sweeps on the tiny workload (K_true = K = 16) the
    oracle's topics phi_k = (C_kw + beta) / (C_k + V beta) (Eq. 4) match the
    generator's true rows after Hungarian matching on the Hellinger distance
    far better than an arbitrary pairing does."""
    from scipy.optimize import linear_sum_assignment
    wl = corpus.WORKLOADS["tiny"]
    model = corpus.TopicModel(wl.V, wl.K_true, wl.zipf_s, wl.conc_c, 1, keep_phi=True)
    lens = corpus.lengths(wl.D, wl.len_kind, wl.len_mean, wl.len_sigma, 1)
    c = corpus.generate_docs(model, lens, wl.doc_alpha, 1)
    phi = model.phi.reshape(wl.K_true, wl.V)
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    o.sweep(150)
    cw = oracle.word_topic_counts(o.z[: o.N], o.word_ptr, c.V, wl.K).astype(np.float64)
    est = (cw.T + wl.beta) / (cw.sum(axis=0)[:, None] + c.V * wl.beta)
    H = np.sqrt(0.5 * ((np.sqrt(est)[:, None, :] - np.sqrt(phi)[None, :, :]) ** 2).sum(-1))
    r, k = linear_sum_assignment(H)
    matched = H[r, k].mean()
    arbitrary = H[np.arange(wl.K), np.random.default_rng(0).permutation(wl.K_true)].mean()
    assert matched < 0.5 and arbitrary > 0.7 and matched < 0.7 * arbitrary, (matched, arbitrary)
