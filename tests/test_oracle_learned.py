"""Pins of the oracle's learned-proposal fold-in (orc_alias_build,
orc_alias_draw, orc_foldin_learned).

* The alias table represents q: column k's own probability plus the slack
  every other column aliases to k, over K, equals q_k (to FP32 rounding).
* Alias draws follow q (chi-square).
* The fold-in chain with the independence-sampler rate keeps the target: with
  a uniform, a good (the CGS posterior mean) and a bad (random Dirichlet)
  proposal, the mean theta agrees with a plain collapsed Gibbs fold-in, as the
  plain fold-in does (measured L1 0.022-0.023 mean; a swapped q ratio gives
  0.24-0.47).
* Separable words stay separable.
"""
import numpy as np
from scipy import stats

import oracle
from tests import test_oracle_foldin as fo


def test_alias_table_represents_q():
    rng = np.random.default_rng(0)
    for K in (1, 2, 7, 50, 1000):
        q = rng.dirichlet(np.ones(K) * 0.5).astype(np.float32)
        prob, alias = oracle.alias_table(q)
        assert ((alias >= 0) & (alias < K)).all() and ((prob >= 0) & (prob <= 1)).all()
        implied = prob.astype(np.float64).copy()
        for j in range(K):
            if alias[j] != j:
                implied[alias[j]] += 1.0 - prob[j]
        np.testing.assert_allclose(implied / K, q, atol=2e-6)


def test_alias_draw_law():
    lib = oracle.load()
    rng = np.random.default_rng(1)
    K = 9
    q = np.array([0.3, 0.0, 0.05, 0.15, 0.1, 0.02, 0.18, 0.1, 0.1], dtype=np.float32)
    prob, alias = oracle.alias_table(q)
    n = 50000
    r = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64)
    got = np.array([lib.orc_alias_draw(int(a), int(b), prob, alias, K) for a, b in r])
    obs = np.bincount(got, minlength=K)
    assert obs[1] == 0
    keep = q > 0
    qk = q[keep].astype(np.float64)
    chi = stats.chisquare(obs[keep], qk / qk.sum() * n)
    assert chi.pvalue > 1e-3, chi


def check_learned_against_cgs(mutation=0):
    cw, ck, wl, V = fo.trained_model()
    c = fo.heldout(24)
    K = wl.K
    cgs = oracle.cgs_foldin_theta(c.doc_ptr, c.doc_word, cw, ck, K, wl.alpha, wl.beta, V,
                                  seed=77, sweeps=1200, burn=100)
    rng = np.random.default_rng(0)
    good = (cgs / cgs.sum(axis=1, keepdims=True)).astype(np.float32)
    bad = rng.dirichlet(np.ones(K) * 0.3, size=c.D).astype(np.float32)
    for q in (good, bad):
        acc = np.zeros((c.D, K))
        R = 48
        for r in range(R):
            _, th = oracle.foldin_learned(c.doc_ptr, c.doc_word, cw, ck, q, K, 2, wl.alpha,
                                          wl.beta, V, seed=1000 + r, sweeps=25, mutation=mutation)
            acc += th
        l1 = np.abs(acc / R - cgs).sum(axis=1)
        assert l1.mean() < 0.05 and l1.max() < 0.08, (l1.mean(), l1.max())


def test_learned_foldin_matches_collapsed_gibbs():
    check_learned_against_cgs()


def test_learned_separable_words():
    K = V = 4
    cw = np.eye(K, dtype=np.int32) * 1000
    ck = cw.sum(axis=0).astype(np.int32)
    rng = np.random.default_rng(3)
    lens = rng.integers(5, 40, size=30)
    dp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    dw = rng.integers(0, V, size=int(dp[-1])).astype(np.int32)
    q = rng.dirichlet(np.ones(K), size=30).astype(np.float32)
    z, th = oracle.foldin_learned(dp, dw, cw, ck, q, K, 2, 0.5, 0.01, V, seed=5, sweeps=20)
    assert (z == dw).mean() > 0.98
    np.testing.assert_allclose(th.sum(axis=1), 1.0, rtol=1e-5)
