"""Host logic of bench.py: the algorithmic byte counts behind the roofline
(Sec. 5.2 layout: per token per sweep the document phase reads perm and reads
and writes z and M proposals, the word phase reads and writes them) and the
--tuning parser."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_bytes_per_token():
    assert bench.sweep_alg_bytes(1) == 36 and bench.sweep_alg_bytes(2) == 52
    for M in (1, 2, 3, 4):
        doc = bench.alg_bytes_per_token("doc_batch", M)
        word = bench.alg_bytes_per_token("word_batch", M)
        assert doc == 4 + 8 * (M + 1) and word == 8 * (M + 1)
        assert doc + word == bench.sweep_alg_bytes(M)
    assert bench.alg_bytes_per_token("finalize_ck", 2) == 0


def test_tuning_parser():
    assert bench.parse_tuning("") is None
    assert bench.parse_tuning("doc_warp_max=256, batch_max_tokens=64") == {
        "doc_warp_max": 256, "batch_max_tokens": 64}
    for bad in ("nope=1", "doc_warp_max", "doc_warp_max=", "huge_chunk=x"):
        with pytest.raises((SystemExit, ValueError)):
            bench.parse_tuning(bad)


def test_foldin_objective_is_its_definition():
    """Mean of log p(w, z | frozen model) per token, written out term by term."""
    import math
    import numpy as np
    rng = np.random.default_rng(3)
    K, V, alpha, beta = 5, 7, 0.3, 0.02
    bbar = float(np.float32(V) * np.float32(beta))
    optr = np.array([0, 4, 4, 9, 10])
    N = int(optr[-1])
    owords = rng.integers(0, V, size=N)
    z = rng.integers(0, K, size=N)
    cw = rng.integers(0, 9, size=(V, K)).astype(np.int32)
    ck = cw.sum(axis=0).astype(np.int32)
    want = 0.0
    for d in range(len(optr) - 1):
        zd = z[optr[d]: optr[d + 1]]
        want += math.lgamma(K * alpha) - math.lgamma(K * alpha + len(zd))
        for k in range(K):
            want += math.lgamma(alpha + np.sum(zd == k)) - math.lgamma(alpha)
    for i in range(N):
        want += math.log((cw[owords[i], z[i]] + beta) / (ck[z[i]] + bbar))
    got = bench.foldin_objective(z, optr, owords, cw, ck, K, alpha, beta, bbar)
    assert abs(got - want / N) <= 1e-12 * abs(want / N)


def test_theta_entropy_is_the_mean_entropy_of_eq4_theta():
    import numpy as np
    rng = np.random.default_rng(4)
    K, alpha = 6, 0.25
    doc_ptr = np.array([0, 3, 3, 10, 12])
    z = rng.integers(0, K, size=12).astype(np.int32)

    class Fake:
        def counts(self, want_ck=True):
            return z, None

    class C:
        pass
    c = C()
    c.D, c.doc_ptr = 4, doc_ptr

    class W:
        pass
    wl = W()
    wl.K, wl.alpha = K, alpha
    hs = []
    for d in range(4):
        zd = z[doc_ptr[d]: doc_ptr[d + 1]]
        if len(zd) == 0:
            continue
        th = (np.bincount(zd, minlength=K) + alpha) / (len(zd) + K * alpha)
        hs.append(-(th * np.log(th)).sum())
    assert abs(bench.theta_entropy(Fake(), c, wl) - np.mean(hs)) < 1e-12


def test_signal_bounds_on_the_tiny_workload():
    """The generator's own topics predict held-out words better than the
    unigram model on the tiny workload's well-separated topics."""
    from paper_1510_08628_gb300 import corpus
    c, wl = corpus.generate("tiny", seed=1)
    rq = corpus.requests("tiny", seed=1, n=200, doc_offset=c.D + 700_000)
    sb = bench.signal_bounds(c, wl, "tiny", 1, rq, c.D + 700_000)
    assert sb["true_model_ceiling"] > sb["unigram"] + 0.5
    assert sb["unigram"] < 0 and sb["true_model_ceiling"] < 0
