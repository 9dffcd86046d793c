"""The seeded synthetic corpora (input generator only, no sampler arithmetic):
deterministic, shaped as stated, and the truncated topic rows of the
ClueWeb-shaped vocabulary keep the entries they claim to keep."""
import numpy as np

from paper_1510_08628_gb300 import corpus


def test_generation_is_deterministic_and_prefix_stable():
    a, wl = corpus.generate("tiny", seed=4)
    b, _ = corpus.generate("tiny", seed=4)
    assert np.array_equal(a.doc_ptr, b.doc_ptr) and np.array_equal(a.doc_word, b.doc_word)
    p, _ = corpus.generate("tiny", seed=4, D=100)          # first 100 documents, same streams
    assert np.array_equal(p.doc_ptr, a.doc_ptr[:101])
    assert np.array_equal(p.doc_word, a.doc_word[: a.doc_ptr[100]])
    assert a.D == wl.D and a.doc_word.min() >= 0 and a.doc_word.max() < wl.V
    assert np.all(np.diff(a.doc_ptr) >= 1)                 # no empty documents (R14)


def test_lognormal_lengths_have_the_stated_mean():
    L = corpus.lengths(200_000, 1, 330.0, 0.8, seed=2)
    assert abs(L.mean() / 330.0 - 1) < 0.01
    r = corpus.lengths(50_000, 1, 92.0, 0.8, seed=2, lo=20, hi=5000)
    assert r.min() >= 1


def test_truncated_topic_rows():
    V, Kt, cut = 20_000, 5, 1e-9
    m = corpus.SparseTopicModel(V, Kt, 1.1, 0.01, seed=3, cut=cut)
    assert m.off[0] == 0 and np.all(np.diff(m.off) > 0)
    for k in range(Kt):
        w = m.words[m.off[k]: m.off[k + 1]]
        pr = m.prob[m.off[k]: m.off[k + 1]].astype(np.float64)
        al = m.alias[m.off[k]: m.off[k + 1]]
        n = len(w)
        assert len(np.unique(w)) == n and w.min() >= 0 and w.max() < V
        # the alias table's implied probabilities sum to one, and every
        # kept entry carries at least the cut (renormalised) of the mass
        q = pr / n
        np.add.at(q, al, (1.0 - pr) / n)
        assert abs(q.sum() - 1.0) < 1e-6
        assert q.min() >= cut * 0.999
    # words of a corpus drawn from truncated rows stay in each row's support
    lens = np.full(200, 50, dtype=np.int64)
    c = corpus.generate_docs(m, lens, 0.1, seed=3, keep_z=True)
    for k in range(Kt):
        sup = set(m.words[m.off[k]: m.off[k + 1]].tolist())
        assert set(c.doc_word[c.true_z == k].tolist()) <= sup
