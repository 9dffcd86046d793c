"""GPU fold-in (warplda_foldin) against the oracle's fold-in, through the C ABI.

The model is the state a GPU context reaches after some sweeps (bit-exact
with the oracle's, checked in test_gpu_parity.py); its C_w and c_k are taken
from the oracle's copy of that state.  z (integers) and theta (one FP32 add
and one IEEE division per entry on both sides) must match exactly, for dense
and hash count tables, M = 1..4, empty, one-token and long documents, and
caller-given document ids.
"""
import numpy as np
import pytest

import oracle
from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300 import warplda
    warplda.load()


def _model(K, M, sweeps, seed=5, D=400):
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl = corpus.generate("tiny", seed=3, D=D)
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, M, seed)
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, M, seed)
    g.sweep(sweeps)
    o.sweep(sweeps)
    cw = oracle.word_topic_counts(o.z[: o.N], o.word_ptr, c.V, K)
    return g, o, cw, c, wl


def _docs(V, lens, seed=1):
    rng = np.random.default_rng(seed)
    dp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    dw = rng.integers(0, V, size=int(dp[-1])).astype(np.int32)
    return dp, dw


@pytest.mark.parametrize("K,M", [(16, 1), (40, 2), (1000, 3), (3000, 2), (5, 4)])
def test_foldin_matches_oracle(K, M):
    g, o, cw, c, wl = _model(K, M, sweeps=3)
    lens = [0, 1, 2, 31, 32, 33, 97, 250, 1, 0, 600] + ([5000] if K <= 2048 else [4095])
    dp, dw = _docs(c.V, lens)
    ids = np.arange(len(lens), dtype=np.int64) * 7 + 3
    th, z = g.foldin(dp, dw, sweeps=6, seed=99, doc_ids=ids)
    zo, tho = oracle.foldin(dp, dw, cw, o.ck, K, M, wl.alpha, wl.beta, c.V, seed=99, sweeps=6,
                            doc_ids=ids)
    assert np.array_equal(z, zo), np.flatnonzero(z != zo)[:10]
    assert np.array_equal(th, tho)


def test_foldin_independent_of_batch_and_model_refresh():
    g, o, cw, c, wl = _model(40, 2, sweeps=2)
    dp, dw = _docs(c.V, [12, 80, 5, 300], seed=4)
    th_all, z_all = g.foldin(dp, dw, sweeps=5, seed=7, doc_ids=[10, 11, 12, 13])
    b, e = dp[1], dp[2]
    th1, z1 = g.foldin(np.array([0, e - b]), dw[b:e], sweeps=5, seed=7, doc_ids=[11])
    assert np.array_equal(z1, z_all[b:e]) and np.array_equal(th1[0], th_all[1])
    # after more training the next fold-in uses the new counts
    g.sweep(2)
    o.sweep(2)
    cw2 = oracle.word_topic_counts(o.z[: o.N], o.word_ptr, c.V, 40)
    th2, z2 = g.foldin(dp, dw, sweeps=5, seed=7, doc_ids=[10, 11, 12, 13])
    zo, tho = oracle.foldin(dp, dw, cw2, o.ck, 40, 2, wl.alpha, wl.beta, c.V, seed=7, sweeps=5,
                            doc_ids=[10, 11, 12, 13])
    assert np.array_equal(z2, zo) and np.array_equal(th2, tho)
    g.sync()


def test_foldin_rejects_bad_input():
    from paper_1510_08628_gb300.warplda import WarpLDAError
    g, o, cw, c, wl = _model(3000, 1, sweeps=1, D=100)
    with pytest.raises(WarpLDAError):
        g.foldin(np.array([0, 3]), np.array([0, 1, c.V], np.int32), sweeps=2, seed=1)
    with pytest.raises(WarpLDAError):   # hash tables: at most 4095 tokens
        dp, dw = _docs(c.V, [4096])
        g.foldin(dp, dw, sweeps=1, seed=1)
    th, z = g.foldin(np.array([0]), np.zeros(0, np.int32), sweeps=3, seed=1)
    assert th.shape == (0, 3000) and z.shape == (0,)


def test_word_counts_match_oracle():
    g, o, cw, c, wl = _model(40, 2, sweeps=3)
    assert np.array_equal(g.word_counts(), cw)


def _skewed_docs(V, lens, hot, exact, absent, seed=2):
    """Documents whose tokens are mostly a few hot words (each fills several
    256-token pieces of the word-major word phase), words with exactly the
    token counts in `exact` (around the staging threshold of 64 request
    tokens), one word absent from the training corpus (L_w = 0) with 100
    tokens, and uniform other words."""
    rng = np.random.default_rng(seed)
    dp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(dp[-1])
    special = set(hot) | set(exact) | {absent}
    others = np.array([w for w in range(V) if w not in special], np.int32)
    dw = others[rng.integers(0, len(others), size=n)]
    pos = rng.permutation(n)
    k = 0
    for w, m in list(exact.items()) + [(absent, 100)]:
        dw[pos[k: k + m]] = w
        k += m
    rest = pos[k:]
    hot_pos = rest[rng.random(len(rest)) < 0.6]
    dw[hot_pos] = rng.choice(np.array(hot, np.int32), size=len(hot_pos))
    return dp, dw.astype(np.int32)


@pytest.mark.parametrize("K,M", [(16, 2), (1000, 1), (2048, 4), (3000, 3)])
def test_word_major_foldin_staged_and_direct_words(K, M):
    """The word-major fold-in (the default) against the oracle and against
    the one-warp-per-document kernel (tuning foldin_kernel = 1): hot words
    over several pieces (their frozen row staged in shared memory, K <=
    2048), words just below and above the staging threshold, a word with no
    training tokens, empty and long documents; K = 3000 stages nothing."""
    from paper_1510_08628_gb300.warplda import WarpLDA
    g, o, cw, c, wl = _model(K, M, sweeps=3)
    cnt = np.diff(o.word_ptr)
    order = np.argsort(-cnt, kind="stable")
    hot = [int(w) for w in order[:3]]
    absent = int(np.flatnonzero(cnt == 0)[0])
    exact = {int(order[10]): 63, int(order[11]): 64, int(order[12]): 65, int(order[13]): 257}
    lens = [0, 1, 300, 2000, 7, 0, 640, 95, 1500, 33] + ([5000] if K <= 2048 else [4095])
    dp, dw = _skewed_docs(c.V, lens, hot, exact, absent)
    ids = np.arange(len(lens), dtype=np.int64) * 11 + 5
    th, z = g.foldin(dp, dw, sweeps=5, seed=31, doc_ids=ids)
    zo, tho = oracle.foldin(dp, dw, cw, o.ck, K, M, wl.alpha, wl.beta, c.V, seed=31, sweeps=5,
                            doc_ids=ids)
    assert np.array_equal(z, zo), np.flatnonzero(z != zo)[:10]
    assert np.array_equal(th, tho)
    # the same model under the per-document kernel
    c2, _ = corpus.generate("tiny", seed=3, D=400)
    g1 = WarpLDA(c2.doc_ptr, c2.doc_word, c2.V, K, wl.alpha, wl.beta, M, 5, tuning={"foldin_kernel": 1})
    g1.sweep(3)
    th1, z1 = g1.foldin(dp, dw, sweeps=5, seed=31, doc_ids=ids)
    assert np.array_equal(z1, z) and np.array_equal(th1, th)
    # no theta requested, and zero sweeps
    _, z2 = g.foldin(dp, dw, sweeps=5, seed=31, doc_ids=ids, theta=False)
    assert np.array_equal(z2, z)
    th0, z0 = g.foldin(dp, dw, sweeps=0, seed=31, doc_ids=ids)
    zo0, tho0 = oracle.foldin(dp, dw, cw, o.ck, K, M, wl.alpha, wl.beta, c.V, seed=31, sweeps=0,
                              doc_ids=ids)
    assert np.array_equal(z0, zo0) and np.array_equal(th0, tho0)
    g.close()
    g1.close()


def test_foldin_kernel_tuning_is_checked():
    from paper_1510_08628_gb300.warplda import WarpLDA, WarpLDAError
    c, wl = corpus.generate("tiny", seed=3, D=50)
    with pytest.raises(WarpLDAError):
        WarpLDA(c.doc_ptr, c.doc_word, c.V, 16, wl.alpha, wl.beta, 2, 1, tuning={"foldin_kernel": 3})
