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
