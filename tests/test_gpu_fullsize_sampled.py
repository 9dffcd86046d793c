"""Full-size parity on the PubMed-shaped (736M tokens, K=10^4, M=2) and
ClueWeb-shaped (1.5B tokens, K=10^6, M=1, sparse count rows) workloads, in
the launch configuration the benchmark times, on sampled outputs.

From the GPU's own state at the start of a phase, the oracle recomputes that
phase for a sample of documents (the longest ones, which the multi-pass tier
takes, and random ones from the batch tier) or of words (the heaviest ones
and random ones), one segment at a time; the GPU's topics and proposals for
those tokens must match bit for bit.  c_k after each phase must equal the
histogram of z (a property that holds at any size).
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


def _sample(lengths, n_random, n_top, rng):
    nz = np.flatnonzero(lengths > 0)
    top = nz[np.argsort(-lengths[nz], kind="stable")[:n_top]]
    rnd = rng.choice(nz, size=min(n_random, len(nz)), replace=False)
    return np.unique(np.concatenate([top, rnd]))


@pytest.mark.parametrize("name", ["pubmed", "clueweb"])
def test_full_size_sampled_phase_parity(name):
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl = corpus.generate(name, seed=1)
    gpu = WarpLDA(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    gpu.sweep(2)
    z, p, ck, it = gpu.get_state()
    # K above 16,384 uses storage-order word positioning
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7,
                        word_rule=1 if wl.K > 16384 else 0)
    N, M = ref.N, ref.M
    rng = np.random.default_rng(3)

    # document phase of sweep it + 1
    ref.z[:N] = z
    ref.prop[: N * M] = p
    ref.ck[:] = ck
    gpu.phase(1)
    z1, p1, ck1, _ = gpu.get_state()
    assert np.array_equal(ck1, np.bincount(z1, minlength=wl.K)), "c_k after the document phase"
    docs = _sample(np.diff(c.doc_ptr), 3000, 20, rng)
    for d in docs:
        ref.doc_phase(it + 1, int(d), int(d) + 1)
    t = ref.perm[np.concatenate([np.arange(c.doc_ptr[d], c.doc_ptr[d + 1]) for d in docs])]
    assert np.array_equal(z1[t], ref.z[t]), "document phase: z"
    pt = (t[:, None] * M + np.arange(M)).reshape(-1)
    assert np.array_equal(p1[pt], ref.prop[pt]), "document phase: proposals"

    # word phase of the same sweep
    ref.z[:N] = z1
    ref.prop[: N * M] = p1
    ref.ck[:] = ck1
    gpu.phase(2)
    z2, p2, ck2, _ = gpu.get_state()
    assert np.array_equal(ck2, np.bincount(z2, minlength=wl.K)), "c_k after the word phase"
    words = _sample(np.diff(ref.word_ptr), 3000, 5, rng)
    for w in words:
        ref.word_phase(it + 1, int(w), int(w) + 1)
    t = np.concatenate([np.arange(ref.word_ptr[w], ref.word_ptr[w + 1]) for w in words])
    assert np.array_equal(z2[t], ref.z[t]), "word phase: z"
    pt = (t[:, None] * M + np.arange(M)).reshape(-1)
    assert np.array_equal(p2[pt], ref.prop[pt]), "word phase: proposals"
    gpu.sync()


@pytest.fixture(scope="module")
def nytimes_model():
    """A NYTimes-shaped model (99M tokens, K = 1000) after 5 sweeps, with its
    frozen C_w and c_k as the oracle sees them."""
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl = corpus.generate("nytimes", seed=1)
    gpu = WarpLDA(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    gpu.sweep(5)
    z, _, ck, _ = gpu.get_state()   # z in word-major order
    wp, _ = gpu.token_order()
    cw = oracle.word_topic_counts(z, wp, c.V, wl.K)
    yield gpu, c, wl, cw, ck
    gpu.close()


def _oracle_rows(rq, pick, ids, cw, ck, c, wl, sweeps, seed):
    lens = np.diff(rq.doc_ptr)[pick]
    dp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    dw = np.concatenate([rq.doc_word[rq.doc_ptr[d]: rq.doc_ptr[d + 1]] for d in pick]).astype(np.int32)
    return oracle.foldin(dp, dw, cw, ck, wl.K, wl.M, wl.alpha, wl.beta, c.V, seed=seed, sweeps=sweeps,
                         doc_ids=ids[pick])


def test_full_size_foldin_sampled_parity(nytimes_model):
    """Fold-in of 20,000 requests in one call against the NYTimes-shaped
    model, as the benchmark times it: the word-major phases stage the frozen
    rows of the Zipf-frequent words in many pieces.  A request's result
    depends only on its own tokens and stream id, so the oracle's fold-in of
    a sample of the requests (the longest and random ones) must give the
    same rows and topics bit for bit."""
    gpu, c, wl, cw, ck = nytimes_model
    rq = corpus.requests("nytimes", seed=1, n=20000, doc_offset=c.D + 1000)
    ids = np.arange(rq.D, dtype=np.int64) * 3 + 11
    th, zf = gpu.foldin(rq.doc_ptr, rq.doc_word, sweeps=4, seed=23, doc_ids=ids)
    rng = np.random.default_rng(5)
    pick = _sample(np.diff(rq.doc_ptr), 60, 4, rng)
    zo, tho = _oracle_rows(rq, pick, ids, cw, ck, c, wl, 4, 23)
    assert np.array_equal(th[pick], tho)
    zg = np.concatenate([zf[rq.doc_ptr[d]: rq.doc_ptr[d + 1]] for d in pick])
    assert np.array_equal(zg, zo)


def test_full_size_serving_sampled_parity(nytimes_model):
    """Serving against the NYTimes-shaped model: 2,000 requests of 20 to
    5,000 tokens (a block each from 512 tokens on) trickling into a server
    while others run; a sample of the served theta rows, the longest
    requests included, equals the oracle's fold-in rows."""
    from paper_1510_08628_gb300.warplda import Server
    gpu, c, wl, cw, ck = nytimes_model
    rq = corpus.requests("nytimes", seed=1, n=2000, doc_offset=c.D + 50000)
    ids = np.arange(rq.D, dtype=np.int64) * 5 + 2
    srv = Server(gpu, slots=512, pool_tokens=600000, max_doc_tokens=5000, sweeps=6, seed=41)
    got, nxt = {}, 0
    for _ in range(100000):
        for _ in range(37):   # a few dozen arrive before each step
            if nxt < rq.D and srv.submit(int(ids[nxt]), rq.doc_word[rq.doc_ptr[nxt]: rq.doc_ptr[nxt + 1]]):
                nxt += 1
        srv.step()
        done, th = srv.poll()
        for i, t in zip(done, th):
            got[int(i)] = t
        if len(got) == rq.D:
            break
    srv.close()
    assert len(got) == rq.D
    rng = np.random.default_rng(7)
    pick = _sample(np.diff(rq.doc_ptr), 40, 6, rng)
    _, tho = _oracle_rows(rq, pick, ids, cw, ck, c, wl, 6, 41)
    for r, d in enumerate(pick):
        assert np.array_equal(got[int(ids[d])], tho[r]), int(d)
