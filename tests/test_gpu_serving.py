"""Continuous batching of fold-in requests (warplda_server_*) against the
oracle's fold-in.

Every served theta row must equal, bit for bit, the row the CPU oracle's
fold-in (oracle.foldin, or oracle.foldin_learned with the encoder rows the
device computes for the same documents) gives for the same document id, seed
and number of sweeps -- whether the requests arrive all at once, trickle in
while others are half-way through their sweeps, or come alone, and for
documents of 0 to 5,000 tokens in one mix.  theta_dk = (C_dk + alpha) /
(L_d + alpha_bar) is one FP32 add and one IEEE division per entry, so equal
rows mean equal per-document counts C_d.  The frozen model (C_w, c_k) is the
oracle's own state after the same training sweeps; admission is by slots and
pool memory.
"""
import numpy as np
import pytest

import oracle
from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu

SWEEPS, SEED = 7, 31


@pytest.fixture(scope="module", params=[40, 3000], ids=["dense", "hash"])
def model(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300.warplda import WarpLDA
    K, M, train = request.param, 2, 5
    c, wl = corpus.generate("tiny", seed=3, D=600)
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, M, 5)
    g.sweep(train)
    g.encoder_init(log2_features=10, hidden=128, batch_rows=128, seed=9)
    g.encoder_train(epochs=3, lr=3e-3, seed=2)
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, M, 5)
    o.sweep(train)
    cw = oracle.word_topic_counts(o.z[: o.N], o.word_ptr, c.V, K)
    rq = corpus.requests("tiny", seed=3, n=60, doc_offset=9000, lo=1, hi=700)
    yield {"g": g, "c": c, "wl": wl, "K": K, "M": M, "cw": cw, "ck": o.ck.copy(), "rq": rq}
    g.close()


def _docs(rq, idx):
    return [rq.doc_word[rq.doc_ptr[d]: rq.doc_ptr[d + 1]] for d in idx]


def _oracle_theta(m, dp, dw, learned):
    """Oracle fold-in of the requests (ids 0..Dn-1): theta [Dn, K]."""
    c, wl, K, M = m["c"], m["wl"], m["K"], m["M"]
    ids = np.arange(len(dp) - 1, dtype=np.int64)
    if learned:
        q = m["g"].encoder_proposal(dp, dw)
        _, th = oracle.foldin_learned(dp, dw, m["cw"], m["ck"], q, K, M, wl.alpha, wl.beta, c.V,
                                      seed=SEED, sweeps=SWEEPS, doc_ids=ids)
    else:
        _, th = oracle.foldin(dp, dw, m["cw"], m["ck"], K, M, wl.alpha, wl.beta, c.V, seed=SEED,
                              sweeps=SWEEPS, doc_ids=ids)
    return th


def _serve(g, docs, order, batches, learned, max_doc=700, slots=64, pool=100000, sweeps=SWEEPS):
    from paper_1510_08628_gb300.warplda import Server
    s = Server(g, slots=slots, pool_tokens=pool, max_doc_tokens=max_doc, sweeps=sweeps, seed=SEED,
               learned=learned)
    out = {}
    pending = list(order)
    it = 0
    while len(out) < len(order):
        # `batches[it]` more requests arrive before step `it`
        take = batches[it] if it < len(batches) else len(pending)
        for _ in range(take):
            if pending and s.submit(pending[0], docs[pending[0]]):
                pending.pop(0)
        s.step()
        ids, th = s.poll()
        for i, t in zip(ids, th):
            out[int(i)] = t
        it += 1
        assert it < 10000
    s.close()
    return out


@pytest.mark.parametrize("learned", [False, True], ids=["plain", "learned"])
def test_served_equals_oracle_alone_and_mixed(model, learned):
    g, rq = model["g"], model["rq"]
    n = rq.D
    want = _oracle_theta(model, rq.doc_ptr, rq.doc_word, learned)
    docs = _docs(rq, range(n))
    all_at_once = _serve(g, docs, list(range(n)), [n], learned)
    trickle = _serve(g, docs, list(range(n))[::-1], [3, 0, 5, 1, 0, 0, 7, 2] * 20, learned)
    for d in range(n):
        assert np.array_equal(all_at_once[d], want[d]), d
        assert np.array_equal(trickle[d], want[d]), d
    alone = _serve(g, docs, [17], [1], learned)
    assert np.array_equal(alone[17], want[17])


@pytest.mark.parametrize("learned", [False, True], ids=["plain", "learned"])
def test_served_mix_of_empty_and_long_documents(model, learned):
    """Requests of 0, 1 and the longest allowed (5,000 tokens; 4,095 with
    hash count tables) among ordinary ones, arriving while others run: each
    theta row equals the oracle's."""
    g, c = model["g"], model["c"]
    rng = np.random.default_rng(11)
    top = 5000 if model["K"] <= 2048 else 4095
    lens = [0, top, 3, 0, 1, 250, top, 40, 0, 777]
    dp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    dw = rng.integers(0, c.V, size=int(dp[-1])).astype(np.int32)
    want = _oracle_theta(model, dp, dw, learned)
    docs = [dw[dp[d]: dp[d + 1]] for d in range(len(lens))]
    got = _serve(g, docs, [5, 0, 1, 9, 2, 3, 4, 6, 7, 8], [2, 0, 1, 3, 0, 4], learned,
                 max_doc=top, slots=8, pool=20000)
    for d in range(len(lens)):
        assert np.array_equal(got[d], want[d]), (d, lens[d])


@pytest.mark.parametrize("learned", [False, True], ids=["plain", "learned"])
def test_served_with_many_sweeps_equals_foldin(model, learned):
    """12 sweeps per request: learned requests then join the step after
    their admission (with fewer than 8 sweeps, as above, the step of it).
    Rows equal warplda_foldin's (itself checked against the oracle), for
    requests arriving all at once and trickled in."""
    g, rq = model["g"], model["rq"]
    n = rq.D
    want, _ = g.foldin(rq.doc_ptr, rq.doc_word, sweeps=12, seed=SEED, doc_ids=np.arange(n), learned=learned)
    docs = _docs(rq, range(n))
    for order, batches in ((list(range(n)), [n]), (list(range(n))[::-1], [3, 0, 5, 1, 0, 0, 7, 2] * 20)):
        got = _serve(g, docs, order, batches, learned, sweeps=12)
        for d in range(n):
            assert np.array_equal(got[d], want[d]), d


def test_served_equals_context_foldin(model):
    """The serving loop and warplda_foldin give the same rows (both are also
    compared with the oracle above)."""
    g, rq = model["g"], model["rq"]
    want, _ = g.foldin(rq.doc_ptr, rq.doc_word, sweeps=SWEEPS, seed=SEED,
                       doc_ids=np.arange(rq.D))
    got = _serve(g, _docs(rq, range(rq.D)), list(range(rq.D)), [rq.D], False)
    for d in range(rq.D):
        assert np.array_equal(got[d], want[d]), d


def test_admission_by_memory(model):
    from paper_1510_08628_gb300.warplda import Server
    g, rq = model["g"], model["rq"]
    docs = _docs(rq, range(10))
    lens = [len(d) for d in docs]
    s = Server(g, slots=8, pool_tokens=max(lens) + 5, max_doc_tokens=700, sweeps=2, seed=1)
    big = int(np.argmax(lens))
    assert s.submit(big, docs[big])
    other = next(i for i in range(10) if i != big and lens[i] > 5)
    assert not s.submit(other, docs[other])        # pool full: EBUSY
    s.step(); s.step()
    ids, th = s.poll()
    assert list(ids) == [big]
    assert s.submit(other, docs[other])            # memory freed
    s.close()
