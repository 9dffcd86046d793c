"""Continuous batching of fold-in requests (warplda_server_*): every request's
theta equals warplda_foldin's for the same document id, seed and proposal,
bit for bit -- alone, in a batch, and when requests arrive while others are
half-way through their sweeps; admission is by slots and pool memory."""
import numpy as np
import pytest

from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl = corpus.generate("tiny", seed=3, D=600)
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, wl.alpha, wl.beta, 2, 5)
    g.sweep(5)
    g.encoder_init(log2_features=10, hidden=128, batch_rows=128, seed=9)
    g.encoder_train(epochs=3, lr=3e-3, seed=2)
    rq = corpus.requests("tiny", seed=3, n=60, doc_offset=9000, lo=1, hi=700)
    return g, rq


def _docs(rq, idx):
    return [rq.doc_word[rq.doc_ptr[d]: rq.doc_ptr[d + 1]] for d in idx]


def _serve(g, rq, order, batches, learned, sweeps=7, slots=64, pool=100000):
    from paper_1510_08628_gb300.warplda import Server
    s = Server(g, slots=slots, pool_tokens=pool, max_doc_tokens=700, sweeps=sweeps, seed=31,
               learned=learned)
    out = {}
    pending = list(order)
    it = 0
    while len(out) < len(order):
        # `batches[it]` more requests arrive before step `it`
        take = batches[it] if it < len(batches) else len(pending)
        for _ in range(take):
            if pending and s.submit(pending[0], _docs(rq, [pending[0]])[0]):
                pending.pop(0)
        s.step()
        ids, th = s.poll()
        for i, t in zip(ids, th):
            out[int(i)] = t
        it += 1
        assert it < 10000
    s.close()
    return out


@pytest.mark.parametrize("learned", [False, True])
def test_served_equals_foldin_alone_and_mixed(model, learned):
    g, rq = model
    n = rq.D
    want, _ = g.foldin(rq.doc_ptr, rq.doc_word, sweeps=7, seed=31, learned=learned,
                       doc_ids=np.arange(n))
    all_at_once = _serve(g, rq, list(range(n)), [n], learned)
    trickle = _serve(g, rq, list(range(n))[::-1], [3, 0, 5, 1, 0, 0, 7, 2] * 20, learned)
    for d in range(n):
        assert np.array_equal(all_at_once[d], want[d]), d
        assert np.array_equal(trickle[d], want[d]), d
    # one request alone
    alone = _serve(g, rq, [17], [1], learned)
    assert np.array_equal(alone[17], want[17])


def test_admission_by_memory(model):
    from paper_1510_08628_gb300.warplda import Server
    g, rq = model
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
