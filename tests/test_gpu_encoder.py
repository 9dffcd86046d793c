"""The fold-in encoder on the GPU (hand-written layer-1 gather kernels,
tcgen05 layer 2) against the FP64 NumPy oracle (oracle/encoder.py, rounding
to BF16 where the device does), and the learned-proposal fold-in against the
oracle's orc_foldin_learned, bit for bit, on the proposal rows the device
produced."""
import numpy as np
import pytest

import oracle
from oracle import encoder as enc
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
    K = 40
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, 2, 5)
    g.sweep(4)
    g.encoder_init(log2_features=10, hidden=128, batch_rows=128, seed=9)
    return g, c, wl, K


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def test_gradients_match_oracle(model):
    g, c, wl, K = model
    rng = np.random.default_rng(0)
    Dn = 100
    dp = c.doc_ptr[: Dn + 1]
    dw = c.doc_word[: int(dp[-1])]
    theta = rng.dirichlet(np.ones(K) * 0.5, size=Dn).astype(np.float32)
    W1, b1, W2, b2 = g.encoder_weights()
    loss, (gW1, gb1, gW2, gb2) = g.encoder_grad(dp, dw, theta)
    p = {"W1": W1.astype(np.float64), "b1": b1.astype(np.float64), "W2": W2.astype(np.float64),
         "b2": b2.astype(np.float64)}
    x = enc.inputs(dp, dw, 10)
    want_loss, want = enc.backward(p, x, theta.astype(np.float64), bf=True)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    assert _rel(gb2, want["b2"]) < 1e-4
    for got, key in ((gW2, "W2"), (gW1, "W1"), (gb1, "b1")):
        # BF16 rounding of dlogits can flip by one unit between FP32 and FP64
        assert _rel(got, want[key]) < 2e-2, key
        close = np.abs(got - want[key]) <= 1e-3 * np.abs(want[key]).max()
        assert close.mean() > 0.99, key


def test_proposal_rows(model):
    g, c, wl, K = model
    Dn = 50
    dp = c.doc_ptr[: Dn + 1]
    dw = c.doc_word[: int(dp[-1])]
    q = g.encoder_proposal(dp, dw)
    np.testing.assert_allclose(q.sum(axis=1), 1.0, rtol=1e-5)
    W1, b1, W2, b2 = g.encoder_weights()
    p = {"W1": W1, "b1": b1, "W2": W2, "b2": b2}
    want = enc.forward(p, enc.inputs(dp, dw, 10), bf=True)["q"]
    assert np.abs(q - want).max() < 1e-4


def test_learned_foldin_bit_exact(model):
    g, c, wl, K = model
    rq = corpus.requests("tiny", seed=3, n=40, doc_offset=9000, lo=1, hi=400)
    q = g.encoder_proposal(rq.doc_ptr, rq.doc_word)
    th, z = g.foldin(rq.doc_ptr, rq.doc_word, sweeps=5, seed=17, learned=True)
    zg, _, ck, _ = g.get_state()
    wp, perm = g.token_order()
    cw = oracle.word_topic_counts(zg, wp, c.V, K)
    zo, tho = oracle.foldin_learned(rq.doc_ptr, rq.doc_word, cw, ck, q, K, 2, wl.alpha, wl.beta,
                                    c.V, seed=17, sweeps=5)
    assert np.array_equal(z, zo), np.flatnonzero(z != zo)[:10]
    assert np.array_equal(th, tho)


def test_training_lowers_the_loss(model):
    g, c, wl, K = model
    losses = g.encoder_train(epochs=4, lr=3e-3, seed=2)
    assert np.isfinite(losses).all()
    assert losses[-1] < losses[0], losses
