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
    """Every gradient entry against the FP64 oracle within a bound of its own.

    The device sums in FP32 and rounds h (before layer 2) and dlogits (before
    the backward products) to BF16.  Each entry's bound is the FP32 error of
    its sum, plus one BF16 step for every rounding in that sum whose FP64
    value lies within the device's FP32 error of a rounding boundary (the
    device may have rounded it the other way), and the whole term for every
    ReLU whose input lies within that error of zero.  Most entries meet no
    such rounding, so their bound is the accumulation error alone: a wrong
    index in any row or column shows."""
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
    th = theta.astype(np.float64)
    want_loss, want = enc.backward(p, x, th, bf=True)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)

    f = enc.forward(p, x, bf=True)
    W1b, W2b, hp, hb, q = f["W1"], f["W2"], f["h_pre"], f["hb"], f["q"]
    u32 = 2.0 ** -24
    acc = 3e-5          # FP32 sums of up to a few hundred terms, relative to the sum of |terms|
    # h_pre: the device's FP32 error; the BF16 steps h may have taken
    e_h = 1e-5 * (np.abs(p["b1"]) + x @ np.abs(W1b))
    s_h = np.abs(enc.bf16(np.maximum(hp + e_h, 0.0)) - enc.bf16(np.maximum(hp - e_h, 0.0)))
    # logits, q and dlogits: those steps plus FP32 error; the BF16 steps of dlogits
    e_lg = s_h @ np.abs(W2b) + 1e-5 * (np.abs(p["b2"]) + hb @ np.abs(W2b))
    e_q = q * (e_lg + e_lg.max(axis=1, keepdims=True) + 1e-5)
    dl = (q - th) / Dn
    e_dl = (e_q + 4 * u32 * (q + th)) / Dn
    s_dl = np.abs(enc.bf16(dl + e_dl) - enc.bf16(dl - e_dl))
    dlb = enc.bf16(dl)

    def check(got, want_, tol, name):
        err = np.abs(np.asarray(got, dtype=np.float64) - want_)
        tol = tol + 1e-12 * np.abs(want_).max()
        ratio = err / tol
        assert (err <= tol).all(), (name, int((err > tol).sum()), float(ratio.max()),
                                    np.unravel_index(int(ratio.argmax()), ratio.shape))
        return tol

    tol_W2 = check(gW2, want["W2"], s_h.T @ np.abs(dlb) + hb.T @ s_dl + s_h.T @ s_dl
                   + acc * (hb.T @ np.abs(dlb)), "W2")
    check(gb2, want["b2"], e_dl.sum(axis=0) + acc * np.abs(dl).sum(axis=0), "b2")
    dH = dlb @ W2b.T
    e_dH = s_dl @ np.abs(W2b.T) + acc * (np.abs(dlb) @ np.abs(W2b.T))
    relu_open = np.abs(hp) <= e_h
    e_dhp = np.where(relu_open, np.abs(dH) + e_dH, np.where(hp > 0.0, e_dH, 0.0))
    dhp = dH * (hp > 0.0)
    check(gb1, want["b1"], e_dhp.sum(axis=0) + acc * np.abs(dhp).sum(axis=0), "b1")
    check(gW1, want["W1"], x.T @ e_dhp + acc * (x.T @ np.abs(dhp)), "W1")

    # the bounds are tight: the median bound is a small part of the sum of
    # |terms| (a BF16 step is 2^-8 of a term, and only some terms may take
    # one), and the gradient of one hidden unit in another's place lies
    # outside them
    assert np.median(tol_W2 / (hb.T @ np.abs(dlb) + 1e-300)) < 1e-2
    live = np.flatnonzero(np.abs(want["W2"]).sum(axis=1) > 0)
    j0, j1 = live[0], live[len(live) // 2]
    swapped = want["W2"].copy()
    swapped[[j0, j1]] = swapped[[j1, j0]]
    assert (np.abs(swapped - want["W2"])[[j0, j1]] > tol_W2[[j0, j1]]).mean() > 0.9


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
