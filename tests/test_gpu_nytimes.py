"""Full-size parity on the NYTimes-shaped workload (D=300K, V=100K, ~99M
tokens, K=1,000, M=2) in the launch configuration the benchmark times: the
GPU state after every phase of three sweeps equals the oracle's bit for bit,
c_k is the histogram of z, and the log-likelihood agrees to 1e-9."""
import numpy as np
import pytest

import oracle
from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu


def test_nytimes_three_sweeps_bit_exact():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl = corpus.generate("nytimes", seed=1)
    gpu = WarpLDA(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    info = gpu.info()
    assert info["mega_words"] > 0 and info["doc_batches"] > 0
    for it in range(1, 4):
        gpu.phase(1)
        ref.doc_phase(it)
        ref.recount()
        z, p, ck, _ = gpu.get_state()
        assert np.array_equal(z, ref.z[: ref.N]), f"doc phase {it}: z"
        assert np.array_equal(p, ref.prop), f"doc phase {it}: proposals"
        assert np.array_equal(ck, ref.ck), f"doc phase {it}: c_k"
        assert np.array_equal(ck, np.bincount(z, minlength=wl.K))
        gpu.phase(2)
        ref.word_phase(it)
        ref.recount()
        ref.iteration = it
        z, p, ck, _ = gpu.get_state()
        assert np.array_equal(z, ref.z[: ref.N]), f"word phase {it}: z"
        assert np.array_equal(p, ref.prop), f"word phase {it}: proposals"
        assert np.array_equal(ck, ref.ck), f"word phase {it}: c_k"
    ll, want = gpu.loglik(), ref.loglik()
    assert abs(ll - want) <= 1e-9 * abs(want)
