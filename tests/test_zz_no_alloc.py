"""warplda_loglik_noalloc: the log-likelihood entry point that allocates no
device memory (for callers whose device memory is owned by a host framework
or fixed by a budget), checked through the C ABI against the context-based
warplda_loglik on two calls in a row, so a stale scratch array would show.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu


def test_loglik_noalloc_matches_loglik_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300 import warplda
    c, wl = corpus.generate("tiny", seed=4, D=600)
    g = warplda.WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, 0.2, 0.01, 2, 17)
    wp, perm = g.token_order()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for sweeps in (2, 3):
        g.sweep(sweeps)
        want = g.loglik()
        z_word = g.get_state()[0]
        z_doc = z_word[perm]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        warplda.loglik_noalloc(c.D, c.V, c.N, 40, 0.2, 0.01, dev(c.doc_ptr), dev(z_doc), dev(wp),
                               dev(z_word), out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - want) <= 1e-9 * abs(want), (got, want)
    # sizes beyond the scratch are refused with a clear error
    with pytest.raises(warplda.WarpLDAError, match="16384"):
        warplda.loglik_noalloc(c.D, c.V, c.N, 20000, 0.2, 0.01, dev(c.doc_ptr), dev(z_doc),
                               dev(wp), dev(z_word), out)
    # a value outside [0, K) is not counted and turns the result into NaN
    bad = z_doc.copy()
    bad[3] = 40
    warplda.loglik_noalloc(c.D, c.V, c.N, 40, 0.2, 0.01, dev(c.doc_ptr), dev(bad), dev(wp),
                           dev(z_word), out)
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
