"""warplda_loglik_noalloc: the log-likelihood entry point that allocates no
device memory (for callers whose device memory is owned by a host framework
or fixed by a budget), checked through the C ABI against the context-based
warplda_loglik on two calls in a row, so a stale scratch array would show;
also at the largest K it accepts (whose histogram needs the opt-in to more
than 48 KB of shared memory) on a caller's own stream.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

from paper_1510_08628_gb300 import corpus

pytestmark = pytest.mark.gpu


def _setup(K, seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300 import warplda
    c, wl = corpus.generate("tiny", seed=4, D=600)
    g = warplda.WarpLDA(c.doc_ptr, c.doc_word, c.V, K, 0.2, 0.01, 2, seed)
    return torch, warplda, c, g


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_loglik_noalloc_matches_loglik_twice():
    torch, warplda, c, g = _setup(40, 17)
    wp, perm = g.token_order()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for sweeps in (2, 3):
        g.sweep(sweeps)
        want = g.loglik()
        z_word = g.get_state()[0]
        z_doc = z_word[perm]
        warplda.loglik_noalloc(c.D, c.V, c.N, 40, 0.2, 0.01, _dev(torch, c.doc_ptr), _dev(torch, z_doc),
                               _dev(torch, wp), _dev(torch, z_word), out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - want) <= 1e-9 * abs(want), (got, want)
    args = (_dev(torch, c.doc_ptr), _dev(torch, z_doc), _dev(torch, wp), _dev(torch, z_word), out)
    # sizes beyond the scratch are refused with a clear error
    with pytest.raises(warplda.WarpLDAError, match="16384"):
        warplda.loglik_noalloc(c.D, c.V, c.N, 20000, 0.2, 0.01, *args)
    # a value outside [0, K) -- in either order -- is not counted and turns
    # the result into NaN
    for which in (1, 3):
        bad = list(args)
        arr = (z_doc if which == 1 else z_word).copy()
        arr[3] = 40
        bad[which] = _dev(torch, arr)
        out.zero_()
        warplda.loglik_noalloc(c.D, c.V, c.N, 40, 0.2, 0.01, *bad)
        torch.cuda.synchronize()
        assert np.isnan(float(out.item())), which
    # N that is not the offsets' token count: NaN
    out.zero_()
    warplda.loglik_noalloc(c.D, c.V, c.N - 1, 40, 0.2, 0.01, *args)
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
    g.close()


def test_loglik_noalloc_largest_K_on_a_caller_stream():
    torch, warplda, c, g = _setup(16384, 5)
    wp, perm = g.token_order()
    g.sweep(2)
    want = g.loglik()
    z_word = g.get_state()[0]
    args = (_dev(torch, c.doc_ptr), _dev(torch, z_word[perm]), _dev(torch, wp), _dev(torch, z_word))
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for i in range(2):
            warplda.loglik_noalloc(c.D, c.V, c.N, 16384, 0.2, 0.01, *args, out[i:i + 1], stream=st)
    st.synchronize()
    for i in range(2):
        got = float(out[i].item())
        assert abs(got - want) <= 1e-9 * abs(want), (i, got, want)
    g.close()
