"""Error paths of the C ABI, exercised without faulting a GPU.

Failures are made on the host: the library's fault injection
(WARPLDA_FAIL_ALLOC=k fails the k-th allocation it asks for as out of
memory, WARPLDA_FAIL_LAUNCH=k makes the k-th kernel launcher return a launch
error without launching) drives warplda_init, warplda_foldin and
warplda_server_create through every allocation and launch they make; each
call must return ENOMEM or ECUDA, free what it took, and leave the library
usable.  A bounded wait is made to run out by polling a serving step with a
zero time limit while the step is still on the GPU: ETIMEDOUT, then a later
poll returns the step's results.
"""
import os

import numpy as np
import pytest

from paper_1510_08628_gb300 import corpus

ENOMEM, ECUDA, ETIMEDOUT = -2, -3, -4


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


class _inject:
    """WARPLDA_FAIL_<what>=k for the duration of a block."""

    def __init__(self, what, k):
        self.var, self.k = f"WARPLDA_FAIL_{what}", k

    def __enter__(self):
        os.environ[self.var] = str(self.k)

    def __exit__(self, *exc):
        os.environ.pop(self.var, None)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


SLACK = 4 << 20   # driver-side bookkeeping between two reads of the free memory


def _sweep_failures(what, code, call, limit=200):
    """Runs call() with the k-th allocation / launch failing, k = 1, 2, ...
    until it succeeds; every failing run must raise `code` and give back its
    device memory.  Returns the number of failure points met."""
    from paper_1510_08628_gb300.warplda import WarpLDAError
    base = _free_bytes()
    for k in range(1, limit):
        with _inject(what, k):
            try:
                out = call()
            except WarpLDAError as e:
                assert e.code == code, (what, k, e)
                assert _free_bytes() >= base - SLACK, (what, k, "device memory not given back")
                continue
        if hasattr(out, "close"):
            out.close()
        return k - 1
    raise AssertionError(f"{what}: still failing after {limit} injection points")


@pytest.mark.skipif(_cuda_ok(), reason="checks the path taken without a CUDA device")
def test_init_without_a_device_fails_cleanly():
    from paper_1510_08628_gb300.warplda import WarpLDA, WarpLDAError
    c = corpus.from_lengths([3, 4, 0, 5], V=10, seed=1)
    with pytest.raises(WarpLDAError) as ei:
        WarpLDA(c.doc_ptr, c.doc_word, 10, 4, 0.1, 0.1, 1, 1)
    assert ei.value.code == ECUDA and "cuda" in str(ei.value).lower()


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1510_08628_gb300 import warplda
    warplda.load()
    c, wl = corpus.generate("tiny", seed=3, D=300)
    # a first context outside the measured runs (module and context set-up)
    g = warplda.WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, wl.alpha, wl.beta, 2, 5)
    g.sweep(3)
    yield c, wl, g
    g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("K", [40, 3000, 40000])
def test_init_allocation_and_launch_failures(gpu, K):
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl, _ = gpu
    make = lambda: WarpLDA(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, 2, 5)
    assert _sweep_failures("ALLOC", ENOMEM, make) >= 10
    assert _sweep_failures("LAUNCH", ECUDA, make) >= 5
    # after all of it the library still works and gives the same chain
    a, b = make(), make()
    a.sweep(2)
    b.sweep(2)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    a.close()
    b.close()


@pytest.mark.gpu
def test_foldin_allocation_and_launch_failures(gpu):
    """Fold-in keeps its scratch in the context between calls, so the
    allocation failures are swept on fresh contexts (their init's allocations
    come first, then the fold-in's); launch failures on the warm context."""
    from paper_1510_08628_gb300.warplda import WarpLDA
    c, wl, g = gpu
    rq = corpus.requests("tiny", seed=3, n=30, doc_offset=9000, lo=1, hi=300)
    want, _ = g.foldin(rq.doc_ptr, rq.doc_word, sweeps=4, seed=3)

    def cold():
        m = WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, wl.alpha, wl.beta, 2, 5)
        try:
            m.sweep(3)
            return m.foldin(rq.doc_ptr, rq.doc_word, sweeps=4, seed=3)
        finally:
            m.close()

    assert _sweep_failures("ALLOC", ENOMEM, cold) >= 12
    warm = lambda: g.foldin(rq.doc_ptr, rq.doc_word, sweeps=4, seed=3)
    assert _sweep_failures("LAUNCH", ECUDA, warm) >= 1
    got, _ = warm()
    assert np.array_equal(got, want)
    assert np.array_equal(cold()[0], want)
    g.sync()


@pytest.mark.gpu
@pytest.mark.parametrize("learned", [False, True])
def test_server_create_allocation_failures(gpu, learned):
    from paper_1510_08628_gb300.warplda import Server
    c, wl, g = gpu
    if learned and not getattr(g, "_enc_ready", False):
        g.encoder_init(log2_features=10, hidden=128, batch_rows=128, seed=9)
        g._enc_ready = True
    make = lambda: Server(g, slots=16, pool_tokens=5000, max_doc_tokens=500, sweeps=2, seed=1,
                          learned=learned)
    assert _sweep_failures("ALLOC", ENOMEM, make) >= 8
    s = make()
    assert s.submit(7, c.doc_word[:50])
    got = []
    for _ in range(2):   # 2 sweeps: the result comes with the second step
        s.step()
        ids, th = s.poll()
        got += [(int(i), t) for i, t in zip(ids, th)]
    assert [i for i, _ in got] == [7] and np.isfinite(got[0][1]).all()
    s.close()


@pytest.mark.gpu
def test_poll_times_out_while_a_step_runs():
    """A serving step long enough to be still running when it is polled with
    a zero time limit: ETIMEDOUT; the next poll with time to spare returns the
    finished requests, each equal to warplda_foldin's row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_08628_gb300.warplda import Server, WarpLDA, WarpLDAError
    c, wl = corpus.generate("tiny", seed=5, D=200)
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, wl.alpha, wl.beta, 2, 5)
    g.sweep(2)
    rng = np.random.default_rng(2)
    L = 20000
    timed_out = False
    for n_docs in (256, 1024, 4096):
        docs = [rng.integers(0, c.V, size=L).astype(np.int32) for _ in range(n_docs)]
        s = Server(g, slots=n_docs, pool_tokens=n_docs * L, max_doc_tokens=L, sweeps=1, seed=4)
        for i, d in enumerate(docs):
            assert s.submit(i, d)
        s.step()
        try:
            ids, th = s.poll(timeout_ms=0)
        except WarpLDAError as e:
            assert e.code == ETIMEDOUT, e
            timed_out = True
            ids, th = s.poll(timeout_ms=120000)
        if not timed_out:
            assert len(ids) == n_docs      # finished within the poll: try a longer step
            s.close()
            continue
        assert sorted(ids.tolist()) == list(range(n_docs))
        dp = np.arange(n_docs + 1, dtype=np.int64) * L
        want, _ = g.foldin(dp, np.concatenate(docs), sweeps=1, seed=4, doc_ids=np.arange(n_docs))
        for i, t in zip(ids, th):
            assert np.array_equal(t, want[int(i)])
        s.close()
        break
    g.close()
    assert timed_out, "no step outlasted a zero-limit poll"


@pytest.mark.gpu
def test_closing_a_context_closes_its_servers():
    """A server holds pointers into its model context: closing the context
    first destroys the servers still open, so nothing touches freed memory."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_08628_gb300.warplda import Server, WarpLDA, WarpLDAError
    c, wl = corpus.generate("tiny", seed=5, D=100)
    g = WarpLDA(c.doc_ptr, c.doc_word, c.V, 40, wl.alpha, wl.beta, 2, 5)
    g.sweep(1)
    s = Server(g, slots=4, pool_tokens=1000, max_doc_tokens=200, sweeps=3, seed=1)
    assert s.submit(1, c.doc_word[:20])
    s.step()
    g.close()
    assert s._h is None          # destroyed with its context
    s.close()                    # and closing it again is harmless
    with pytest.raises(WarpLDAError):
        Server(g, slots=4, pool_tokens=1000, max_doc_tokens=200, sweeps=3, seed=1)

