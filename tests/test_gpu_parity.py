"""GPU sampler against the CPU oracle, through the C ABI.

Bit-exact parity of z, the proposals and c_k (all integer state) after whole
sweeps and after single phases, on the ``tiny`` workload and on small
adversarial corpora that reach every kernel tier: empty documents and words,
K = 1 and 2, hash and dense count tables, documents and words longer than a
block batch (multi-pass tier), M = 1..4, and launch tunings that move segments
between tiers.  The log-likelihood (FP64, different summation order) is
compared at 1e-9 relative.
"""
import os
import tempfile

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


def _gpu(c, V, K, alpha, beta, M, seed, tuning=None):
    from paper_1510_08628_gb300.warplda import WarpLDA
    return WarpLDA(c.doc_ptr, c.doc_word, V, K, alpha, beta, M, seed, tuning=tuning)


def _same_state(gpu, ref, tag=""):
    z, p, ck, _ = gpu.get_state()
    N, M = ref.N, ref.M
    assert np.array_equal(z, ref.z[:N]), f"{tag}: z differs at {np.flatnonzero(z != ref.z[:N])[:10]}"
    assert np.array_equal(p, ref.prop[: N * M]), f"{tag}: proposals differ"
    assert np.array_equal(ck, ref.ck), f"{tag}: c_k differs"


def test_init_matches_oracle(tiny_corpus):
    c, wl = tiny_corpus
    gpu = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    wp, perm = gpu.token_order()
    assert np.array_equal(wp, ref.word_ptr) and np.array_equal(perm, ref.perm[: ref.N])
    _same_state(gpu, ref, "init")


def test_tiny_workload_20_sweeps_bit_exact(tiny_corpus):
    c, wl = tiny_corpus
    gpu = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, 7)
    done = 0
    for cp in (1, 2, 5, 10, 20):
        gpu.sweep(cp - done)
        ref.sweep(cp - done)
        done = cp
        _same_state(gpu, ref, f"sweep {cp}")
        z, ck = gpu.counts()
        assert np.array_equal(z, ref.z_docmajor())
    ll, want = gpu.loglik(), ref.loglik()
    assert abs(ll - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("K,M", [(40, 2), (5, 3), (3000, 1)])
def test_phase_by_phase(K, M):
    c, wl = corpus.generate("tiny", seed=3, D=300)
    gpu = _gpu(c, c.V, K, 0.2, 0.01, M, 21)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.2, 0.01, M, 21)
    for it in range(1, 4):
        gpu.phase(1)
        ref.doc_phase(it)
        ref.recount()
        z, ck = gpu.counts()
        assert np.array_equal(z, ref.z_docmajor()), f"doc phase {it}"
        assert np.array_equal(ck, ref.ck)
        gpu.phase(2)
        ref.word_phase(it)
        ref.recount()
        ref.iteration = it
        _same_state(gpu, ref, f"word phase {it}")


def _edge_corpus(kind, seed=5):
    rng = np.random.default_rng(seed)
    if kind == "empty_segments":
        lens = [0, 3, 0, 0, 7, 1, 0, 12, 0]
        c = corpus.from_lengths(lens, V=40, seed=seed)
        return c
    if kind == "giant_doc":
        lens = [5, 9000, 3, 14, 4100, 2]
        return corpus.from_lengths(lens, V=300, seed=seed)
    if kind == "giant_word":
        lens = rng.integers(1, 60, size=600)
        c = corpus.from_lengths(lens, V=200, seed=seed)
        w = c.doc_word.copy()
        w[rng.random(len(w)) < 0.5] = 17          # one word with ~half the tokens
        return corpus.Corpus(c.doc_ptr, w, 200)
    if kind == "mixed":
        lens = np.concatenate([rng.integers(0, 30, size=400), [5000, 4093, 4094, 1]])
        return corpus.from_lengths(lens, V=500, seed=seed, zipf_s=1.2)
    if kind == "short_docs":
        # thousands of 0-3 token documents: batches end at their document cap
        lens = rng.integers(0, 4, size=3000)
        lens[::97] = 200
        return corpus.from_lengths(lens, V=300, seed=seed)
    raise ValueError(kind)


EDGE_CASES = [
    ("empty_segments", 3, 1), ("empty_segments", 1, 2), ("giant_doc", 2, 2), ("giant_doc", 16, 4),
    ("giant_word", 30, 2), ("giant_word", 1, 1), ("mixed", 7, 3), ("mixed", 5000, 2),
    ("mixed", 4097, 1), ("giant_word", 200, 4), ("short_docs", 50, 2), ("short_docs", 2049, 2),
]


@pytest.mark.parametrize("kind,K,M", EDGE_CASES)
def test_edge_corpora_bit_exact(kind, K, M):
    c = _edge_corpus(kind)
    gpu = _gpu(c, c.V, K, 0.3, 0.02, M, 99)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.3, 0.02, M, 99)
    for s in (1, 2, 4):
        gpu.sweep(1 if s != 4 else 2)
        ref.sweep(1 if s != 4 else 2)
        _same_state(gpu, ref, f"{kind} K={K} M={M} sweep {s}")
    ll, want = gpu.loglik(), ref.loglik()
    assert abs(ll - want) <= 1e-9 * abs(want)


TUNINGS = [None, {"batch_max_tokens": 64}, {"batch_max_tokens": 2000, "region_budget": 1024},
           {"huge_chunk": 300, "batch_max_tokens": 500}, {"batch_max_tokens": 4095},
           {"doc_warp_max": 512}, {"doc_warp_max": 20, "batch_max_tokens": 3000},
           {"doc_batch_kernel": 2}, {"doc_batch_kernel": 2, "batch_max_tokens": 64},
           {"doc_batch_kernel": 2, "region_budget": 600},
           {"batch_max_tokens": 64, "cluster_max_tokens": -1},
           {"batch_max_tokens": 64, "cluster_max_tokens": 300}]

CL = {"cluster_max_tokens": -1}   # the cluster tier as far as shared memory allows


@pytest.mark.parametrize("kind,K,M,tun,rule,on_cluster", [
    ("giant_word", 30, 2, CL, 0, True),
    ("giant_word", 3000, 1, CL, 0, True),
    ("giant_word", 1, 3, CL, 0, True),
    ("giant_word", 200, 4, {"cluster_max_tokens": 5000}, 0, False),
    ("mixed", 5000, 3, {"batch_max_tokens": 64, "cluster_max_tokens": 400}, 0, True),
    ("mixed", 16384, 2, {"batch_max_tokens": 100, "cluster_max_tokens": -1}, 0, True),
    ("giant_word", 40, 2, CL, 1, True),
    ("mixed", 3000, 2, {"batch_max_tokens": 64, "cluster_max_tokens": -1}, 1, True),
    ("giant_word", 30, 2, None, 0, False),
])
def test_cluster_tier_bit_exact(kind, K, M, tun, rule, on_cluster):
    """Words between a block batch and a cluster's shared memory, sampled on
    a thread-block cluster with the count rows reduced over distributed
    shared memory, against the oracle -- both word-positioning rules, dense
    and hash K, and caps that put some long words on the cluster and the
    others in the multi-pass tier."""
    c = _edge_corpus(kind)
    t = dict(tun or {})
    t["word_positioning"] = rule
    gpu = _gpu(c, c.V, K, 0.3, 0.02, M, 99, tuning=t)
    info = gpu.info()
    assert (info["cluster_words"] > 0) == on_cluster, info
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.3, 0.02, M, 99, word_rule=rule)
    for s in (1, 2):
        gpu.sweep(s)
        ref.sweep(s)
        _same_state(gpu, ref, f"cluster tier {kind} K={K} M={M} rule={rule}")
    gpu.sync()
    ll, want = gpu.loglik(), ref.loglik()
    assert abs(ll - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("kind,K,M,dk", [("mixed", 7, 3, 2), ("mixed", 5000, 2, 1), ("giant_doc", 16, 4, 2),
                                         ("short_docs", 2049, 2, 1), ("empty_segments", 3, 1, 2),
                                         ("short_docs", 50, 1, 2), ("mixed", 300, 4, 2),
                                         ("mixed", 5000, 3, 1), ("giant_word", 30, 2, 2)])
def test_other_document_kernel_bit_exact(kind, K, M, dk):
    """The document kernel the default does not pick for K (tuning
    doc_batch_kernel: 1 = block batch kernel with hash tables, 2 = pipelined
    kernel with dense tables) against the oracle."""
    c = _edge_corpus(kind)
    gpu = _gpu(c, c.V, K, 0.3, 0.02, M, 99, tuning={"doc_batch_kernel": dk})
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.3, 0.02, M, 99)
    for s in (1, 2):
        gpu.sweep(s)
        ref.sweep(s)
        _same_state(gpu, ref, f"document kernel {dk}: {kind} K={K} M={M}")


def test_pipelined_document_kernel_rejects_bad_tuning():
    from paper_1510_08628_gb300.warplda import WarpLDAError
    c = _edge_corpus("mixed")
    with pytest.raises(WarpLDAError, match="doc_batch_kernel"):
        _gpu(c, c.V, 50, 0.1, 0.01, 2, 5, tuning={"doc_batch_kernel": 3})


def test_schedule_independence():
    c = _edge_corpus("mixed")
    states = []
    for t in TUNINGS:
        gpu = _gpu(c, c.V, 50, 0.1, 0.01, 2, 5, tuning=t)
        gpu.sweep(3)
        states.append(gpu.get_state())
        gpu.close()
    for s in states[1:]:
        for a, b in zip(states[0], s):
            assert np.array_equal(np.asarray(a), np.asarray(b))


def test_save_load_resume_bit_exact(tiny_corpus):
    c, wl = tiny_corpus
    a = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, 2, 13)
    a.sweep(10)
    b = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, 2, 13)
    b.sweep(5)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        b.save(path)
        b2 = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, 2, 13)
        b2.load_state(path)
    b2.sweep(5)
    for x, y in zip(a.get_state(), b2.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_counts_dev_and_bad_state(tiny_corpus):
    import torch
    from paper_1510_08628_gb300.warplda import WarpLDAError
    c, wl = tiny_corpus
    g = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, wl.M, 3)
    g.sweep(2)
    zt = torch.empty(c.N, dtype=torch.int32, device="cuda")
    ckt = torch.empty(wl.K, dtype=torch.int32, device="cuda")
    g.counts_dev(zt, ckt)
    torch.cuda.synchronize()
    z, ck = g.counts()
    assert np.array_equal(zt.cpu().numpy(), z) and np.array_equal(ckt.cpu().numpy(), ck)
    # pinned host buffers take the direct gather; same values as the copy path
    zp = torch.full((c.N,), -1, dtype=torch.int32, pin_memory=True).numpy()
    ckp = torch.full((wl.K,), -1, dtype=torch.int32, pin_memory=True).numpy()
    z2, ck2 = g.counts(z_out=zp, ck_out=ckp)
    assert np.array_equal(z2, z) and np.array_equal(ck2, ck) and np.array_equal(zp, z)
    zs, ps, _, it = g.get_state()
    bad = zs.copy()
    bad[5] = wl.K
    with pytest.raises(WarpLDAError):
        g.set_state(bad, ps, it)
    g.set_state(zs, ps, it)
    assert np.array_equal(g.get_state()[0], zs)


def test_invalid_arguments_rejected():
    from paper_1510_08628_gb300.warplda import WarpLDA, WarpLDAError
    c = corpus.from_lengths([3, 4], V=10, seed=1)
    for kw in ({"K": 0}, {"K": 1 << 20}, {"M": 0}, {"M": 5}, {"alpha": 0.0}, {"beta": -1.0}):
        args = dict(K=4, alpha=0.1, beta=0.1, M=1)
        args.update(kw)
        with pytest.raises(WarpLDAError):
            WarpLDA(c.doc_ptr, c.doc_word, 10, args["K"], args["alpha"], args["beta"], args["M"], 1)
    bad = c.doc_word.copy()
    bad[0] = 10
    with pytest.raises(WarpLDAError):
        WarpLDA(c.doc_ptr, bad, 10, 4, 0.1, 0.1, 1, 1)


def test_sync_reports_clean_checks(tiny_corpus):
    c, wl = tiny_corpus
    g = _gpu(c, c.V, wl.K, wl.alpha, wl.beta, wl.M, 17)
    g.sweep(3)
    g.sync()
    g.phase(1)
    g.sync()
    g.phase(2)
    g.sync()


@pytest.mark.parametrize("kind,K,M,tuning", [("mixed", 7, 3, None), ("mixed", 5000, 2, None),
                                             ("giant_word", 30, 2, None),
                                             ("giant_word", 200, 4, {"huge_chunk": 300}),
                                             ("mixed", 50, 2, {"batch_max_tokens": 64})])
def test_storage_order_word_positioning_bit_exact(kind, K, M, tuning):
    """The paper's literal word positioning (storage order; tuning
    word_positioning = 1) against the oracle's rule-1 word phase."""
    c = _edge_corpus(kind)
    t = dict(tuning or {})
    t["word_positioning"] = 1
    gpu = _gpu(c, c.V, K, 0.3, 0.02, M, 99, tuning=t)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.3, 0.02, M, 99, word_rule=1)
    for s in (1, 2):
        gpu.sweep(s)
        ref.sweep(s)
        _same_state(gpu, ref, f"storage {kind} K={K} M={M}")


@pytest.mark.parametrize("kind,K,M,tuning", [("giant_word", 100000, 2, None),
                                             ("mixed", 20000, 3, {"batch_max_tokens": 64}),
                                             ("giant_doc", (1 << 20) - 1, 1, None),
                                             ("giant_word", 16385, 4, {"huge_chunk": 300}),
                                             ("short_docs", 70000, 1, None),
                                             ("mixed", 40000, 2, {"doc_batch_kernel": 2}),
                                             ("short_docs", 70000, 1, {"doc_batch_kernel": 2})])
def test_large_K_sparse_rows_bit_exact(kind, K, M, tuning):
    """K above 16384: long segments count into hash rows in device memory and
    word proposals use storage-order positioning (forced), so the oracle runs
    its rule-1 word phase.  Covers the largest K the packed tables allow."""
    c = _edge_corpus(kind)
    gpu = _gpu(c, c.V, K, 0.3, 0.02, M, 99, tuning=tuning)
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, 0.3, 0.02, M, 99, word_rule=1)
    for s in (1, 2):
        gpu.sweep(s)
        ref.sweep(s)
        _same_state(gpu, ref, f"large K {kind} K={K} M={M}")
    gpu.sync()
    ll, want = gpu.loglik(), ref.loglik()
    assert abs(ll - want) <= 1e-9 * abs(want)


def test_large_K_dense_model_calls_rejected():
    from paper_1510_08628_gb300.warplda import WarpLDA, WarpLDAError
    c = corpus.from_lengths([30, 40, 5], V=50, seed=1)
    g = WarpLDA(c.doc_ptr, c.doc_word, 50, 30000, 0.1, 0.01, 1, 1)
    g.sweep(1)
    with pytest.raises(WarpLDAError, match="16384"):
        g.word_counts()
    with pytest.raises(WarpLDAError, match="16384"):
        g.foldin(c.doc_ptr, c.doc_word, 2, 1)


def _expected_batch_lists(doc_ptr, perm, batches):
    """sperm / sinfo of the document batches from their definition: each
    batch's tokens (a contiguous doc-major range) listed by ascending
    word-major index, with (document slot << 16 | position in the batch)."""
    N = len(perm)
    sperm = np.zeros(N, np.int64)
    sinfo = np.zeros(N, np.int64)
    bid = np.full(N, -1, np.int64)
    b0 = doc_ptr[batches[:, 0]]
    b1 = doc_ptr[batches[:, 1]]
    for i in range(len(batches)):
        bid[b0[i]:b1[i]] = i
    pos = np.flatnonzero(bid >= 0)
    order = np.lexsort((perm[pos], bid[pos]))
    p = pos[order]
    g = bid[p]
    start = np.searchsorted(g, np.arange(len(batches)))
    dest = b0[g] + (np.arange(len(p)) - start[g])
    doc = np.searchsorted(doc_ptr, p, side="right") - 1
    sperm[dest] = perm[p]
    sinfo[dest] = ((doc - batches[g, 0]) << 16) | (p - b0[g])
    return sperm, sinfo


@pytest.mark.parametrize("kind,K,tuning", [("mixed", 7, None), ("mixed", 5000, None),
                                           ("giant_doc", 16, None), ("empty_segments", 3, None),
                                           ("mixed", 50, {"batch_max_tokens": 64}),
                                           ("mixed", 3000, {"doc_warp_max": 20})])
def test_device_token_order_build(kind, K, tuning):
    """The token store built on the device (Sec. 5.2): word offsets and perm
    equal the stable sort of the tokens by word, and the document batches'
    word-major lists equal their definition."""
    c = _edge_corpus(kind)
    g = _gpu(c, c.V, K, 0.3, 0.02, 2, 99, tuning=tuning)
    wp, perm = g.token_order()
    assert np.array_equal(wp, np.concatenate([[0], np.cumsum(np.bincount(c.doc_word, minlength=c.V))]))
    order = np.argsort(c.doc_word, kind="stable")
    want = np.empty(c.N, np.int64)
    want[order] = np.arange(c.N)
    assert np.array_equal(perm, want)
    batches, sperm, sinfo = g.doc_batches()
    es, ei = _expected_batch_lists(c.doc_ptr.astype(np.int64), perm.astype(np.int64), batches.astype(np.int64))
    assert np.array_equal(sperm, es)
    assert np.array_equal(sinfo.astype(np.int64), ei)


def test_init_trace_reports_every_stage(capfd, monkeypatch):
    """WARPLDA_TRACE_INIT=1: warplda_init prints one timed line per stage to
    stderr, and the context it builds is the same as without the trace."""
    c = _edge_corpus("mixed")
    monkeypatch.setenv("WARPLDA_TRACE_INIT", "1")
    g = _gpu(c, c.V, 50, 0.3, 0.02, 2, 11)
    monkeypatch.delenv("WARPLDA_TRACE_INIT")
    err = capfd.readouterr().err
    stages = [ln for ln in err.splitlines() if ln.startswith("warplda_init ")]
    assert len(stages) == 10, err
    for name in ("word check and word sort", "perm", "grids, initial z and c_k"):
        assert any(name in ln for ln in stages), (name, err)
    ref = _gpu(c, c.V, 50, 0.3, 0.02, 2, 11)
    assert "warplda_init " not in capfd.readouterr().err
    for x, y in zip(g.get_state(), ref.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    g.close()
    ref.close()

@pytest.mark.parametrize("V", [512, 513, 5000, 1 << 17, 1 << 18, (1 << 18) + 1, 1_000_000])
def test_device_word_sort_digit_splits(V):
    """The device word sort splits the key bits over passes of at most 9
    bits (one pass up to 512 words, two up to 2^18, three beyond): word
    offsets and perm equal the stable sort of the tokens by word, with word
    ids across the whole range and many ties."""
    rng = np.random.default_rng(V)
    lens = rng.integers(0, 300, size=2000)
    lens[::97] = 0
    N = int(lens.sum())
    spread = rng.integers(0, V, size=N)
    heavy = rng.choice(np.array([0, 1, V // 2, V - 2, V - 1]), size=N)
    doc_word = np.where(rng.random(N) < 0.4, heavy, spread).astype(np.int32)
    c = corpus.Corpus(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64), doc_word, V)
    g = _gpu(c, V, 64, 0.3, 0.02, 2, 3)
    wp, perm = g.token_order()
    assert np.array_equal(wp, np.concatenate([[0], np.cumsum(np.bincount(c.doc_word, minlength=V))]))
    want = np.empty(N, np.int64)
    want[np.argsort(c.doc_word, kind="stable")] = np.arange(N)
    assert np.array_equal(perm, want)
    g.close()
