"""The paper's distributed sweep (Sec. 5.3.2) on CPU ranks over gloo.

P ranks each own a contiguous document row set and a greedy-balanced word
column set; token blocks move by all-to-all between the phases and c_k is
all-reduced.  The partitioned chain must equal the single-process oracle's
bit for bit (z, proposals, c_k), at P = 2 and 3, for both word-positioning
rules, on a corpus with empty documents and words.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _corpus():
    sys.path.insert(0, ROOT)
    from paper_1510_08628_gb300 import corpus
    rng = np.random.default_rng(11)
    lens = np.concatenate([rng.integers(0, 40, size=300), [0, 900, 0, 3]])
    return corpus.from_lengths(lens, V=700, seed=11, zipf_s=1.1)


def _rank(rank, P, port, word_rule, sweeps, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle.partitioned import PartitionedOracle
    dist.init_process_group("gloo", rank=rank, world_size=P)
    c = _corpus()
    po = PartitionedOracle(c.doc_ptr, c.doc_word, c.V, 24, 0.3, 0.02, 2, 5, rank, P, word_rule=word_rule)
    po.sweep(sweeps)
    z, p, ck = po.gather()
    if rank == 0:
        q.put((z, p, ck, po.sent_records))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("P,word_rule", [(2, 0), (3, 0), (2, 1)])
def test_partitioned_sweep_equals_single_process(P, word_rule):
    mp = pytest.importorskip("torch.multiprocessing")
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, P, port, word_rule, 3, q)) for r in range(P)]
    for p in ps:
        p.start()
    z, prop, ck, sent = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    c = _corpus()
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 24, 0.3, 0.02, 2, 5, word_rule=word_rule)
    ref.sweep(3)
    assert np.array_equal(z, ref.z[: ref.N])
    assert np.array_equal(prop, ref.prop[: ref.N * 2])
    assert np.array_equal(ck, ref.ck)
    assert sent > 0          # blocks did cross ranks


def test_partitions_cover_and_balance():
    sys.path.insert(0, ROOT)
    import oracle
    from oracle.partitioned import doc_partition, word_partition
    c = _corpus()
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 4, 0.3, 0.02, 1, 5)
    for P in (1, 2, 3, 5):
        b = doc_partition(o.doc_ptr, P)
        assert b[0] == 0 and b[-1] == o.D and np.all(np.diff(b) >= 0)
        owner = word_partition(o.word_ptr, P)
        load = np.bincount(owner, weights=np.diff(o.word_ptr), minlength=P)
        assert load.sum() == o.N
        # greedy by descending size: no set exceeds the mean by more than the largest word
        assert load.max() - o.N / P <= np.diff(o.word_ptr).max()


def _rank_planted(rank, P, port, mistake, q):
    """As _rank, with one mistake planted in the exchange (oracle side, CPU)."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle.partitioned import PartitionedOracle

    class Planted(PartitionedOracle):
        def _reduce_ck(self, owned):
            if mistake == "local_ck":          # c_k from this rank's tokens only
                self.ck = np.bincount(self.o.z[owned], minlength=self.o.K).astype(np.int32)
            else:
                super()._reduce_ck(owned)

        def _exchange(self, to_words):
            if mistake == "drop_block" and to_words:
                saved = self.block[(0, 1)]
                self.block[(0, 1)] = saved[: len(saved) // 2]   # half a block never arrives
                super()._exchange(to_words)
                self.block[(0, 1)] = saved
            else:
                super()._exchange(to_words)

    dist.init_process_group("gloo", rank=rank, world_size=P)
    c = _corpus()
    po = Planted(c.doc_ptr, c.doc_word, c.V, 24, 0.3, 0.02, 2, 5, rank, P)
    po.sweep(2)
    z, p, ck = po.gather()
    if rank == 0:
        q.put((z, p, ck))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mistake", ["local_ck", "drop_block"])
def test_planted_exchange_mistakes_are_caught(mistake):
    mp = pytest.importorskip("torch.multiprocessing")
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_planted, args=(r, 2, port, mistake, q)) for r in range(2)]
    for p in ps:
        p.start()
    z, prop, ck = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    c = _corpus()
    ref = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, 24, 0.3, 0.02, 2, 5)
    ref.sweep(2)
    same = (np.array_equal(z, ref.z[: ref.N]) and np.array_equal(prop, ref.prop[: ref.N * 2])
            and np.array_equal(ck, ref.ck))
    assert not same, f"planted mistake {mistake} went unnoticed"
