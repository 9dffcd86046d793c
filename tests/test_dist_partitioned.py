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
