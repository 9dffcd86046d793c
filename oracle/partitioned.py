"""Partitioned WarpLDA sweep over P ranks (Sec. 5.3.2) -- test infrastructure.

Only ``tests/`` may import this module.  It restates the paper's distributed
layout on CPU ranks joined by ``torch.distributed`` (gloo), on top of the
oracle's per-document and per-word steps:

* the documents are cut into P contiguous row sets R_i of about N/P tokens,
  and the words into P column sets C_j, words taken most frequent first and
  each given to the column set with the fewest tokens so far (the greedy
  balancing of Sec. 5.3.2); the token block P_ij = R_i x C_j;
* rank i runs the document phase on R_i and the word phase on C_i;
* after the document phase rank i sends rank j the current topic and
  proposals of every token of P_ij (one all-to-all of token blocks), and after
  the word phase the blocks go back (rank j sends P_ij to rank i);
* c_k after each phase is the sum over ranks (all-reduce) of the histograms
  of the tokens each rank owns in that phase.

Every token's phase-start counts, c_k and Philox stream (keyed by its
word-major index) are those of the single-process oracle, so the partitioned
chain is the same chain bit for bit.  Blocks travel as int32 records
(z, p_1..p_M) in ascending word-major order, which both ends derive from the
partition, so no sizes are exchanged.
"""
from __future__ import annotations

import numpy as np

from . import Oracle


def doc_partition(doc_ptr, P: int) -> np.ndarray:
    """Bounds [P+1] of P contiguous document ranges of about N/P tokens."""
    doc_ptr = np.asarray(doc_ptr, dtype=np.int64)
    D, N = len(doc_ptr) - 1, int(doc_ptr[-1])
    b = np.zeros(P + 1, dtype=np.int64)
    for i in range(1, P):
        b[i] = min(D, max(b[i - 1], int(np.searchsorted(doc_ptr, N * i / P, side="left"))))
    b[P] = D
    return b


def word_partition(word_ptr, P: int) -> np.ndarray:
    """owner[V]: words by descending length (ties by id), each to the column
    set with the fewest tokens so far (ties to the lowest rank)."""
    L = np.diff(np.asarray(word_ptr, dtype=np.int64))
    order = sorted(range(len(L)), key=lambda w: (-int(L[w]), w))
    load = [0] * P
    owner = np.zeros(len(L), dtype=np.int64)
    for w in order:
        j = min(range(P), key=lambda r: (load[r], r))
        owner[w] = j
        load[j] += int(L[w])
    return owner


class PartitionedOracle:
    """The oracle's state on rank `rank` of P; every rank holds word-major
    arrays of all N tokens but keeps current only the tokens it owns."""

    def __init__(self, doc_ptr, doc_word, V, K, alpha, beta, M, seed, rank: int, P: int,
                 word_rule: int = 0):
        import torch.distributed as dist
        self.dist = dist
        self.o = Oracle(doc_ptr, doc_word, V, K, alpha, beta, M, seed, word_rule=word_rule)
        o = self.o
        self.rank, self.P = int(rank), int(P)
        N = o.N
        self.db = doc_partition(o.doc_ptr, P)
        self.wowner = word_partition(o.word_ptr, P)
        inv = np.empty(N, dtype=np.int64)
        inv[o.perm[:N]] = np.arange(N)                      # word-major -> doc-major position
        doc_of = np.searchsorted(o.doc_ptr, inv, side="right") - 1
        word_of = np.searchsorted(o.word_ptr, np.arange(N), side="right") - 1
        self.down = np.searchsorted(self.db, doc_of, side="right") - 1   # doc-phase owner
        self.wown = self.wowner[word_of]                                  # word-phase owner
        self.block = {(i, j): np.flatnonzero((self.down == i) & (self.wown == j))
                      for i in range(P) for j in range(P)}
        mine = np.flatnonzero(self.wowner == self.rank)
        # runs of consecutive owned words, for the oracle's range calls
        self.word_runs = []
        for w in mine:
            if self.word_runs and self.word_runs[-1][1] == w:
                self.word_runs[-1][1] = w + 1
            else:
                self.word_runs.append([int(w), int(w) + 1])
        self.ck = o.ck.copy()                               # the init histogram, same on all ranks
        self.sent_records = 0

    def _records(self, idx: np.ndarray) -> np.ndarray:
        o, M = self.o, self.o.M
        rec = np.empty((len(idx), M + 1), dtype=np.int32)
        rec[:, 0] = o.z[idx]
        for i in range(M):
            rec[:, 1 + i] = o.prop[idx * M + i]
        return rec.reshape(-1)

    def _store(self, idx: np.ndarray, flat: np.ndarray) -> None:
        o, M = self.o, self.o.M
        rec = flat.reshape(len(idx), M + 1)
        o.z[idx] = rec[:, 0]
        for i in range(M):
            o.prop[idx * M + i] = rec[:, 1 + i]

    def _exchange(self, to_words: bool) -> None:
        """All-to-all of token blocks: doc owners to word owners or back."""
        import torch
        me, P, M = self.rank, self.P, self.o.M
        send_idx = [self.block[(me, j)] if to_words else self.block[(j, me)] for j in range(P)]
        recv_idx = [self.block[(i, me)] if to_words else self.block[(me, i)] for i in range(P)]
        send = np.concatenate([self._records(ix) for ix in send_idx]) if P else np.zeros(0, np.int32)
        out = torch.empty(sum(len(ix) for ix in recv_idx) * (M + 1), dtype=torch.int32)
        self.dist.all_to_all_single(out, torch.from_numpy(send),
                                    [len(ix) * (M + 1) for ix in recv_idx],
                                    [len(ix) * (M + 1) for ix in send_idx])
        got = out.numpy()
        o0 = 0
        for ix in recv_idx:
            n = len(ix) * (M + 1)
            self._store(ix, got[o0:o0 + n])
            o0 += n
        self.sent_records += sum(len(ix) for j, ix in enumerate(send_idx) if j != me)

    def _reduce_ck(self, owned: np.ndarray) -> None:
        import torch
        h = np.bincount(self.o.z[owned], minlength=self.o.K).astype(np.int32)
        t = torch.from_numpy(h)
        self.dist.all_reduce(t)
        self.ck = t.numpy().astype(np.int32)

    def sweep(self, n: int = 1) -> None:
        o, me = self.o, self.rank
        mine_doc = np.flatnonzero(self.down == me)
        mine_word = np.flatnonzero(self.wown == me)
        for _ in range(n):
            it = o.iteration + 1
            o.ck[:] = self.ck
            o.doc_phase(it, int(self.db[me]), int(self.db[me + 1]))
            self._reduce_ck(mine_doc)
            self._exchange(to_words=True)
            o.ck[:] = self.ck
            for w0, w1 in self.word_runs:
                o.word_phase(it, w0, w1)
            self._reduce_ck(mine_word)
            self._exchange(to_words=False)
            o.iteration = it

    def gather(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(z, prop, c_k) of all tokens, assembled from the doc owners."""
        import torch
        o, M = self.o, self.o.M
        owned = self.down == self.rank
        z = np.where(owned, o.z[: o.N], 0).astype(np.int32)
        p = np.where(np.repeat(owned, M), o.prop[: o.N * M], 0).astype(np.int32)
        tz, tp = torch.from_numpy(z), torch.from_numpy(p)
        self.dist.all_reduce(tz)
        self.dist.all_reduce(tp)
        return tz.numpy(), tp.numpy(), self.ck.copy()
