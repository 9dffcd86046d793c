"""Seeded synthetic LDA corpora shaped like the paper's workloads.

The generator (``gen_corpus.c``) follows the LDA generative process of
Sec. 2.1; it is an input generator only and holds none of the sampler's
arithmetic, so both the CUDA sampler and the CPU oracle can be fed from it.

Workloads (Table 3 shapes; the datasets themselves are not used):

* ``tiny``   -- D=1,000, V=5,000, Poisson(100) lengths, K_true=16, Zipf 1.0;
  fit K=16, alpha=50/K, beta=0.01, M=1.
* ``nytimes`` -- D=300K, V=100K, lognormal(mean 330, sigma 0.8) lengths
  (~99M tokens), K_true=200, Zipf 1.05; fit K=1,000, alpha=50/K, beta=0.01, M=2.
* ``pubmed`` -- D=8M, V=140K, lognormal(mean 92, sigma 0.8) (~736M tokens),
  K_true=1,000, Zipf 1.1; fit K=10,000, alpha=0.1, beta=0.01, M=2.
* ``clueweb`` -- D=20M, V=1M, lognormal(mean 75), K_true=5,000, Zipf 1.1;
  fit K=10^6, alpha=0.01, beta=0.01, M=1.

Topic-word rows are Dirichlet(c * V * zipf_s) with c = 0.01 (mean per-word
concentration 0.01, expected word frequencies Zipf), doc-topic Dirichlet(0.1).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_corpus.c")
_OUT = os.path.join(_HERE, "_build", "libgencorpus.so")
_LOCK = threading.Lock()
_LIB = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp,
                    "-lm"], check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            c = ctypes
            lib.gen_lengths.argtypes = [c.c_int64, c.c_int, c.c_double, c.c_double, c.c_int64,
                                        c.c_int64, c.c_uint64, c.c_int64, _i64p]
            lib.gen_topics.argtypes = [c.c_int64, c.c_int, c.c_double, c.c_double, c.c_uint64,
                                       _f32p, _i32p, _i32p, c.c_void_p]
            lib.gen_words.argtypes = [c.c_int64, _i64p, c.c_int64, c.c_int, c.c_double, _f32p,
                                      _i32p, c.c_uint64, c.c_int64, _i32p, c.c_void_p]
            lib.gen_topics_sparse.argtypes = [c.c_int64, c.c_int, c.c_double, c.c_double, c.c_uint64,
                                              c.c_double, c.c_int, _i32p, _i64p, c.c_void_p,
                                              c.c_void_p, c.c_void_p, c.c_void_p]
            lib.gen_words_sparse.argtypes = [c.c_int64, _i64p, c.c_int, c.c_double, _i64p, _i32p,
                                             _f32p, _i32p, c.c_uint64, c.c_int64, _i32p, c.c_void_p]
            _LIB = lib
        return _LIB


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    D: int
    V: int
    K_true: int
    zipf_s: float
    len_kind: int          # 0 Poisson, 1 lognormal, 2 clipped lognormal
    len_mean: float
    len_sigma: float
    K: int
    alpha: float
    beta: float
    M: int
    sweeps: int
    len_lo: int = 1
    len_hi: int = 1 << 40
    conc_c: float = 0.01
    doc_alpha: float = 0.1

    def fit_alpha(self) -> float:
        return float(np.float32(self.alpha))


WORKLOADS = {
    "tiny": Workload("tiny", 1_000, 5_000, 16, 1.0, 0, 100.0, 0.0, 16,
                     float(np.float32(50.0) / np.float32(16)), 0.01, 1, 20),
    "nytimes": Workload("nytimes", 300_000, 100_000, 200, 1.05, 1, 330.0, 0.8, 1000,
                        float(np.float32(50.0) / np.float32(1000)), 0.01, 2, 100),
    "pubmed": Workload("pubmed", 8_000_000, 140_000, 1000, 1.1, 1, 92.0, 0.8, 10_000,
                       0.1, 0.01, 2, 50),
    "clueweb": Workload("clueweb", 20_000_000, 1_000_000, 5000, 1.1, 1, 75.0, 0.8, 1_000_000,
                        0.01, 0.01, 1, 20),
}


@dataclasses.dataclass
class Corpus:
    doc_ptr: np.ndarray     # int64[D+1]
    doc_word: np.ndarray    # int32[N]
    V: int
    true_z: np.ndarray | None = None

    @property
    def D(self) -> int:
        return len(self.doc_ptr) - 1

    @property
    def N(self) -> int:
        return int(self.doc_ptr[-1])


# Above this many K_true x V entries the topic rows are truncated (sparse).
SPARSE_TOPICS_ENTRIES = 1 << 30
SPARSE_TOPICS_CUT = 1e-9


class SparseTopicModel:
    """Topic-word rows with entries below 1e-9 of each row's mass dropped
    (renormalised), for ClueWeb-shaped vocabularies: per topic the kept word
    ids and an alias table over them."""

    def __init__(self, V: int, K_true: int, zipf_s: float, conc_c: float, seed: int,
                 cut: float = SPARSE_TOPICS_CUT):
        self.V, self.K_true, self.cut = int(V), int(K_true), float(cut)
        self.rank_to_word = np.zeros(self.V, dtype=np.int32)
        nnz = np.zeros(self.K_true, dtype=np.int64)
        lib = _lib()
        lib.gen_topics_sparse(self.V, self.K_true, zipf_s, conc_c, seed, self.cut, 0,
                              self.rank_to_word, nnz, None, None, None, None)
        self.off = np.zeros(self.K_true + 1, dtype=np.int64)
        np.cumsum(nnz, out=self.off[1:])
        n = int(self.off[-1])
        self.words = np.zeros(n, dtype=np.int32)
        self.prob = np.zeros(n, dtype=np.float32)
        self.alias = np.zeros(n, dtype=np.int32)
        lib.gen_topics_sparse(self.V, self.K_true, zipf_s, conc_c, seed, self.cut, 1,
                              self.rank_to_word, nnz, self.off.ctypes.data, self.words.ctypes.data,
                              self.prob.ctypes.data, self.alias.ctypes.data)


class TopicModel:
    """The generating topic-word rows (alias tables) of one workload."""

    def __init__(self, V: int, K_true: int, zipf_s: float, conc_c: float, seed: int,
                 keep_phi: bool = False):
        self.V, self.K_true = int(V), int(K_true)
        self.prob = np.zeros(self.K_true * self.V, dtype=np.float32)
        self.alias = np.zeros(self.K_true * self.V, dtype=np.int32)
        self.rank_to_word = np.zeros(self.V, dtype=np.int32)
        self.phi = np.zeros(self.K_true * self.V, dtype=np.float64) if keep_phi else None
        _lib().gen_topics(self.V, self.K_true, zipf_s, conc_c, seed, self.prob, self.alias,
                          self.rank_to_word,
                          self.phi.ctypes.data if self.phi is not None else None)


def topic_model(wl: Workload, seed: int):
    """Dense alias tables, or truncated rows when K_true x V is too large."""
    if wl.K_true * wl.V > SPARSE_TOPICS_ENTRIES:
        return SparseTopicModel(wl.V, wl.K_true, wl.zipf_s, wl.conc_c, seed)
    return TopicModel(wl.V, wl.K_true, wl.zipf_s, wl.conc_c, seed)


def lengths(D: int, kind: int, mean: float, sigma: float, seed: int, doc_offset: int = 0,
            lo: int = 1, hi: int = 1 << 40) -> np.ndarray:
    out = np.zeros(D, dtype=np.int64)
    _lib().gen_lengths(D, kind, mean, sigma, lo, hi, seed, doc_offset, out)
    return out


def generate_docs(model: TopicModel, lens: np.ndarray, doc_alpha: float, seed: int,
                  doc_offset: int = 0, keep_z: bool = False) -> Corpus:
    D = len(lens)
    doc_ptr = np.zeros(D + 1, dtype=np.int64)
    np.cumsum(lens, out=doc_ptr[1:])
    N = int(doc_ptr[-1])
    doc_word = np.zeros(max(N, 1), dtype=np.int32)
    tz = np.zeros(max(N, 1), dtype=np.int32) if keep_z else None
    if isinstance(model, SparseTopicModel):
        _lib().gen_words_sparse(D, doc_ptr, model.K_true, doc_alpha, model.off, model.words,
                                model.prob, model.alias, seed, doc_offset, doc_word,
                                tz.ctypes.data if tz is not None else None)
    else:
        _lib().gen_words(D, doc_ptr, model.V, model.K_true, doc_alpha, model.prob, model.alias,
                         seed, doc_offset, doc_word, tz.ctypes.data if tz is not None else None)
    return Corpus(doc_ptr, doc_word[:N], model.V, tz[:N] if tz is not None else None)


def generate(name: str, seed: int = 1234, D: int | None = None, doc_offset: int = 0,
             keep_z: bool = False) -> tuple[Corpus, Workload]:
    """Corpus of a named workload; ``D`` overrides the document count (the
    first D documents of the full corpus, same generator streams)."""
    wl = WORKLOADS[name]
    nd = wl.D if D is None else int(D)
    model = topic_model(wl, seed)
    lens = lengths(nd, wl.len_kind, wl.len_mean, wl.len_sigma, seed, doc_offset, wl.len_lo,
                   wl.len_hi)
    return generate_docs(model, lens, wl.doc_alpha, seed, doc_offset, keep_z), wl


def from_lengths(lens, V: int, seed: int, K_true: int = 8, zipf_s: float = 1.0,
                 doc_alpha: float = 0.1) -> Corpus:
    """Small corpus with given document lengths (edge-case tests)."""
    model = TopicModel(V, K_true, zipf_s, 0.01, seed)
    return generate_docs(model, np.asarray(lens, dtype=np.int64), doc_alpha, seed)


def requests(name: str, seed: int, n: int, doc_offset: int, lo: int = 20, hi: int = 5000) -> Corpus:
    """Unseen documents of a workload's generator (its topics, its length law
    clipped to [lo, hi]) -- fold-in requests; doc_offset keeps their streams
    apart from the training corpus."""
    wl = WORKLOADS[name]
    model = topic_model(wl, seed)
    lens = np.clip(lengths(n, wl.len_kind, wl.len_mean, wl.len_sigma, seed, doc_offset), lo, hi)
    return generate_docs(model, lens, wl.doc_alpha, seed, doc_offset)
