"""Plain CPU WarpLDA oracle -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import this package.
The product path (``paper_1510_08628_gb300``) never imports it, and this
package imports nothing from the product.

The arithmetic lives in ``warplda_oracle.c`` (plain C, FP32 accept tests with
``-ffp-contract=off``, FP64 log-likelihood); this module only builds it with
gcc and marshals numpy arrays through ctypes.  See the C file's header for the
paper passages each function follows and the readings taken.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "warplda_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

PHASE_INIT, PHASE_DOC, PHASE_WORD = 0, 1, 2

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def lib_path(mutation: int = 0) -> str:
    name = "liborc.so" if mutation == 0 else f"liborc_m{mutation}.so"
    return os.path.join(_BUILD, name)


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no FP contraction)."""
    out = lib_path(mutation)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", f"-DORC_MUTATION={mutation}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutation: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutation in _LIBS:
            return _LIBS[mutation]
        lib = ctypes.CDLL(build(mutation))
        c = ctypes
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_accept.argtypes = [c.c_uint32, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int,
                                   c.c_int, c.c_float, c.c_float]
        lib.orc_accept.restype = c.c_int
        lib.orc_draw_mixture.argtypes = [c.c_uint32, c.c_uint32, _i32p, c.c_int, c.c_int,
                                         c.c_float]
        lib.orc_draw_mixture.restype = c.c_int
        lib.orc_word_major.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, _i64p, _i32p]
        lib.orc_word_major.restype = c.c_int
        lib.orc_init.argtypes = [c.c_int64, c.c_int, c.c_int, c.c_uint64, _i32p, _i32p]
        lib.orc_topic_counts.argtypes = [c.c_int64, c.c_int, _i32p, _i32p]
        lib.orc_doc_phase.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, c.c_int, c.c_int,
                                      c.c_float, c.c_float, c.c_float, c.c_uint64, c.c_uint32,
                                      _i32p, _i32p, _i32p]
        lib.orc_word_phase.argtypes = [c.c_int64, c.c_int64, _i64p, c.c_int, c.c_int,
                                       c.c_float, c.c_float, c.c_float, c.c_uint64, c.c_uint32,
                                       _i32p, _i32p, _i32p]
        lib.orc_sweeps.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, _i64p, c.c_int, c.c_int,
                                   c.c_float, c.c_float, c.c_float, c.c_float, c.c_float,
                                   c.c_uint64, c.c_uint32, c.c_int, _i32p, _i32p, _i32p]
        lib.orc_loglik.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, _i64p, c.c_int,
                                   c.c_float, c.c_float, _i32p]
        lib.orc_loglik.restype = c.c_double
        lib.orc_token_chains.argtypes = [c.c_int, c.c_int, _i32p, _i32p, _i32p, _i32p, c.c_int,
                                         _i32p, c.c_int, c.c_float, c.c_float, c.c_float,
                                         c.c_float, c.c_float, c.c_uint64, c.c_uint32,
                                         c.c_int64, c.c_int, _i32p, _i32p]
        lib.orc_cgs_sweeps.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, _i32p, c.c_int,
                                       c.c_float, c.c_float, c.c_uint64, c.c_uint32, c.c_int,
                                       _i32p]
        _f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
        _f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        lib.orc_frozen_word_draw.argtypes = [c.c_uint32, c.c_uint32, _i32p, c.c_int, c.c_float]
        lib.orc_frozen_word_draw.restype = c.c_int
        lib.orc_foldin.argtypes = [c.c_int64, _i64p, _i32p, _i64p, c.c_int, c.c_int, c.c_float,
                                   c.c_float, c.c_float, c.c_float, c.c_float, _i32p, _i32p,
                                   c.c_uint64, c.c_int, _i32p, c.c_void_p]
        lib.orc_cgs_foldin.argtypes = [c.c_int64, _i64p, _i32p, c.c_int, c.c_float, c.c_float,
                                       c.c_float, _i32p, _i32p, c.c_uint64, c.c_int, c.c_int,
                                       _f64p]
        lib.orc_alias_build.argtypes = [_f32p, c.c_int, _f32p, _i32p]
        lib.orc_alias_draw.argtypes = [c.c_uint32, c.c_uint32, _f32p, _i32p, c.c_int]
        lib.orc_alias_draw.restype = c.c_int
        lib.orc_foldin_learned.argtypes = [c.c_int64, _i64p, _i32p, _i64p, c.c_int, c.c_int,
                                           c.c_float, c.c_float, c.c_float, c.c_float, c.c_float,
                                           _i32p, _i32p, _f32p, c.c_uint64, c.c_int, _i32p,
                                           c.c_void_p]
        lib.orc_word_phase_rule.argtypes = [c.c_int64, c.c_int64, _i64p, c.c_int, c.c_int,
                                            c.c_float, c.c_float, c.c_float, c.c_uint64, c.c_uint32,
                                            _i32p, _i32p, _i32p, c.c_int]
        lib.orc_sweeps_rule.argtypes = [c.c_int64, c.c_int64, _i64p, _i32p, _i64p, c.c_int, c.c_int,
                                        c.c_float, c.c_float, c.c_float, c.c_float, c.c_float,
                                        c.c_uint64, c.c_uint32, c.c_int, _i32p, _i32p, _i32p, c.c_int]
        lib.orc_num_threads.restype = c.c_int
        lib.orc_set_num_threads.argtypes = [c.c_int]
        _LIBS[mutation] = lib
        return lib


def f32(x) -> float:
    """Round a Python float to the FP32 value both sides receive."""
    return float(np.float32(x))


def derived(K: int, V: int, alpha: float, beta: float) -> tuple[float, float, float]:
    """alpha_bar = K*alpha, beta_bar = V*beta, K_beta = K*beta, each one FP32 product."""
    a, b = np.float32(alpha), np.float32(beta)
    return (float(np.float32(K) * a), float(np.float32(V) * b), float(np.float32(K) * b))


class Oracle:
    """WarpLDA state held as numpy arrays, advanced by the C oracle.

    Arrays: z[N] and prop[N*M] in word-major order, perm[N] (doc-major
    position -> word-major index), word_ptr[V+1], ck[K].
    """

    def __init__(self, doc_ptr, doc_word, V, K, alpha, beta, M, seed, mutation: int = 0,
                 word_rule: int = 0):
        self.lib = load(mutation)
        self.word_rule = int(word_rule)   # 0: j-th smallest topic (R7); 1: storage order (R7')
        self.doc_ptr = np.ascontiguousarray(doc_ptr, dtype=np.int64)
        self.doc_word = np.ascontiguousarray(doc_word, dtype=np.int32)
        self.D = len(self.doc_ptr) - 1
        self.V, self.K, self.M = int(V), int(K), int(M)
        self.N = int(self.doc_ptr[-1])
        self.alpha, self.beta = f32(alpha), f32(beta)
        self.alpha_bar, self.beta_bar, self.K_beta = derived(self.K, self.V, alpha, beta)
        self.seed = int(seed)
        self.word_ptr = np.zeros(self.V + 1, dtype=np.int64)
        self.perm = np.zeros(max(self.N, 1), dtype=np.int32)
        rc = self.lib.orc_word_major(self.D, self.V, self.doc_ptr, self.doc_word, self.word_ptr,
                                     self.perm)
        if rc != 0:
            raise ValueError("word id outside [0, V)")
        self.z = np.zeros(max(self.N, 1), dtype=np.int32)
        self.prop = np.zeros(max(self.N * self.M, 1), dtype=np.int32)
        self.ck = np.zeros(self.K, dtype=np.int32)
        self.lib.orc_init(self.N, self.K, self.M, self.seed, self.z, self.prop)
        self.lib.orc_topic_counts(self.N, self.K, self.z, self.ck)
        self.iteration = 0

    # one phase at a time (used by the invariant tests and sampled parity)
    def doc_phase(self, it=None, d0=0, d1=None):
        it = self.iteration + 1 if it is None else it
        d1 = self.D if d1 is None else d1
        self.lib.orc_doc_phase(d0, d1, self.doc_ptr, self.perm, self.K, self.M, self.alpha,
                               self.alpha_bar, self.beta_bar, self.seed, it, self.z, self.prop,
                               self.ck)

    def word_phase(self, it=None, w0=0, w1=None):
        it = self.iteration + 1 if it is None else it
        w1 = self.V if w1 is None else w1
        self.lib.orc_word_phase_rule(w0, w1, self.word_ptr, self.K, self.M, self.beta, self.K_beta,
                                     self.beta_bar, self.seed, it, self.z, self.prop, self.ck,
                                     self.word_rule)

    def recount(self):
        self.lib.orc_topic_counts(self.N, self.K, self.z, self.ck)

    def sweep(self, n: int = 1):
        self.lib.orc_sweeps_rule(self.D, self.V, self.doc_ptr, self.perm, self.word_ptr, self.K,
                                 self.M, self.alpha, self.beta, self.alpha_bar, self.beta_bar,
                                 self.K_beta, self.seed, self.iteration, n, self.z, self.prop,
                                 self.ck, self.word_rule)
        self.iteration += n

    def loglik(self) -> float:
        return float(self.lib.orc_loglik(self.D, self.V, self.doc_ptr, self.perm, self.word_ptr,
                                         self.K, self.alpha, self.beta, self.z))

    def z_docmajor(self) -> np.ndarray:
        return self.z[self.perm[: self.N]].copy()


def philox(ctr, key, mutation: int = 0) -> np.ndarray:
    lib = load(mutation)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def set_threads(n: int) -> None:
    load().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(load().orc_num_threads())


def word_topic_counts(z_wordmajor, word_ptr, V: int, K: int) -> np.ndarray:
    """Dense C_w [V, K] (int32) of word-major topics (the frozen model of fold-in)."""
    z = np.asarray(z_wordmajor, dtype=np.int64)
    wp = np.asarray(word_ptr, dtype=np.int64)
    w = np.repeat(np.arange(V, dtype=np.int64), np.diff(wp))
    cw = np.zeros(V * K, dtype=np.int64)
    np.add.at(cw, w * K + z[: len(w)], 1)
    return cw.reshape(V, K).astype(np.int32)


def foldin(doc_ptr, doc_word, cw, ck, K: int, M: int, alpha: float, beta: float, V: int,
           seed: int, sweeps: int, doc_ids=None, theta: bool = True, mutation: int = 0):
    """Fold-in of new documents against frozen counts (orc_foldin): (z, theta)."""
    lib = load(mutation)
    dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
    dw = np.ascontiguousarray(doc_word, dtype=np.int32)
    Dn = len(dp) - 1
    ids = np.arange(Dn, dtype=np.int64) if doc_ids is None else np.ascontiguousarray(doc_ids, dtype=np.int64)
    abar, bbar, kbeta = derived(K, V, alpha, beta)
    z = np.zeros(max(int(dp[-1]), 1), dtype=np.int32)
    th = np.zeros(max(Dn * K, 1), dtype=np.float32) if theta else None
    lib.orc_foldin(Dn, dp, dw if len(dw) else np.zeros(1, np.int32), ids, K, M, f32(alpha), abar,
                   f32(beta), kbeta, bbar, np.ascontiguousarray(cw, dtype=np.int32).ravel(),
                   np.ascontiguousarray(ck, dtype=np.int32), seed, sweeps, z,
                   th.ctypes.data if th is not None else None)
    return z[: int(dp[-1])], (th[: Dn * K].reshape(Dn, K) if th is not None else None)


def cgs_foldin_theta(doc_ptr, doc_word, cw, ck, K: int, alpha: float, beta: float, V: int,
                     seed: int, sweeps: int, burn: int) -> np.ndarray:
    """Mean theta over sweeps burn+1..sweeps of a plain collapsed Gibbs fold-in."""
    lib = load()
    dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
    Dn = len(dp) - 1
    acc = np.zeros(Dn * K, dtype=np.float64)
    _, bbar, _ = derived(K, V, alpha, beta)
    lib.orc_cgs_foldin(Dn, dp, np.ascontiguousarray(doc_word, dtype=np.int32), K, f32(alpha),
                       f32(beta), bbar, np.ascontiguousarray(cw, dtype=np.int32).ravel(),
                       np.ascontiguousarray(ck, dtype=np.int32), seed, sweeps, burn, acc)
    return (acc / max(sweeps - burn, 1)).reshape(Dn, K)


def alias_table(q, mutation: int = 0):
    """Walker/Vose alias table of q (orc_alias_build): (prob, alias)."""
    q = np.ascontiguousarray(q, dtype=np.float32)
    K = len(q)
    prob = np.zeros(K, dtype=np.float32)
    alias = np.zeros(K, dtype=np.int32)
    load(mutation).orc_alias_build(q, K, prob, alias)
    return prob, alias


def foldin_learned(doc_ptr, doc_word, cw, ck, q, K: int, M: int, alpha: float, beta: float,
                   V: int, seed: int, sweeps: int, doc_ids=None, theta: bool = True,
                   mutation: int = 0):
    """Fold-in with the learned proposal q[Dn, K] (orc_foldin_learned): (z, theta)."""
    lib = load(mutation)
    dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
    dw = np.ascontiguousarray(doc_word, dtype=np.int32)
    Dn = len(dp) - 1
    ids = np.arange(Dn, dtype=np.int64) if doc_ids is None else np.ascontiguousarray(doc_ids, dtype=np.int64)
    abar, bbar, kbeta = derived(K, V, alpha, beta)
    z = np.zeros(max(int(dp[-1]), 1), dtype=np.int32)
    th = np.zeros(max(Dn * K, 1), dtype=np.float32) if theta else None
    lib.orc_foldin_learned(Dn, dp, dw if len(dw) else np.zeros(1, np.int32), ids, K, M,
                           f32(alpha), f32(beta), abar, kbeta, bbar,
                           np.ascontiguousarray(cw, dtype=np.int32).ravel(),
                           np.ascontiguousarray(ck, dtype=np.int32),
                           np.ascontiguousarray(q, dtype=np.float32).ravel(), seed, sweeps, z,
                           th.ctypes.data if th is not None else None)
    return z[: int(dp[-1])], (th[: Dn * K].reshape(Dn, K) if th is not None else None)
