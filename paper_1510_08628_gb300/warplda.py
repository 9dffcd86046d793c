"""Python binding of libwarplda.so (include/warplda.h): argument marshalling only.

Every step of the sampler runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers and return codes to
exceptions.  There is no CPU fallback: if the library or a GPU is missing the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, ESTATE, EIO = 0, -1, -2, -3, -4, -5, -6
EINTERNAL = -8
PHASE_DOC, PHASE_WORD = 1, 2

_LOCK = threading.Lock()
_LIB = None


class WarpLDAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"warplda error {code}: {msg}")
        self.code = code


class Tuning(ctypes.Structure):
    _fields_ = [("batch_max_tokens", ctypes.c_int32), ("huge_chunk", ctypes.c_int32),
                ("region_budget", ctypes.c_int32), ("doc_warp_max", ctypes.c_int32),
                ("word_positioning", ctypes.c_int32), ("doc_batch_kernel", ctypes.c_int32),
                ("cluster_max_tokens", ctypes.c_int32), ("foldin_kernel", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int64), ("V", ctypes.c_int64), ("N", ctypes.c_int64),
                ("K", ctypes.c_int32), ("M", ctypes.c_int32),
                ("launches_per_sweep", ctypes.c_int32), ("batch_max_tokens", ctypes.c_int32),
                ("doc_batches", ctypes.c_int64), ("word_batches", ctypes.c_int64),
                ("huge_docs", ctypes.c_int64), ("huge_doc_tokens", ctypes.c_int64),
                ("mega_words", ctypes.c_int64), ("mega_word_tokens", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("pipe_doc_tokens", ctypes.c_int64),
                ("cluster_words", ctypes.c_int64), ("cluster_word_tokens", ctypes.c_int64),
                ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


# Symbols declared in include/warplda.h, with their ctypes signatures.
_P = ctypes.c_void_p
_SIGS = {
    "warplda_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_int32, ctypes.c_uint64, _P, _P]),
    "warplda_sweep": (ctypes.c_int, [_P, ctypes.c_int32]),
    "warplda_phase": (ctypes.c_int, [_P, ctypes.c_int32]),
    "warplda_counts": (ctypes.c_int, [_P, _P, _P]),
    "warplda_counts_dev": (ctypes.c_int, [_P, _P, _P]),
    "warplda_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "warplda_set_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32]),
    "warplda_token_order": (ctypes.c_int, [_P, _P, _P]),
    "warplda_doc_batches": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "warplda_loglik": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "warplda_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "warplda_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "warplda_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "warplda_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "warplda_kernel_times": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_char_p),
                                            ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_double)]),
    "warplda_sync": (ctypes.c_int, [_P]),
    "warplda_server_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, _P]),
    "warplda_server_submit": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P]),
    "warplda_server_step": (ctypes.c_int, [_P, _P]),
    "warplda_server_poll": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32]),
    "warplda_server_destroy": (None, [_P]),
    "warplda_word_counts": (ctypes.c_int, [_P, _P]),
    "warplda_encoder_init": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_uint64]),
    "warplda_encoder_weights": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "warplda_encoder_grad": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "warplda_encoder_train": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _P]),
    "warplda_encoder_proposal": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
    "warplda_gemm_bf16": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, _P]),
    "warplda_foldin": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_int32, _P, _P]),
    "warplda_destroy": (None, [_P]),
    "warplda_loglik_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                              _P, _P, _P, _P, _P, _P]),
    "warplda_last_error": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libwarplda.so (building it with nvcc if it is missing)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise WarpLDAError(ECUDA, f"{path} not built")
            path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
        return lib


def _check(rc: int) -> int:
    if rc < 0:
        msg = load().warplda_last_error()
        raise WarpLDAError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


def loglik_noalloc(D: int, V: int, N: int, K: int, alpha: float, beta: float, doc_ptr_dev,
                   z_docmajor_dev, word_ptr_dev, z_wordmajor_dev, out_dev, stream=None) -> None:
    """warplda_loglik_noalloc on device tensors (no allocation; asynchronous)."""
    st = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(load().warplda_loglik_noalloc(int(D), int(V), int(N), int(K), ctypes.c_float(alpha),
                                         ctypes.c_float(beta), _dev_ptr(doc_ptr_dev),
                                         _dev_ptr(z_docmajor_dev), _dev_ptr(word_ptr_dev),
                                         _dev_ptr(z_wordmajor_dev), _dev_ptr(out_dev), st))


class WarpLDA:
    """One sampler context (warplda_ctx) on the current CUDA device."""

    def __init__(self, doc_ptr, doc_word, V: int, K: int, alpha: float, beta: float, M: int,
                 seed: int, stream=None, tuning: dict | None = None):
        lib = load()
        self.doc_ptr = np.ascontiguousarray(doc_ptr, dtype=np.int64)
        doc_word = np.ascontiguousarray(doc_word, dtype=np.int32)
        self.D = len(self.doc_ptr) - 1
        self.N = int(self.doc_ptr[-1])
        self.V, self.K, self.M = int(V), int(K), int(M)
        tun = None
        if tuning:
            tun = Tuning()
            for k, v in tuning.items():
                setattr(tun, k, int(v))
        st = None
        if stream is not None:
            st = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        h = ctypes.c_void_p()
        _check(lib.warplda_init(ctypes.byref(h), self.D, self.V, self.N, _ptr(self.doc_ptr),
                                _ptr(doc_word), self.K, ctypes.c_float(alpha),
                                ctypes.c_float(beta), self.M, ctypes.c_uint64(seed & (2**64 - 1)),
                                st, ctypes.byref(tun) if tun is not None else None))
        self._h = h

    # -- sampler --------------------------------------------------------------
    def sweep(self, n: int = 1) -> None:
        _check(load().warplda_sweep(self._h, int(n)))

    def phase(self, which: int) -> None:
        _check(load().warplda_phase(self._h, int(which)))

    # -- results --------------------------------------------------------------
    def counts(self, want_z: bool = True, want_ck: bool = True, z_out=None, ck_out=None):
        """z in document order and c_k on the host.  z_out / ck_out: optional
        caller-held int32 arrays (e.g. views of pinned memory, which the copy
        reaches at full speed) of N and K entries to fill instead."""
        def buf(out, n, want):
            if out is not None:
                if out.dtype != np.int32 or not out.flags["C_CONTIGUOUS"] or out.size < n:
                    raise ValueError(f"output buffer must be contiguous int32 with >= {n} entries")
                return out
            return np.empty(max(n, 1), dtype=np.int32) if want else None
        z = buf(z_out, self.N, want_z)
        ck = buf(ck_out, self.K, want_ck)
        _check(load().warplda_counts(self._h, _ptr(z), _ptr(ck)))
        return (z[: self.N] if z is not None else None), (ck[: self.K] if ck is not None else None)

    def counts_dev(self, z_dev=None, ck_dev=None) -> None:
        _check(load().warplda_counts_dev(self._h, _dev_ptr(z_dev), _dev_ptr(ck_dev)))

    def get_state(self):
        z = np.empty(max(self.N, 1), dtype=np.int32)
        p = np.empty(max(self.N * self.M, 1), dtype=np.int32)
        ck = np.empty(self.K, dtype=np.int32)
        it = ctypes.c_uint32()
        _check(load().warplda_get_state(self._h, _ptr(z), _ptr(p), _ptr(ck), ctypes.byref(it)))
        return z[: self.N], p[: self.N * self.M], ck, int(it.value)

    def set_state(self, z, prop, sweeps_done: int) -> None:
        z = np.ascontiguousarray(z, dtype=np.int32)
        prop = np.ascontiguousarray(prop, dtype=np.int32)
        _check(load().warplda_set_state(self._h, _ptr(z), _ptr(prop), int(sweeps_done)))

    def token_order(self):
        wp = np.empty(self.V + 1, dtype=np.int64)
        perm = np.empty(max(self.N, 1), dtype=np.int32)
        _check(load().warplda_token_order(self._h, _ptr(wp), _ptr(perm)))
        return wp, perm[: self.N]

    def doc_batches(self):
        """(batches [n, 4], sperm [N], sinfo [N]) of the document batch tier."""
        nb = ctypes.c_int64()
        _check(load().warplda_doc_batches(self._h, ctypes.byref(nb), None, None, None))
        n = int(nb.value)
        b = np.empty((max(n, 1), 4), dtype=np.int32)
        sp = np.empty(max(self.N, 1), dtype=np.int32)
        si = np.empty(max(self.N, 1), dtype=np.uint32)
        _check(load().warplda_doc_batches(self._h, None, _ptr(b), _ptr(sp), _ptr(si)))
        return b[:n], sp[: self.N], si[: self.N]

    def loglik(self) -> float:
        out = ctypes.c_double()
        _check(load().warplda_loglik(self._h, ctypes.byref(out)))
        return float(out.value)

    def save(self, path: str) -> None:
        _check(load().warplda_save(self._h, path.encode()))

    def load_state(self, path: str) -> None:
        _check(load().warplda_load(self._h, path.encode()))

    def foldin(self, doc_ptr, doc_word, sweeps: int, seed: int, doc_ids=None,
               theta: bool = True, z: bool = True, learned: bool = False, theta_out=None, z_out=None):
        """Fold in new documents against the current model: (theta[Dn, K], z[Nn]);
        learned=True uses the encoder's proposal.  theta_out / z_out: the
        caller's float32 [Dn, K] / int32 [Nn] arrays to fill (e.g. pinned)."""
        dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
        dw = np.ascontiguousarray(doc_word, dtype=np.int32)
        Dn, Nn = len(dp) - 1, int(dp[-1])
        ids = None if doc_ids is None else np.ascontiguousarray(doc_ids, dtype=np.int64)
        th = zo = None
        if theta:
            th = theta_out if theta_out is not None else np.empty((Dn, self.K), dtype=np.float32)
            if th.dtype != np.float32 or th.shape != (Dn, self.K) or not th.flags.c_contiguous:
                raise ValueError("theta_out must be a C-contiguous float32 [Dn, K] array")
        if z:
            zo = z_out if z_out is not None else np.empty(Nn, dtype=np.int32)
            if zo.dtype != np.int32 or zo.shape != (Nn,) or not zo.flags.c_contiguous:
                raise ValueError("z_out must be a C-contiguous int32 [Nn] array")
        ptr = lambda a: a.ctypes.data if a is not None and a.size else None
        _check(load().warplda_foldin(self._h, Dn, ptr(dp), ptr(dw), ptr(ids), int(sweeps),
                                     int(seed), 1 if learned else 0, ptr(th), ptr(zo)))
        return th, zo

    # ---- fold-in encoder (learned document proposal) ----
    def encoder_init(self, log2_features: int = 16, hidden: int = 512, batch_rows: int = 256,
                     seed: int = 1) -> None:
        self._enc = (int(log2_features), int(hidden))
        _check(load().warplda_encoder_init(self._h, log2_features, hidden, batch_rows, int(seed)))

    def encoder_weights(self, set_to=None):
        F, H = 1 << self._enc[0], self._enc[1]
        if set_to is not None:
            W1, b1, W2, b2 = (np.ascontiguousarray(a, dtype=np.float32) for a in set_to)
            _check(load().warplda_encoder_weights(self._h, 1, W1.ctypes.data, b1.ctypes.data,
                                                  W2.ctypes.data, b2.ctypes.data))
            return None
        W1 = np.empty((F, H), np.float32)
        b1 = np.empty(H, np.float32)
        W2 = np.empty((H, self.K), np.float32)
        b2 = np.empty(self.K, np.float32)
        _check(load().warplda_encoder_weights(self._h, 0, W1.ctypes.data, b1.ctypes.data,
                                              W2.ctypes.data, b2.ctypes.data))
        return W1, b1, W2, b2

    def encoder_grad(self, doc_ptr, doc_word, theta):
        F, H = 1 << self._enc[0], self._enc[1]
        dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
        dw = np.ascontiguousarray(doc_word, dtype=np.int32)
        th = np.ascontiguousarray(theta, dtype=np.float32)
        loss = ctypes.c_double()
        g = (np.empty((F, H), np.float32), np.empty(H, np.float32),
             np.empty((H, self.K), np.float32), np.empty(self.K, np.float32))
        _check(load().warplda_encoder_grad(self._h, len(dp) - 1, dp.ctypes.data, dw.ctypes.data,
                                           th.ctypes.data, ctypes.byref(loss),
                                           *(a.ctypes.data for a in g)))
        return float(loss.value), g

    def encoder_train(self, epochs: int, lr: float, seed: int = 1):
        out = np.zeros(max(epochs, 1), np.float64)
        _check(load().warplda_encoder_train(self._h, int(epochs), ctypes.c_float(lr), int(seed),
                                            out.ctypes.data))
        return out[:epochs]

    def encoder_proposal(self, doc_ptr, doc_word):
        dp = np.ascontiguousarray(doc_ptr, dtype=np.int64)
        dw = np.ascontiguousarray(doc_word, dtype=np.int32)
        q = np.empty((len(dp) - 1, self.K), np.float32)
        _check(load().warplda_encoder_proposal(self._h, len(dp) - 1, dp.ctypes.data,
                                               dw.ctypes.data if dw.size else None,
                                               q.ctypes.data if q.size else None))
        return q

    def word_counts(self):
        """C_w [V, K] (int32) of the current state."""
        cw = np.empty((self.V, self.K), np.int32)
        _check(load().warplda_word_counts(self._h, cw.ctypes.data))
        return cw

    def sync(self) -> None:
        """Wait for queued work; raise if a kernel's index check failed."""
        _check(load().warplda_sync(self._h))

    def info(self) -> dict:
        inf = Info()
        _check(load().warplda_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def profile(self, enable: bool) -> None:
        _check(load().warplda_profile(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n = _check(load().warplda_kernel_times(self._h, cap, names, launches, ms))
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n, cap))}

    def close(self) -> None:
        """Destroys the context; its servers (which hold pointers into it)
        are destroyed first."""
        for srv in list(getattr(self, "_servers", {}).values()):
            srv.close()
        if getattr(self, "_h", None):
            load().warplda_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gemm_bf16(A, B, C, bias=None, stream=None) -> None:
    """C = A @ B.T (+ bias) on the tensor cores; torch tensors on the device
    (A, B bfloat16 [M, K] / [N, K], C float32 [M, N])."""
    M, K = A.shape
    N = B.shape[0]
    st = stream.cuda_stream if stream is not None else None
    _check(load().warplda_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                    bias.data_ptr() if bias is not None else None, M, N, K, st))


EBUSY = -7


class Server:
    """Continuous batching of fold-in requests (warplda_server_*): submit()
    admits a request if a slot and pool memory are free (False otherwise),
    step() advances every admitted request by one sweep, poll() returns the
    finished ones as (ids, theta)."""

    def __init__(self, model: "WarpLDA", slots: int, pool_tokens: int, max_doc_tokens: int,
                 sweeps: int, seed: int, learned: bool = False):
        self.K = model.K
        self._model = model
        if not getattr(model, "_h", None):
            raise WarpLDAError(ESTATE, "the model context is closed")
        h = ctypes.c_void_p()
        _check(load().warplda_server_create(model._h, slots, pool_tokens, max_doc_tokens, sweeps,
                                            int(seed), 1 if learned else 0, ctypes.byref(h)))
        self._h = h
        if not hasattr(model, "_servers"):
            model._servers = weakref.WeakValueDictionary()
        model._servers[id(self)] = self
        self._slots = slots

    def submit(self, rid: int, words) -> bool:
        w = np.ascontiguousarray(words, dtype=np.int32)
        rc = load().warplda_server_submit(self._h, int(rid), len(w), w.ctypes.data if w.size else None)
        if rc == EBUSY:
            return False
        _check(rc)
        return True

    def step(self) -> int:
        n = ctypes.c_int32()
        _check(load().warplda_server_step(self._h, ctypes.byref(n)))
        return int(n.value)

    def poll(self, timeout_ms: int = 60000):
        ids = np.empty(self._slots, np.int64)
        th = np.empty((self._slots, self.K), np.float32)
        n = ctypes.c_int32()
        _check(load().warplda_server_poll(self._h, self._slots, ids.ctypes.data, th.ctypes.data,
                                          ctypes.byref(n), int(timeout_ms)))
        return ids[: n.value], th[: n.value]

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().warplda_server_destroy(self._h)
            self._h = None
            srvs = getattr(getattr(self, "_model", None), "_servers", None)
            if srvs is not None:
                srvs.pop(id(self), None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
