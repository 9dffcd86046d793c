"""Plain NumPy (FP64) oracle of the fold-in encoder -- test infrastructure only.

Only ``tests/`` and ``bench.py``'s CPU legs may import this module.  The
paper has no encoder; this is the learned document proposal of the scope's
next row 2, with these readings:

  L1  features: word w hashes to f(w) = ((w * 2654435761) mod 2^32) >> (32 - log2F);
      a document's input is x_f = (# of its tokens with f(w) = f) / L_d.
  L2  network: h_pre = b1 + W1^T x (W1: [F, H]), h = ReLU(h_pre),
      logits = b2 + W2^T h (W2: [H, K]), q = softmax(logits).  The device
      computes with BF16 weights and FP32 accumulation and rounds h to BF16
      before the second layer (a tensor-core GEMM); ``bf16=True`` makes this
      oracle round at the same points (weights, h, and the backward GEMMs'
      dlogits), ``bf16=False`` computes plain FP64 (used by the
      finite-difference pin).
  L3  loss: soft cross-entropy against the training document's theta of
      Eq. 4, loss = -(1/B) sum_d sum_k theta_dk log q_dk.
  L4  gradients: back-propagation of L3 (dlogits = (q - theta) / B).
  L5  optimiser: Adam (Kingma & Ba 2015, Alg. 1) on FP32 master weights,
      beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.

Everything here is written out step by step to be checked by eye.
"""
from __future__ import annotations

import numpy as np

HASH_MUL = 2654435761


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), as float64."""
    a = np.asarray(x, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((bits >> 16) & 1)
    out = ((bits + rounding) & 0xFFFF0000).astype(np.uint32)
    return out.view(np.float32).astype(np.float64)


def feature(words, log2F: int) -> np.ndarray:
    """L1 feature hash of word ids."""
    w = np.asarray(words, dtype=np.uint64)
    return ((w * np.uint64(HASH_MUL)) & np.uint64(0xFFFFFFFF)) >> np.uint64(32 - log2F)


def inputs(doc_ptr, doc_word, log2F: int) -> np.ndarray:
    """Dense x [B, F] of L1 (small problems only)."""
    F = 1 << log2F
    B = len(doc_ptr) - 1
    x = np.zeros((B, F))
    f = feature(doc_word, log2F)
    for d in range(B):
        b, e = int(doc_ptr[d]), int(doc_ptr[d + 1])
        for t in range(b, e):
            x[d, f[t]] += 1.0
        if e > b:
            x[d] /= float(e - b)
    return x


def forward(p: dict, x: np.ndarray, bf: bool = True) -> dict:
    """L2 forward pass; returns every intermediate."""
    W1 = bf16(p["W1"]) if bf else np.asarray(p["W1"], dtype=np.float64)
    W2 = bf16(p["W2"]) if bf else np.asarray(p["W2"], dtype=np.float64)
    h_pre = np.asarray(p["b1"], dtype=np.float64) + x @ W1
    h = np.maximum(h_pre, 0.0)
    hb = bf16(h) if bf else h
    logits = np.asarray(p["b2"], dtype=np.float64) + hb @ W2
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    q = e / e.sum(axis=1, keepdims=True)
    return {"W1": W1, "W2": W2, "h_pre": h_pre, "h": h, "hb": hb, "logits": logits, "q": q}


def loss(q: np.ndarray, theta: np.ndarray) -> float:
    """L3 soft cross-entropy, averaged over the batch."""
    return float(-(theta * np.log(q)).sum() / q.shape[0])


def backward(p: dict, x: np.ndarray, theta: np.ndarray, bf: bool = True) -> tuple[float, dict]:
    """L4 gradients of L3 with respect to W1, b1, W2, b2."""
    f = forward(p, x, bf)
    B = x.shape[0]
    dlogits = (f["q"] - theta) / B
    dlb = bf16(dlogits) if bf else dlogits
    g = {"b2": dlogits.sum(axis=0), "W2": f["hb"].T @ dlb}
    dh = dlb @ f["W2"].T
    dh_pre = dh * (f["h_pre"] > 0.0)
    g["b1"] = dh_pre.sum(axis=0)
    g["W1"] = x.T @ dh_pre
    return loss(f["q"], theta), g


def adam(p: dict, g: dict, state: dict, lr: float, step: int,
         b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """L5 one Adam step (in place; ``step`` counts from 1)."""
    for k in ("W1", "b1", "W2", "b2"):
        m = state.setdefault("m" + k, np.zeros_like(p[k], dtype=np.float64))
        v = state.setdefault("v" + k, np.zeros_like(p[k], dtype=np.float64))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** step)
        vh = v / (1 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def theta_targets(doc_ptr, z_docmajor, K: int, alpha: float) -> np.ndarray:
    """theta of Eq. 4 for training documents, from their assignments."""
    B = len(doc_ptr) - 1
    out = np.zeros((B, K))
    for d in range(B):
        zd = z_docmajor[int(doc_ptr[d]): int(doc_ptr[d + 1])]
        c = np.bincount(zd, minlength=K).astype(np.float64)
        out[d] = (c + alpha) / (len(zd) + K * alpha)
    return out
