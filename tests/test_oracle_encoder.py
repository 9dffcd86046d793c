"""Pins of the encoder oracle (oracle/encoder.py, FP64 NumPy).

* Back-propagation (L4) against central finite differences of the loss in
  plain FP64, every parameter block.
* Uniform logits give loss = log K exactly; the bias gradient sums to zero.
* One Adam step from zero moments moves each weight by lr * g / (|g| + eps)
  (the first step of Kingma & Ba's Alg. 1 in closed form).
* bf16 rounding equals torch's float32 -> bfloat16 conversion.
* The feature hash stays in [0, F) and has its closed-form value on w = 1.
"""
import numpy as np
import pytest

from oracle import encoder as enc


def _problem(seed=0, F_log2=6, H=8, K=5, B=4):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, 0.5, size=(1 << F_log2, H)), "b1": rng.normal(0, 0.1, size=H),
         "W2": rng.normal(0, 0.5, size=(H, K)), "b2": rng.normal(0, 0.1, size=K)}
    lens = rng.integers(3, 12, size=B)
    dp = np.concatenate([[0], np.cumsum(lens)])
    dw = rng.integers(0, 1000, size=int(dp[-1]))
    x = enc.inputs(dp, dw, F_log2)
    theta = rng.dirichlet(np.ones(K), size=B)
    return p, x, theta


def test_backprop_matches_finite_differences():
    p, x, theta = _problem()
    _, g = enc.backward(p, x, theta, bf=False)
    eps = 1e-6
    for k in ("W1", "b1", "W2", "b2"):
        flat = p[k].reshape(-1)
        idx = range(flat.size) if flat.size <= 64 else np.flatnonzero(x.sum(0) > 0)[:4] * p[k].shape[1]
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp = enc.loss(enc.forward(p, x, bf=False)["q"], theta)
            flat[i] = old - eps
            lm = enc.loss(enc.forward(p, x, bf=False)["q"], theta)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k].reshape(-1)[i]) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, g[k].reshape(-1)[i])


def test_uniform_logits():
    p, x, theta = _problem(1)
    p["W2"][:] = 0
    p["b2"][:] = 0
    l, g = enc.backward(p, x, theta, bf=False)
    assert abs(l - np.log(5)) < 1e-12
    assert abs(g["b2"].sum()) < 1e-12


def test_adam_first_step_closed_form():
    p, x, theta = _problem(2)
    _, g = enc.backward(p, x, theta, bf=False)
    before = {k: v.copy() for k, v in p.items()}
    enc.adam(p, g, {}, lr=1e-3, step=1)
    for k in p:
        want = before[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        np.testing.assert_allclose(p[k], want, rtol=1e-9, atol=1e-15)


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(size=4000).astype(np.float32),
                        np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-9, -2.5, 0.0, 65504.0], np.float32)])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(enc.bf16(a), want)


def test_feature_hash():
    f = enc.feature(np.arange(100000), 16)
    assert f.min() >= 0 and f.max() < (1 << 16)
    assert int(enc.feature(np.array([1]), 16)[0]) == 2654435761 >> 16
