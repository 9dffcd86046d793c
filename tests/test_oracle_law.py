"""Distribution pins of the oracle's document and word phases.

Each test builds S identical copies of a tiny segment (a document, or a word),
puts them through ONE oracle phase -- every copy draws from its own Philox
blocks because the stream is keyed by token -- and compares the empirical
joint law of the outcome with the exact law written out here in float64 from
the paper:

* the MH step of Alg. 1 with the Eq. 7 acceptance rates (pi^word in the
  document phase, pi^doc in the word phase), counts frozen at the phase start
  (delayed update, Sec. 4.2), chained over the M proposals;
* the Eq. 6 proposals as the mixture of Sec. 2.2 with weight L / (L + G)
  (G = alpha_bar for documents, K beta for words), the p_A branch a uniform
  position of the post-acceptance assignments (Sec. 4.3 random positioning).

A dropped term, swapped operand, wrong count, wrong source state or wrong
mixture weight in the oracle moves one of these laws (see
test_oracle_mutations.py).  The chain test pins Eq. 5 as the stationary law.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle

S = 200_000
P_MIN = 1e-4          # per-test threshold; each test runs a handful of comparisons


def _step_law(s, props, C, g, ck, gbar):
    """Exact law of the final state of M chained MH steps (Alg. 1, Eq. 7)."""
    dist = {s: 1.0}
    for t in props:
        nd = {}
        for cur, p in dist.items():
            if t == cur:
                nd[cur] = nd.get(cur, 0.0) + p
                continue
            a = min(1.0, (C[t] + g) * (ck[cur] + gbar) / ((C[cur] + g) * (ck[t] + gbar)))
            nd[t] = nd.get(t, 0.0) + p * a
            nd[cur] = nd.get(cur, 0.0) + p * (1 - a)
        dist = nd
    return dist


def _prop_law(zpost, K, G):
    """Exact Eq. 6 mixture: L/(L+G) * count/L + G/(L+G) / K."""
    L = len(zpost)
    cnt = np.bincount(zpost, minlength=K)
    return L / (L + G) * cnt / L + G / (L + G) / K


def _check_joint(obs_z, obs_p, z0, props, C, g, ck, gbar, K, G, M, tag):
    L = len(z0)
    laws = [_step_law(z0[j], props[j], C, g, ck, gbar) for j in range(L)]
    configs = list(itertools.product(range(K), repeat=L))
    pz = np.array([np.prod([laws[j].get(c[j], 0.0) for j in range(L)]) for c in configs])
    code = np.zeros(len(obs_z), dtype=np.int64)
    for j in range(L):
        code = code * K + obs_z[:, j]
    # joint law of the post-acceptance assignments
    cnt = np.bincount(code, minlength=len(configs))
    keep = pz > 0
    assert cnt[~keep].sum() == 0, f"{tag}: impossible z' configuration observed"
    r = stats.chisquare(cnt[keep], pz[keep] / pz[keep].sum() * cnt.sum())
    assert r.pvalue > P_MIN, f"{tag}: z' law p={r.pvalue}"
    # joint law of (z', p_ji) for every token j and step i
    for j in range(L):
        for i in range(M):
            exp = np.zeros((len(configs), K))
            for ci, c in enumerate(configs):
                exp[ci] = pz[ci] * _prop_law(np.array(c), K, G)
            obs = np.bincount(code * K + obs_p[:, j, i], minlength=len(configs) * K)
            e = exp.ravel()
            keep = e > 0
            assert obs[~keep].sum() == 0
            r = stats.chisquare(obs[keep], e[keep] / e[keep].sum() * obs.sum())
            assert r.pvalue > P_MIN, f"{tag}: proposal law token {j} step {i} p={r.pvalue}"


def run_doc_law(M, mutation=0, seed=3):
    K = 3
    words = np.array([0, 1, 0], dtype=np.int32)
    z0 = np.array([0, 2, 2])
    props = np.array([[1, 2], [0, 1], [1, 0]])[:, :M]
    ck = np.array([5, 3, 7], dtype=np.int32)
    alpha, abar, bbar = 0.5, 1.5, 2.0
    L = len(words)
    doc_ptr = np.arange(0, L * S + 1, L, dtype=np.int64)
    doc_word = np.tile(words, S)
    lib = oracle.load(mutation)
    word_ptr = np.zeros(3, dtype=np.int64)
    perm = np.zeros(L * S, dtype=np.int32)
    assert lib.orc_word_major(S, 2, doc_ptr, doc_word, word_ptr, perm) == 0
    z = np.zeros(L * S, dtype=np.int32)
    prop = np.zeros(L * S * M, dtype=np.int32)
    pr = perm.reshape(S, L)
    z[pr] = z0[None, :]
    for i in range(M):
        prop[pr * M + i] = props[None, :, i]
    lib.orc_doc_phase(0, S, doc_ptr, perm, K, M, oracle.f32(alpha), oracle.f32(abar),
                      oracle.f32(bbar), seed, 1, z, prop, ck)
    obs_z = z[pr]
    obs_p = np.stack([prop[pr * M + i] for i in range(M)], axis=2)
    cd = np.bincount(z0, minlength=K)
    return obs_z, obs_p, dict(z0=z0, props=props, C=cd, g=alpha, ck=ck, gbar=bbar, K=K,
                              G=abar, M=M)


def run_word_law(M, mutation=0, seed=4, rule=0):
    K = 3
    z0 = np.array([0, 2, 2])
    props = np.array([[1, 0], [0, 1], [1, 2]])[:, :M]
    ck = np.array([4, 6, 9], dtype=np.int32)
    beta, kbeta, bbar = 0.25, 0.75, 1.25
    L = 3
    word_ptr = np.arange(0, L * S + 1, L, dtype=np.int64)
    z = np.tile(z0, S).astype(np.int32)
    prop = np.tile(props, (S, 1)).astype(np.int32).ravel()
    lib = oracle.load(mutation)
    lib.orc_word_phase_rule(0, S, word_ptr, K, M, oracle.f32(beta), oracle.f32(kbeta),
                            oracle.f32(bbar), seed, 1, z, prop, ck, rule)
    obs_z = z.reshape(S, L)
    obs_p = prop.reshape(S, L, M)
    cw = np.bincount(z0, minlength=K)
    return obs_z, obs_p, dict(z0=z0, props=props, C=cw, g=beta, ck=ck, gbar=bbar, K=K,
                              G=kbeta, M=M)


@pytest.mark.parametrize("M", [1, 2])
def test_doc_phase_law(M):
    obs_z, obs_p, ex = run_doc_law(M)
    _check_joint(obs_z, obs_p, tag="doc", **ex)


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("rule", [0, 1])
def test_word_phase_law(M, rule):
    # rule 1: the paper's literal positioning over the word's tokens in
    # storage order -- the same law as the order-statistic rule (R7')
    obs_z, obs_p, ex = run_word_law(M, rule=rule)
    _check_joint(obs_z, obs_p, tag="word", **ex)


def eq5_target(Cd, Cw, ck, alpha, beta, bbar):
    p = (Cd + alpha) * (Cw + beta) / (ck + bbar)
    return p / p.sum()


def run_chains(K, M, mutation=0, seed=11, n_chains=300_000, n_sweeps=4, start="stationary"):
    rng = np.random.default_rng(seed + 100 * K + M)
    Ld, Lw = 9, 14
    zd = rng.integers(0, K, size=Ld).astype(np.int32)
    zw = np.sort(rng.integers(0, K, size=Lw)).astype(np.int32)
    Cd = np.bincount(zd, minlength=K).astype(np.int32)
    Cw = np.bincount(zw, minlength=K).astype(np.int32)
    ck = (Cd + Cw + rng.integers(0, 30, size=K)).astype(np.int32)
    alpha, beta, V = 0.4, 0.3, 5
    abar, bbar, kbeta = oracle.derived(K, V, alpha, beta)
    target = eq5_target(Cd, Cw, ck, np.float32(alpha), np.float32(beta), bbar)
    if start == "stationary":
        s0 = rng.choice(K, size=n_chains, p=target).astype(np.int32)
    else:
        s0 = np.zeros(n_chains, dtype=np.int32)
    out = np.zeros(n_chains, dtype=np.int32)
    lib = oracle.load(mutation)
    lib.orc_token_chains(K, M, Cd, Cw, ck, zd, Ld, zw, Lw, oracle.f32(alpha), oracle.f32(beta),
                         abar, bbar, kbeta, seed, 1000, n_chains, n_sweeps, s0, out)
    return out, target


@pytest.mark.parametrize("K,M", [(2, 1), (2, 2), (16, 1), (16, 2)])
@pytest.mark.parametrize("start", ["stationary", "zero"])
def test_chain_converges_to_eq5(K, M, start):
    out, target = run_chains(K, M, n_sweeps=4 if start == "stationary" else 40, start=start)
    obs = np.bincount(out, minlength=K)
    r = stats.chisquare(obs, target * len(out))
    assert r.pvalue > 1e-3 / 16, (K, M, start, r.pvalue)
