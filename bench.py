"""Benchmark: tokens per second of one full WarpLDA MH sweep (document phase +
word phase) on a synthetic LDA corpus shaped like PubMed (D=8M, V=140K,
~736M tokens, K=10,000, M=2), with the HBM roofline of the dominant kernel and
of the whole sweep, the CPU oracle as the reported baseline, and the
end-to-end throughput through the C ABI from host buffers; then fold-in,
the learned document proposal and the serving loop on a model of the
NYTimes-shaped corpus (D=300K, V=100K, ~99M tokens, K=1,000), and on that
corpus the log-likelihood trajectories of M = 1, 2, 4 and of the paper's
storage-order word positioning (Fig. 7).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload pubmed|nytimes|clueweb|tiny]
                  [--foldin-workload nytimes|...] [--docs D] [--tuning key=value,...]
                  [--m-sweep | --no-m-sweep] [--foldin-docs N]
  python bench.py --impl reference ...   (the CPU oracle on the same workload)

One "step" is one sweep.  Prints one JSON line (rank 0).  With N > 1
(torchrun) every rank samples an independent replica of the workload on its
own GPU (the sampler has no cross-GPU exchange on this path); `value` is the
total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tokens/sec per MH sweep"
UNIT = "tokens/s"
FALLBACK_HBM_GBS = 6800.0

# algorithmic HBM bytes per token of each kernel class (int32 values):
# the document phase reads perm (4) and z + M proposals (4(M+1)) and writes
# them back (4(M+1)); the word phase reads and writes z + M proposals; the
# multi-pass tier splits the same traffic over its passes.
def alg_bytes_per_token(kind: str, M: int) -> float:
    return {
        "doc_batch": 4 + 8 * (M + 1),
        "doc_pipe": 4 + 8 * (M + 1),
        "word_cluster": 8 * (M + 1),
        "word_batch": 8 * (M + 1),
        "word_mega_hist": 4,
        "word_mega_accept": 4 * (M + 1) + 4,
        "word_mega_draw": 4 * M,
        "doc_huge_hist": 8,
        "doc_huge_accept": 4 + 4 * (M + 1) + 4,
        "doc_huge_draw": 4 + 4 * M,
    }.get(kind, 0.0)


def sweep_alg_bytes(M: int) -> int:
    return 20 + 16 * M


def measured_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources each kernel class is compiled from (its traffic record stays
# valid while these files are unchanged)
KERNEL_SOURCES = {
    "doc_batch": ["wl_batch.cu", "wl_common.cuh", "wl_block.cuh"],
    "doc_pipe": ["wl_docpipe.cu", "wl_common.cuh", "wl_block.cuh"],
    "word_cluster": ["wl_cluster.cu", "wl_common.cuh", "wl_block.cuh"],
    "word_batch": ["wl_batch.cu", "wl_common.cuh", "wl_block.cuh"],
    "word_mega_accept": ["wl_huge.cu", "wl_common.cuh", "wl_block.cuh"],
    "word_mega_draw": ["wl_huge.cu", "wl_common.cuh", "wl_block.cuh"],
    "word_mega_hist": ["wl_huge.cu", "wl_common.cuh", "wl_block.cuh"],
}


def kernel_fingerprint(kernel: str) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1510_08628_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, sorted(os.listdir(d))):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu capture of the kernel's
    current sources, or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except Exception:
        return None
    e = rec.get(workload, {}).get(kernel)
    if not e or e.get("sources") != kernel_fingerprint(kernel):
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_rate(c, wl, seed: int, sweeps: int, warm: int = 0):
    """Tokens/s of the CPU oracle over `sweeps` sweeps of corpus c."""
    import oracle
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, seed)
    if warm:
        o.sweep(warm)
    t = time.perf_counter()
    o.sweep(sweeps)
    dt = time.perf_counter() - t
    return c.N * sweeps / dt, oracle.num_threads(), dt


def sample_docs(name: str) -> int | None:
    return {"nytimes": 300_000, "pubmed": 600_000, "tiny": None}.get(name)


def heldout_split(rq):
    """Document completion: even in-document positions are folded in, odd ones
    are held out."""
    obs_len, ho_len, obs, ho = [], [], [], []
    for d in range(rq.D):
        w = rq.doc_word[rq.doc_ptr[d]: rq.doc_ptr[d + 1]]
        obs.append(w[0::2])
        ho.append(w[1::2])
        obs_len.append(len(w[0::2]))
        ho_len.append(len(w[1::2]))
    optr = np.concatenate([[0], np.cumsum(obs_len)]).astype(np.int64)
    hptr = np.concatenate([[0], np.cumsum(ho_len)]).astype(np.int64)
    return optr, np.concatenate(obs).astype(np.int32), hptr, np.concatenate(ho).astype(np.int32)


def heldout_ll(theta, hptr, hwords, cw, ck, beta, bbar):
    """Mean over held-out tokens of log sum_k theta_dk phi_wk, phi of Eq. 4."""
    denom = ck.astype(np.float64) + bbar
    tot, n = 0.0, 0
    for d in range(len(hptr) - 1):
        w = hwords[hptr[d]: hptr[d + 1]]
        if len(w) == 0:
            continue
        phi = (cw[w].astype(np.float64) + beta) / denom
        tot += float(np.log(phi @ theta[d].astype(np.float64)).sum())
        n += len(w)
    return tot / max(n, 1)


def theta_entropy(gpu, c, wl) -> float:
    """Mean entropy (nats) of the encoder's training targets -- theta of
    Eq. 4 from the context's current z, one per document: the floor of the
    encoder's cross-entropy loss (loss = entropy + KL)."""
    z, _ = gpu.counts(want_ck=False)
    D, K, a = c.D, wl.K, float(wl.alpha)
    L = np.diff(c.doc_ptr).astype(np.float64)
    doc = np.repeat(np.arange(D, dtype=np.int64), np.diff(c.doc_ptr))
    u, cnt = np.unique(doc * K + z, return_counts=True)
    ud = u // K
    den = L + K * a
    th = (cnt + a) / den[ud]
    H = np.zeros(D)
    np.add.at(H, ud, -th * np.log(th))
    th0 = a / den
    H += (K - np.bincount(ud, minlength=D)) * (-th0 * np.log(th0))
    return float(H[L > 0].mean())


def foldin_objective(z, optr, owords, cw, ck, K, alpha, beta, bbar) -> float:
    """Mean per token of log p(w, z | frozen model) of folded-in documents:
    the Dirichlet-multinomial term of each document's counts (alpha) plus
    log phi_hat[z, w] of Eq. 4 -- the target the fold-in chain samples
    (Eq. 5 with the word side frozen), which rises as the chain converges."""
    from scipy.special import gammaln
    L = np.diff(optr)
    D, N = len(L), int(optr[-1])
    doc = np.repeat(np.arange(D, dtype=np.int64), L)
    z = np.asarray(z[:N], dtype=np.int64)
    _, cnt = np.unique(doc * K + z, return_counts=True)
    a, abar = float(alpha), float(K) * float(alpha)
    td = float(np.sum(gammaln(abar) - gammaln(abar + L.astype(np.float64))))
    td += float(np.sum(gammaln(a + cnt) - gammaln(a)))
    w = np.asarray(owords[:N], dtype=np.int64)
    tw = float(np.sum(np.log((cw[w, z].astype(np.float64) + beta) / (ck[z].astype(np.float64) + bbar))))
    return (td + tw) / max(N, 1)


def signal_bounds(c, wl, name, corpus_seed, rq, doc_offset):
    """Held-out log-likelihood per token (odd positions of the requests) of
    two reference predictors: the unigram model of the training corpus, and
    the generator itself -- its true topic rows, with each document's topic
    mixture predicted by the Polya urn of its true even-position topics
    (the generator's own sequential law): the ceiling of any topic model."""
    from paper_1510_08628_gb300 import corpus
    wlw = corpus.WORKLOADS[name]
    out = {}
    wc = np.bincount(c.doc_word, minlength=c.V).astype(np.float64)
    pw = (wc + wl.beta) / (c.N + c.V * wl.beta)
    ho = np.concatenate([rq.doc_word[rq.doc_ptr[d] + 1: rq.doc_ptr[d + 1]: 2] for d in range(rq.D)])
    out["unigram"] = float(np.log(pw[ho]).mean())
    if wlw.K_true * wlw.V <= 50_000_000:
        tm = corpus.TopicModel(wlw.V, wlw.K_true, wlw.zipf_s, wlw.conc_c, corpus_seed, keep_phi=True)
        r2 = corpus.generate_docs(tm, np.diff(rq.doc_ptr), wlw.doc_alpha, corpus_seed, doc_offset,
                                  keep_z=True)
        phi = tm.phi.reshape(wlw.K_true, wlw.V)
        tot, n = 0.0, 0
        for d in range(rq.D):
            w = r2.doc_word[r2.doc_ptr[d]: r2.doc_ptr[d + 1]]
            tz = r2.true_z[r2.doc_ptr[d]: r2.doc_ptr[d + 1]]
            if len(w) < 2:
                continue
            post = (np.bincount(tz[0::2], minlength=wlw.K_true) + wlw.doc_alpha) / (
                len(tz[0::2]) + wlw.K_true * wlw.doc_alpha)
            tot += float(np.log(post @ phi[:, w[1::2]]).sum())
            n += len(w[1::2])
        out["true_model_ceiling"] = tot / max(n, 1)
    return out


def learned_curve(gpu, c, wl, name, seed, corpus_seed, n_req, sweeps):
    """Fold-in of the requests' even positions, plain vs learned proposal,
    after S sweeps: held-out log-likelihood of the odd positions (document
    completion) and the fold-in objective (the chain's target); for each,
    the sweeps each proposal needs to come within 0.5% of plain fold-in's
    value at the largest S."""
    from paper_1510_08628_gb300 import corpus
    off = c.D + 700_000
    rq = corpus.requests(name, seed=corpus_seed, n=n_req, doc_offset=off)
    optr, owords, hptr, hwords = heldout_split(rq)
    cw = gpu.word_counts()
    _, ck = gpu.counts(want_z=False)
    bbar = float(np.float32(c.V) * np.float32(wl.beta))
    curve = {"plain": {}, "learned": {}}
    obj = {"plain": {}, "learned": {}}
    for S in sweeps:
        for kind in ("plain", "learned"):
            th, z = gpu.foldin(optr, owords, sweeps=S, seed=seed + 29, z=True,
                               learned=(kind == "learned"))
            curve[kind][S] = heldout_ll(th, hptr, hwords, cw, ck, wl.beta, bbar)
            obj[kind][S] = foldin_objective(z, optr, owords, cw, ck, wl.K, wl.alpha, wl.beta, bbar)

    def need(cv):
        target = cv["plain"][sweeps[-1]]
        tol = 0.005 * abs(target)
        return {k: next((S for S in sweeps if cv[k][S] >= target - tol), None) for k in cv}

    return {"docs": rq.D, "split": "even positions folded in, odd held out",
            "ll_per_token": {k: {str(S): v for S, v in curve[k].items()} for k in curve},
            "target": "plain fold-in after %d sweeps, within 0.5%%" % sweeps[-1],
            "sweeps_to_target": need(curve),
            "objective_per_token": {k: {str(S): v for S, v in obj[k].items()} for k in obj},
            "sweeps_to_target_objective": need(obj),
            "signal": signal_bounds(c, wl, name, corpus_seed, rq, off)}


def learned_bench(gpu, c, wl, args):
    """The learned document proposal for fold-in: encoder training on the
    corpus's own (document, theta) pairs (loss beside its entropy floor),
    then held-out log-likelihood and the fold-in objective after S fold-in
    sweeps, plain vs learned, serving at equal load with the sweeps each
    needs, and fold-in throughput; the same on the tiny workload (16
    strongly separated topics)."""
    from paper_1510_08628_gb300 import corpus
    from paper_1510_08628_gb300.warplda import WarpLDA
    floor = theta_entropy(gpu, c, wl)
    gpu.encoder_init(log2_features=16, hidden=512, batch_rows=256, seed=args.seed)
    t = time.perf_counter()
    losses = gpu.encoder_train(epochs=args.encoder_epochs, lr=args.encoder_lr, seed=args.seed)
    train_s = time.perf_counter() - t
    heldout = learned_curve(gpu, c, wl, args.workload, args.seed, args.corpus_seed, 1000,
                            [1, 2, 3, 4, 6, 8, 12, 16, 24, 30])
    need = heldout["sweeps_to_target_objective"]
    # the offered load of the main serving comparison (half the plain
    # fold-in's throughput, capped)
    rate = min(0.5 * getattr(args, "_plain_docs_per_s", 200_000.0), 100_000.0)
    heldout["serving_at_objective_target"] = [
        serving_bench(gpu, c, wl, args, kind == "learned", rate, sweeps=need[kind] or args.foldin_sweeps)
        for kind in ("plain", "learned")]
    ct, wt = corpus.generate("tiny", seed=1)
    gt = WarpLDA(ct.doc_ptr, ct.doc_word, ct.V, wt.K, wt.alpha, wt.beta, 2, 7)
    gt.sweep(200)
    gt.encoder_init(log2_features=12, hidden=128, batch_rows=256, seed=3)
    tl = gt.encoder_train(epochs=60, lr=3e-3, seed=4)
    tiny = learned_curve(gt, ct, wt, "tiny", 71, 1, 500, [1, 2, 3, 4, 8, 16])
    tiny["encoder_loss"] = [float(tl[0]), float(tl[-1])]
    tiny["model"] = "tiny workload (D=1000, K=16, M=2), 200 sweeps; encoder 2^12 features, 128 hidden, 60 epochs"
    # serving at equal load, each proposal with the sweeps it needs to reach
    # the held-out target
    need = tiny["sweeps_to_target"]
    tiny["serving_at_target"] = [
        serving_bench(gt, ct, wt, args, kind == "learned", 20_000.0, n=4000, name="tiny",
                      sweeps=need[kind] or 16) for kind in ("plain", "learned")]
    gt.close()

    # throughput of the learned fold-in (encoder forward + alias tables + sweeps)
    big = corpus.requests(args.workload, seed=args.corpus_seed, n=args.foldin_docs,
                          doc_offset=c.D + 1000)
    t = time.perf_counter()
    gpu.foldin(big.doc_ptr, big.doc_word, sweeps=args.foldin_sweeps, seed=args.seed + 17, z=False,
               learned=True)
    wall = time.perf_counter() - t
    return {"encoder": {"features": 1 << 16, "hidden": 512, "K": wl.K, "epochs": args.encoder_epochs,
                        "lr": args.encoder_lr, "train_seconds": train_s,
                        "epoch_loss": [float(x) for x in losses],
                        "theta_target_entropy": floor,
                        "pairs": "the corpus's own documents with theta of Eq. 4 of the current z"},
            "heldout": heldout, "heldout_tiny": tiny,
            "docs_per_s": big.D / wall, "docs": big.D, "sweeps": args.foldin_sweeps,
            "includes": "encoder forward + alias tables + fold-in kernel + H2D/D2H (C ABI call)"}


def serving_bench(gpu, c, wl, args, learned: bool, rate: float, n: int = 6000, name=None, sweeps=None):
    """Fold-in requests arriving as a Poisson stream at `rate` docs/s, served
    with continuous batching (warplda_server_*): each step advances every
    admitted request by one sweep; requests arriving meanwhile join the next
    step.  Latency = completion (poll) time - arrival time."""
    from paper_1510_08628_gb300 import corpus
    from paper_1510_08628_gb300.warplda import Server
    rq = corpus.requests(name or args.workload, seed=args.corpus_seed, n=n, doc_offset=c.D + 2_000_000)
    rng = np.random.default_rng(args.seed)
    arrive = np.cumsum(rng.exponential(1.0 / rate, size=n))
    S = sweeps or args.foldin_sweeps
    srv = Server(gpu, slots=8192, pool_tokens=4_000_000, max_doc_tokens=5000, sweeps=S,
                 seed=args.seed + 41, learned=learned)
    lat = np.zeros(n)
    got, nxt, queue, steps = 0, 0, [], 0
    gpu.profile(True)   # per-launch CUDA events by class, both streams
    t0 = time.perf_counter()
    while got < n:
        now = time.perf_counter() - t0
        while nxt < n and arrive[nxt] <= now:
            queue.append(nxt)
            nxt += 1
        while queue:
            d = queue[0]
            if not srv.submit(d, rq.doc_word[rq.doc_ptr[d]: rq.doc_ptr[d + 1]]):
                break
            queue.pop(0)
        active = srv.step()
        steps += 1
        ids, _ = srv.poll()
        t = time.perf_counter() - t0
        for i in ids:
            lat[int(i)] = t - arrive[int(i)]
        got += len(ids)
        if active == 0 and not queue and nxt < n:
            time.sleep(max(0.0, min(0.001, arrive[nxt] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    kt = gpu.kernel_times()
    gpu.profile(False)
    srv.close()
    # device time per step of each kind of launch (the new requests' work is
    # on a second stream, beside the running requests' sweep)
    per_step = {k: round(ms / max(steps, 1), 4) for k, (_, ms) in kt.items() if k.startswith("serve")}
    return {"proposal": "learned" if learned else "plain", "offered_docs_per_s": rate, "docs": n,
            "sweeps": S, "docs_per_s": n / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "steps": steps,
            "device_ms_per_step": per_step}


TUNING_KEYS = ("batch_max_tokens", "huge_chunk", "region_budget", "doc_warp_max", "word_positioning",
               "doc_batch_kernel", "cluster_max_tokens", "foldin_kernel")


def parse_tuning(text: str) -> dict | None:
    """`key=value,key=value` -> the sampler's tuning fields (None: defaults)."""
    out = {}
    for item in filter(None, (x.strip() for x in text.split(","))):
        k, _, v = item.partition("=")
        if k not in TUNING_KEYS or not v:
            raise SystemExit(f"bad --tuning item {item!r}; keys: {', '.join(TUNING_KEYS)}")
        out[k] = int(v)
    return out or None


def m_sweep(c, wl, args, stream, iters: int = 100, every: int = 10):
    """Joint log-likelihood (Sec. 6.1) against iterations for M = 1, 2, 4 on
    the same corpus and seed (the paper's Fig. 7 comparison), and for M = 2
    with the paper's literal storage-order word positioning against the
    order-statistic rule; with the device time per sweep of each."""
    import torch
    from paper_1510_08628_gb300.warplda import WarpLDA
    out = {}
    for label, M, tun in (("M=1", 1, None), ("M=2", 2, None), ("M=4", 4, None),
                          ("M=2 storage-order word positioning", 2, {"word_positioning": 1})):
        g = WarpLDA(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, M, args.seed, stream=stream,
                    tuning=tun)
        pts = [(0, g.loglik())]
        ms = 0.0
        for it in range(every, iters + 1, every):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.sweep(every)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            pts.append((it, g.loglik()))
        g.close()
        out[label] = {"loglik": pts, "ms_per_sweep": ms / iters}
    return {"iterations": iters, "runs": out}


def foldin_bench(gpu, c, wl, args, torch, stream):
    """Fold-in of unseen documents of the workload's generator (lengths
    clipped to [20, 5000]) against the trained model: docs/s end to end
    through warplda_foldin (host CSR in, theta out), and the CPU oracle on a
    sample of the same requests."""
    from paper_1510_08628_gb300 import corpus
    rq = corpus.requests(args.workload, seed=args.corpus_seed, n=args.foldin_docs,
                         doc_offset=c.D + 1000)
    S = args.foldin_sweeps
    small = int(rq.doc_ptr[min(64, rq.D)])
    gpu.foldin(rq.doc_ptr[: min(64, rq.D) + 1], rq.doc_word[:small], sweeps=2, seed=1)  # model build
    # the request CSR and theta in pinned host memory, as a server would hold them
    dp = torch.from_numpy(rq.doc_ptr).pin_memory().numpy()
    dw = torch.from_numpy(rq.doc_word).pin_memory().numpy()
    th_buf = torch.empty((rq.D, wl.K), dtype=torch.float32, pin_memory=True).numpy()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start.record(stream)
    th, _ = gpu.foldin(dp, dw, sweeps=S, seed=args.seed + 17, z=False, theta_out=th_buf)
    stop.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_s = start.elapsed_time(stop) / 1000.0
    kt = gpu.kernel_times()
    gpu.profile(False)
    # algorithmic bytes per token and sweep of the word-major phases: the
    # document phase reads and writes z and the proposals (4 + 4M each way),
    # the word phase streams a 16-byte record and reads and writes the same
    alg = {"foldin_doc": 2 * (4 + 4 * wl.M), "foldin_word": 16 + 2 * (4 + 4 * wl.M)}
    kernels = {}
    for name, (n, ms) in kt.items():
        e = {"launches": n, "total_ms": ms}
        if name in alg and n > 0:
            e["alg_bytes_per_token"] = alg[name]
            e["gbs"] = alg[name] * rq.N * min(n, S) / (ms / 1e3) / 1e9
        kernels[name] = e
    out = {"docs": rq.D, "tokens": rq.N, "sweeps": S, "K": wl.K, "M": wl.M,
           "docs_per_s": rq.D / wall, "tokens_sweeps_per_s": rq.N * S / wall, "seconds": wall,
           "device_seconds": dev_s, "includes": "host checks + H2D of the CSR + fold-in kernels + "
                                                 "D2H of theta into pinned memory (synchronous C ABI call)",
           "kernels": kernels,
           "proposal": "plain", "lengths": "lognormal of the workload, clipped to [20, 5000]",
           "kernel": ("one warp per document, all sweeps in one launch"
                      if (getattr(args, "_tuning", None) or {}).get("foldin_kernel") == 1 else
                      "word-major phases (document phase per document, word phase per word)")}
    if not args.no_cpu_baseline:
        import oracle
        n = min(400, rq.D)
        e = int(rq.doc_ptr[n])
        z, ck = gpu.counts()
        wp, perm = gpu.token_order()
        zw = np.empty_like(z)
        zw[perm] = z
        cw = oracle.word_topic_counts(zw, wp, c.V, wl.K)
        t = time.perf_counter()
        oracle.foldin(rq.doc_ptr[: n + 1], rq.doc_word[:e], cw, ck, wl.K, wl.M, wl.alpha, wl.beta,
                      c.V, seed=args.seed + 17, sweeps=S)
        dt = time.perf_counter() - t
        out["cpu_baseline"] = {"docs_per_s": n / dt, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": f"first {n} requests ({e} tokens), "
                                                           f"{S} sweeps ({dt:.1f} s)"}
    return out


def run_reference(args, ws, rank):
    from paper_1510_08628_gb300 import corpus
    if rank != 0:
        return
    nd = sample_docs(args.workload)
    c, wl = corpus.generate(args.workload, seed=args.corpus_seed, D=nd)
    import oracle
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, args.seed)
    o.sweep(args.warmup)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        o.sweep(1)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = c.N * args.steps / total
    sample = (f"first {c.D} documents ({c.N} tokens) of the {args.workload} corpus, "
              f"full sweeps" if nd else f"{args.workload} corpus, full sweeps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "K": wl.K, "M": wl.M, "N": c.N, "D": c.D,
                   "V": c.V, "sampler": "CPU oracle (plain C, OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="pubmed", help="pubmed | nytimes | clueweb | tiny")
    ap.add_argument("--foldin-workload", default="nytimes",
                    help="corpus whose trained model the fold-in, learned-proposal and serving "
                         "measurements use")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--corpus-seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--foldin-docs", type=int, default=20000,
                    help="fold-in requests timed after the sweeps (0: none)")
    ap.add_argument("--foldin-sweeps", type=int, default=30)
    ap.add_argument("--model-sweeps", type=int, default=100,
                    help="sweeps the model has when the fold-in measurements start")
    ap.add_argument("--encoder-epochs", type=int, default=16,
                    help="epochs of encoder training for the learned fold-in proposal (0: skip)")
    ap.add_argument("--encoder-lr", type=float, default=3e-3, help="Adam step size of encoder training")
    ap.add_argument("--m-sweep", action="store_true",
                    help="record log-likelihood against iterations for M = 1, 2, 4 (Fig. 7) on the timed "
                         "workload (by default it is recorded on the fold-in workload's corpus)")
    ap.add_argument("--no-m-sweep", action="store_true", help="skip the M comparison")
    ap.add_argument("--tuning", default="",
                    help="launch tuning of the sampler as key=value pairs separated by commas "
                         "(batch_max_tokens, huge_chunk, region_budget, doc_warp_max, word_positioning, "
                         "doc_batch_kernel, cluster_max_tokens, foldin_kernel)")
    ap.add_argument("--docs", type=int, default=0,
                    help="use only the first DOCS documents of the workload (small profiling cases)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            import torch
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch

    from paper_1510_08628_gb300 import corpus
    from paper_1510_08628_gb300.warplda import WarpLDA

    assert torch.cuda.is_available(), "the native arm needs a GPU"
    torch.cuda.set_device(local)

    # CPU baseline first (before any GPU work): the oracle on a bounded sample
    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        nd = sample_docs(args.workload)
        cs, wls = corpus.generate(args.workload, seed=args.corpus_seed, D=nd)
        rate, cores, dt = oracle_rate(cs, wls, args.seed, sweeps=4)
        cpu_base = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": f"4 full sweeps of the first {cs.D} documents ({cs.N} tokens) of "
                              f"the {args.workload} corpus ({dt:.1f} s)"}
        del cs

    c, wl = corpus.generate(args.workload, seed=args.corpus_seed, D=args.docs or None)
    seed = args.seed + 1000 * rank
    stream = torch.cuda.current_stream()
    tun = parse_tuning(args.tuning)
    args._tuning = tun
    gpu = WarpLDA(c.doc_ptr, c.doc_word, c.V, wl.K, wl.alpha, wl.beta, wl.M, seed, stream=stream,
                  tuning=tun)
    info = gpu.info()
    gpu.sweep(args.warmup)
    torch.cuda.synchronize()
    gpu.sync()   # raises if a kernel's index check failed

    # timed region: K sweeps on the library's stream
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        start.record(stream)
        gpu.sweep(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    gpu.sync()
    ms = start.elapsed_time(stop)
    ms_max = reduce_max(ms, ws)
    value = c.N * args.steps * ws / (ms_max / 1000.0)

    # per-kernel CUDA-event timing (a second timed pass, events on the same stream)
    gpu.profile(True)
    gpu.sweep(args.steps)
    kt = gpu.kernel_times()
    gpu.profile(False)
    peak, peak_kind = measured_peaks()
    tier_tokens = {
        "doc_batch": c.N - info["huge_doc_tokens"] - info["pipe_doc_tokens"],
        "doc_pipe": info["pipe_doc_tokens"],
        "word_batch": c.N - info["mega_word_tokens"] - info["cluster_word_tokens"],
        "word_cluster": info["cluster_word_tokens"],
        "word_mega_hist": info["mega_word_tokens"], "word_mega_accept": info["mega_word_tokens"],
        "word_mega_draw": info["mega_word_tokens"], "doc_huge_hist": info["huge_doc_tokens"],
        "doc_huge_accept": info["huge_doc_tokens"], "doc_huge_draw": info["huge_doc_tokens"],
    }
    # a kernel class may launch more than once per sweep (the block batches
    # of two sizes): its algorithmic bytes per sweep are spread over them
    kernels = {}
    for k, (n, tot) in kt.items():
        avg = tot / n
        per_sweep = n / args.steps
        alg = alg_bytes_per_token(k, wl.M) * tier_tokens.get(k, 0) / per_sweep
        kernels[k] = {"launches": n, "avg_ms": avg, "share": None,
                      "alg_bytes": alg, "gbs": (alg / (avg / 1000) / 1e9) if alg else None}
    total_k = sum(v["avg_ms"] * v["launches"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = v["avg_ms"] * v["launches"] / total_k if total_k else None
    dom = max((k for k in kernels if kernels[k]["alg_bytes"]), key=lambda k: kernels[k]["avg_ms"] *
              kernels[k]["launches"])
    d = kernels[dom]
    sweep_s = ms / 1000.0 / args.steps
    sweep_gbs = sweep_alg_bytes(wl.M) * c.N / sweep_s / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": d["gbs"], "peak": peak, "unit": "GB/s",
            "frac": d["gbs"] / peak, "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": recorded_traffic(dom, args.workload),
            "alg_bytes_per_launch": d["alg_bytes"]}

    gpu.close()
    msweep = None
    if args.m_sweep and not args.no_m_sweep and rank == 0:
        msweep = m_sweep(c, wl, args, stream)
        msweep["workload"] = args.workload

    # end to end through the C ABI from pinned host buffers: init (H2D of the
    # corpus, token-order build) + K sweeps + D2H of z and c_k
    e2e = None
    if not args.no_e2e:
        dp = torch.from_numpy(c.doc_ptr).pin_memory().numpy()
        dw = torch.from_numpy(c.doc_word).pin_memory().numpy()
        # the step's result lands in pinned host buffers held by the caller
        zout = torch.empty(max(c.N, 1), dtype=torch.int32, pin_memory=True).numpy()
        ckout = torch.empty(wl.K, dtype=torch.int32, pin_memory=True).numpy()
        # warm-up: the same calls once, untimed, on the same pinned buffers
        # (the first copies through freshly pinned pages run several times
        # slower while the pages are mapped for the device)
        gw = WarpLDA(dp, dw, c.V, wl.K, wl.alpha, wl.beta, wl.M, seed, stream=stream, tuning=tun)
        gw.sweep(1)
        gw.counts(z_out=zout, ck_out=ckout)
        gw.close()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        g2 = WarpLDA(dp, dw, c.V, wl.K, wl.alpha, wl.beta, wl.M, seed, stream=stream, tuning=tun)
        g2.sweep(args.steps)
        z, ck = g2.counts(z_out=zout, ck_out=ckout)
        t1 = time.perf_counter()
        g2.close()
        e2e_s = reduce_max(t1 - t0, ws)
        e2e = {"value": c.N * args.steps * ws / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int((dp.nbytes + dw.nbytes) / args.steps),
               "d2h_bytes_per_step": int((z.nbytes + ck.nbytes) / args.steps),
               "seconds": e2e_s, "includes": "init (H2D of the corpus, device token-order build) + sweeps + "
                                             "D2H of z and c_k into pinned host buffers",
               "warmup": "the same calls once, untimed, on the same pinned buffers"}

    # fold-in, the learned proposal and serving: a model of the fold-in
    # workload, trained first (its own context; the sweep's is closed)
    foldin = None
    if args.foldin_docs > 0 and rank == 0:
        import copy
        fa = copy.copy(args)
        fa.workload = args.foldin_workload
        if fa.workload == args.workload:
            cf, wf = c, wl
        else:
            cf, wf = corpus.generate(fa.workload, seed=args.corpus_seed)
        model = WarpLDA(cf.doc_ptr, cf.doc_word, cf.V, wf.K, wf.alpha, wf.beta, wf.M, seed, stream=stream,
                        tuning=tun)
        model.sweep(args.model_sweeps)   # train the model
        foldin = foldin_bench(model, cf, wf, fa, torch, stream)
        fa._plain_docs_per_s = foldin["docs_per_s"]
        foldin["workload"] = fa.workload
        foldin["model_sweeps"] = args.model_sweeps
        if args.encoder_epochs > 0:
            foldin["learned"] = learned_bench(model, cf, wf, fa)
        # serving at equal load for both proposals: half the plain fold-in's
        # measured throughput, capped
        rate = min(0.5 * foldin["docs_per_s"], 100_000.0)
        foldin["serving"] = [serving_bench(model, cf, wf, fa, False, rate)]
        if args.encoder_epochs > 0:
            foldin["serving"].append(serving_bench(model, cf, wf, fa, True, rate))
        model.close()
        if msweep is None and not args.no_m_sweep:
            # the M comparison (Fig. 7) on the fold-in workload's corpus
            msweep = m_sweep(cf, wf, args, stream)
            msweep["workload"] = fa.workload

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "D": c.D, "V": c.V, "N": c.N, "K": wl.K,
                       "M": wl.M, "alpha": wl.alpha, "beta": wl.beta,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": f"inputs larger than L2 (state {info['device_bytes'] / 1e9:.2f} GB)",
                       "accept_arith": "FP32 RN, no FMA", "tuning": tun or "defaults"},
            "roofline": roof,
            "sweep_roofline": {"alg_bytes_per_token": sweep_alg_bytes(wl.M), "achieved": sweep_gbs,
                               "peak": peak, "unit": "GB/s", "frac": sweep_gbs / peak},
            "kernels": kernels,
            "cpu_baseline": cpu_base,
            "e2e": e2e,
            "gpu_launches": info["launches_per_sweep"] * args.steps,
            "foldin": foldin,
            "m_sweep": msweep,
            "clocks": clk.summary(),
            "paper_context": {"value": 110e6, "unit": UNIT,
                              "hardware": "2x Xeon E5-2692v2 (24 cores), NYTimes/PubMed, M=2"},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
