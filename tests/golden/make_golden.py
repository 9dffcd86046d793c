"""Writes oracle_trajectories.json: oracle-only regression values.

Run from the repository root:  python tests/golden/make_golden.py
Calls only oracle/ (and the seeded corpus generator for its inputs).  The
stored hashes pin the oracle against unintended change; any intended change
to the oracle's arithmetic regenerates this file and names, in its commit
message, the paper passage or reading that justifies it.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1510_08628_gb300 import corpus  # noqa: E402

CASES = [
    # name, workload, corpus seed, D, K, M, sampler seed, checkpoints
    ("tiny_M1", "tiny", 1, None, 16, 1, 7, [1, 5, 20]),
    ("tiny_K5_M2", "tiny", 2, 200, 5, 2, 9, [1, 3, 10]),
    ("tiny_K40_M3", "tiny", 3, 150, 40, 3, 11, [1, 4]),
]


def run_case(name, wl_name, cseed, D, K, M, seed, checkpoints):
    c, wl = corpus.generate(wl_name, seed=cseed, D=D)
    o = oracle.Oracle(c.doc_ptr, c.doc_word, c.V, K, wl.alpha, wl.beta, M, seed=seed)
    rec = {"N": o.N, "checkpoints": {}}
    done = 0
    for cp in checkpoints:
        o.sweep(cp - done)
        done = cp
        rec["checkpoints"][str(cp)] = {
            "z_sha256": hashlib.sha256(o.z_docmajor().tobytes()).hexdigest(),
            "prop_sha256": hashlib.sha256(o.prop.tobytes()).hexdigest(),
            "ck_sha256": hashlib.sha256(o.ck.tobytes()).hexdigest(),
            "loglik": o.loglik(),
        }
    return rec


def main():
    out = {"note": "oracle-only values; see make_golden.py", "cases": {}}
    for case in CASES:
        out["cases"][case[0]] = {"args": list(case[1:]), **run_case(*case)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_trajectories.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
