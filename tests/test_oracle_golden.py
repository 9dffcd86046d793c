"""The oracle reproduces its stored trajectories (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): a guard against unintended
change of the oracle's arithmetic."""
import json
import os

import pytest

from tests.golden import make_golden

with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_trajectories.json")) as f:
    GOLDEN = json.load(f)


@pytest.mark.parametrize("case", make_golden.CASES, ids=[c[0] for c in make_golden.CASES])
def test_oracle_matches_stored_trajectory(case):
    want = GOLDEN["cases"][case[0]]
    got = make_golden.run_case(*case)
    assert got["N"] == want["N"]
    for cp, w in want["checkpoints"].items():
        g = got["checkpoints"][cp]
        for key in ("z_sha256", "prop_sha256", "ck_sha256"):
            assert g[key] == w[key], (case[0], cp, key)
        assert abs(g["loglik"] - w["loglik"]) <= 1e-12 * abs(w["loglik"])
