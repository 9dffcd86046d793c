"""Host logic of bench.py: the algorithmic byte counts behind the roofline
(Sec. 5.2 layout: per token per sweep the document phase reads perm and reads
and writes z and M proposals, the word phase reads and writes them) and the
--tuning parser."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_bytes_per_token():
    assert bench.sweep_alg_bytes(1) == 36 and bench.sweep_alg_bytes(2) == 52
    for M in (1, 2, 3, 4):
        doc = bench.alg_bytes_per_token("doc_batch", M)
        word = bench.alg_bytes_per_token("word_batch", M)
        assert doc == 4 + 8 * (M + 1) and word == 8 * (M + 1)
        assert doc + word == bench.sweep_alg_bytes(M)
    assert bench.alg_bytes_per_token("finalize_ck", 2) == 0


def test_tuning_parser():
    assert bench.parse_tuning("") is None
    assert bench.parse_tuning("doc_warp_max=256, batch_max_tokens=64") == {
        "doc_warp_max": 256, "batch_max_tokens": 64}
    for bad in ("nope=1", "doc_warp_max", "doc_warp_max=", "huge_chunk=x"):
        with pytest.raises((SystemExit, ValueError)):
            bench.parse_tuning(bad)
