"""Stored fixtures: the oracle digest (written by tests/golden/make_golden.py,
oracle only) and the paper's printed numbers."""
import json
import os

from tests.golden import make_golden

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_tiny_oracle_digest_unchanged():
    with open(os.path.join(HERE, "tiny_oracle_digest.json")) as fh:
        want = json.load(fh)
    got = make_golden.digest()
    for key in ("input_sha256", "output_sha256", "sum", "sum_abs", "v_f3_k100"):
        assert got[key] == want[key], key
