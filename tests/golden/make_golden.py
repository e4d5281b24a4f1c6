"""Write tests/golden/tiny_oracle_digest.json from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The digest records the oracle's integer visibilities of the tiny workload
(N=16, P=2, F=8, T=256, uniform integers in [-7, 7], seed 1107) so that a
silent change of the generator or the oracle shows up in the tests."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1107_4264_gb300 import synth  # noqa: E402


def digest():
    x = synth.tiny_input(synth.TINY).numpy()
    v = oracle.correlate_i8(x)
    return {
        "workload": synth.TINY.name,
        "seed": synth.TINY.seed,
        "input_sha256": hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest(),
        "output_sha256": hashlib.sha256(np.ascontiguousarray(v.astype("<i8")).tobytes()).hexdigest(),
        "sum": int(v.sum()),
        "sum_abs": int(np.abs(v).sum()),
        "v_f3_k100": v[3, 100].tolist(),
        "written_by": "tests/golden/make_golden.py (calls only oracle/)",
    }


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle_digest.json")
    with open(path, "w") as fh:
        json.dump(digest(), fh, indent=1)
        fh.write("\n")
    print("wrote", path)
