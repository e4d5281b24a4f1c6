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


def _paper():
    with open(os.path.join(HERE, "paper_values.json")) as fh:
        return json.load(fh)


def test_work_model_matches_paper_normalisation():
    """The bench's executed-work model against the paper's own counts.

    Eq. flops (Sec. 2.1) per integration of T samples of F channels is
    8 F T (1/2) 2N(2N+1).  Sec. 6.1 counts the work of the diagonal blocks
    too: with N/RT diagonal blocks of 2RT x 2RT inputs, the total is the
    desired work times 2(N + RT)/(2N + 1).  The planar engine's blocks hold
    128 inputs, RT = 64 stations at P = 2, so for N a multiple of 64 and T a
    multiple of 64 (no padding) its executed operations must equal that
    normalised count exactly; first on the Table 3 case (N=512, F=6, I=1024)."""
    import bench
    from paper_1107_4264_gb300 import build as engine_build
    engine_build.build()
    p = _paper()
    rt = p["normalisation"]["block_stations_RT_here"]
    cases = [(p["table3_n512"]["nstation"], p["table3_n512"]["nfreq"], p["table3_n512"]["ntime"]),
             (256, 1024, 1024), (128, 8, 64), (1024, 3, 128), (64, 5, 192)]
    for N, F, T in cases:
        eq = 8 * F * T * N * (2 * N + 1)
        normalised = eq * 2 * (N + rt) // (2 * N + 1)
        assert eq * 2 * (N + rt) % (2 * N + 1) == 0
        assert bench.executed_ops(N, 2, F, T) == normalised, (N, F, T)
    # the Table 3 case: 2.58e10 desired, 2.90e10 with the diagonal waste
    N, F, T = cases[0]
    assert 8 * F * T * N * (2 * N + 1) == 25794969600
    assert bench.executed_ops(N, 2, F, T) == 28991029248


def test_stored_product_and_eq_flops_conventions():
    """The headline counts one CMAC per stored (baseline, polarisation
    product) per sample, 8 F T 2N(N+1); Eq. flops counts 8 F T N(2N+1).
    Their ratio, which the bench applies to print the Eq.-flops rate, is
    (2N+1)/(2(N+1)) (the two differ by the diagonal baselines' repeated
    cross-polarisation product)."""
    from paper_1107_4264_gb300 import synth
    w = synth.LARGE_N
    useful = w.useful_ops
    assert useful == 8 * w.nfreq * w.ntime * 2 * w.nstation * (w.nstation + 1)
    eq = 8 * w.nfreq * w.ntime * w.nstation * (2 * w.nstation + 1)
    assert abs(useful * (2 * w.nstation + 1) / (2 * (w.nstation + 1)) - eq) < 1e-6 * eq
