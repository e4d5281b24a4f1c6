"""8-bit input on the FP8 tensor path (XC_PREC_FP8): e4m3 holds every integer
with |x| <= 16 exactly, products are exact in fp32 and the exact-chunk rule
keeps every partial sum an integer, so 4-bit to 5-bit data stays bit-exact
against the int64 oracle.  Larger values are reported, not silently rounded."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def run_fp8(x, dev, N, P, F, T):
    eng = xc.Correlator(N, P, F, T, "int8", precision=xc.XC_PREC_FP8)
    try:
        out = eng.correlate(x.to(dev), sync=False)
        st = xc.xc_synchronize(eng.h, torch.cuda.current_stream().cuda_stream)
        return out.cpu().numpy(), st
    finally:
        eng.close()


# (N, P, F, T): TMA-staged converter (rows 16-byte strided) and direct loads
# (N=37 x 2 pols: 148-byte rows; N=35 x 1), ragged blocks, several K-blocks.
SHAPES = [(16, 2, 8, 256), (200, 2, 6, 300), (37, 2, 5, 200), (35, 1, 4, 130), (64, 2, 3, 1100)]


@pytest.mark.parametrize("N,P,F,T", SHAPES, ids=["tiny", "n400", "direct_n74", "direct_p1", "T1100"])
@pytest.mark.parametrize("lo,hi", [(-7, 7), (-16, 16)], ids=["4bit", "pm16"])
def test_fp8_path_bit_exact(N, P, F, T, lo, hi, dev):
    x = synth.uniform_int8((T, F, N, P, 2), lo, hi, 1000 + N + T + hi)
    got, st = run_fp8(x, dev, N, P, F, T)
    assert st == xc.XC_OK, xc.status_string(st)
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


def test_fp8_path_all_16(dev):
    N, P, F, T = 24, 2, 2, 512
    x = torch.full((T, F, N, P, 2), -16, dtype=torch.int8)
    x[::2, :, ::3] = 16
    got, st = run_fp8(x, dev, N, P, F, T)
    assert st == xc.XC_OK
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


@pytest.mark.parametrize("N,P", [(16, 2), (37, 2)], ids=["tma", "direct"])
def test_fp8_path_reports_out_of_range(N, P, dev):
    F, T = 3, 128
    x = synth.uniform_int8((T, F, N, P, 2), -7, 7, 77)
    x[5, 1, 3, 0, 1] = 17
    _, st = run_fp8(x, dev, N, P, F, T)
    assert st == xc.XC_ERR_OVERFLOW_RISK, xc.status_string(st)


def test_fp8_range_status_clears(dev):
    # After a range report the status word is clear: the next in-range call is exact and OK.
    N, P, F, T = 16, 2, 2, 128
    x = synth.uniform_int8((T, F, N, P, 2), -16, 16, 78)
    bad = x.clone()
    bad[0, 0, 0, 0, 0] = -17
    eng = xc.Correlator(N, P, F, T, "int8", precision=xc.XC_PREC_FP8)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        out = eng.new_output()
        eng.correlate(bad.to(dev), out=out)
        assert xc.xc_synchronize(eng.h, stream) == xc.XC_ERR_OVERFLOW_RISK
        eng.correlate(x.to(dev), out=out)
        assert xc.xc_synchronize(eng.h, stream) == xc.XC_OK
        got = out.cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))
