"""The small-array engine (XC_TILE_SMALL): 8-bit input with W = 2 N P in
{16, 32, 64, 128, 256} real rows per channel.

Each input is two real rows of a 128-row tile holding 128 / W channels (or,
at W = 256, of two tiles holding one channel); 128 x 128 MMAs per 16-sample
step form the real Gram matrix of the tile rows (three lower tile blocks at
W = 256), and the epilogue combines its 2 x 2 sub-blocks into V.  Every case
is compared with the oracle bit for bit (the 8-bit path is exact): all five
widths with both polarisation counts,
channel counts that leave the last tile part-empty, integrations shorter than
one 64-sample stage, ragged against it, exactly one exact-fp32 chunk, one
sample past it, and several chunks; full-scale -128 input at the chunk
length where the fp32 sums reach 2^24; T split across CTAs (few channels,
long T) with and without accumulation; and, at the sweep's channel count, a
sample of channels spread over the whole launch.  XC_TILE_AUTO must pick the
engine for these sizes and agree with the planar engine (XC_TILE_128).  With
e4m3 operands (XC_PREC_FP8) 4-bit-class data (|x| <= 16) is bit-exact too,
and a larger value is reported."""
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


def run(x, dev, tile=xc.XC_TILE_SMALL, accumulate=False, out=None, reps=1):
    T, F, N, P, _ = x.shape
    eng = xc.Correlator(N, P, F, T, "int8", tile=tile, accumulate=accumulate)
    try:
        if out is None:
            out = eng.new_output()
        xd = x.to(dev)
        for _ in range(reps):
            eng.correlate(xd, out=out)
        eng.synchronize()
        return out.cpu().numpy()
    finally:
        eng.close()


# (N, P, F, T): W = 16, 32, 64, 128, 256 with P = 2 and P = 1; F not a
# multiple of the channels per tile; T short, ragged, one chunk, chunk + 1,
# several chunks.
CASES = [(4, 2, 17, 300), (8, 2, 9, 1000), (16, 2, 5, 1024), (32, 2, 3, 1025),
         (8, 1, 13, 70), (16, 1, 7, 2500), (32, 1, 3, 33), (64, 1, 2, 3000),
         (16, 2, 1, 1), (4, 2, 8, 64), (64, 2, 7, 1000), (64, 2, 3, 2500), (128, 1, 5, 300),
         (64, 2, 1, 33)]


@pytest.mark.parametrize("N,P,F,T", CASES, ids=["N%d_P%d_F%d_T%d" % c for c in CASES])
def test_small_engine_bit_exact(N, P, F, T, dev):
    assert xc.load().xc_small_engine_channels(N, P) == max(1, 128 // (2 * N * P))
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7100 + 3 * N + F + T)
    np.testing.assert_array_equal(run(x, dev), oracle.correlate_i8(x.numpy()))


@pytest.mark.parametrize("N", [32, 64])
def test_small_engine_full_scale_chunk(N, dev):
    """All samples -128 over exactly 1024 samples: every fp32 sum of the
    Gram matrix reaches 128^2 * 1024 = 2^24, the largest exact chunk."""
    P, F, T = 2, 2, 1024
    x = torch.full((T, F, N, P, 2), -128, dtype=torch.int8)
    got = run(x, dev)
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))
    assert got[0, 0, 0, 0] == 2 * 128 * 128 * T  # re(x) re(x) + im(x) im(x)


@pytest.mark.parametrize("accumulate", [False, True], ids=["store", "accumulate"])
@pytest.mark.parametrize("N", [16, 64])
def test_small_engine_split_t(accumulate, N, dev):
    """Two (N=16) or four (N=64) channel groups and 20 chunks: T is split
    across CTAs and the partial sums meet in the output by integer atomics."""
    P, F, T = 2, 4, 20000
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7201)
    want = oracle.correlate_i8(x.numpy())
    if accumulate:
        got = run(x, dev, accumulate=True, out=torch.zeros(want.shape, dtype=torch.int32, device=dev), reps=2)
        np.testing.assert_array_equal(got, 2 * want)
    else:
        np.testing.assert_array_equal(run(x, dev, reps=2), want)


def test_small_engine_accumulate_single_segment(dev):
    N, P, F, T = 8, 2, 400, 1500
    xa = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7202)
    xb = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7203)
    eng = xc.Correlator(N, P, F, T, "int8", accumulate=True)
    try:
        out = eng.new_output()
        out.zero_()
        eng.correlate(xa.to(dev), out=out)
        eng.correlate(xb.to(dev), out=out, sync=True)
        got = out.cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_array_equal(got, oracle.correlate_i8(xa.numpy()) + oracle.correlate_i8(xb.numpy()))


@pytest.mark.parametrize("N,P", [(16, 2), (32, 2), (8, 2), (64, 1), (64, 2)])
def test_auto_picks_small_engine_and_matches_planar(N, P, dev):
    F, T = 37, 500
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7300 + N)
    auto = run(x, dev, tile=xc.XC_TILE_AUTO)
    planar = run(x, dev, tile=xc.XC_TILE_128)
    np.testing.assert_array_equal(auto, planar)
    np.testing.assert_array_equal(auto, oracle.correlate_i8(x.numpy()))


@pytest.mark.parametrize("N,F", [(16, 65528), (32, 65104), (64, 16520)])
def test_small_engine_sweep_size_sampled(N, F, dev):
    """The N sweep's sizes (T = 1000): the whole launch, checked on channels
    spread over it (first, last, and across the persistent CTAs' turns)."""
    P, T = 2, 1000
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7400 + N, device=dev)
    got = run(x, dev)
    chans = sorted({0, 1, 2, 151, 152, 303, 304, F // 3, F // 2, F - 2, F - 1} |
                   set(range(5000, F, 9973)))
    xs = x[:, chans].cpu().numpy()
    want = oracle.correlate_i8(xs)
    np.testing.assert_array_equal(got[chans], want)


def test_tile_small_rejected_where_it_does_not_apply(dev):
    eng = xc.Correlator(24, 2, 4, 64, "int8", tile=xc.XC_TILE_SMALL)  # W = 96
    try:
        x = torch.zeros(eng.in_shape, dtype=torch.int8, device=dev)
        with pytest.raises(xc.XcError):
            eng.correlate(x, sync=True)
    finally:
        eng.close()
    assert xc.load().xc_small_engine_channels(24, 2) == 0
    assert xc.load().xc_small_engine_channels(96, 2) == 0


@pytest.mark.parametrize("N", [16, 64])
def test_noalloc_small_engine(N, dev):
    """xc_correlate_noalloc runs the small-array engine for these sizes, with
    results identical to xc_correlate's."""
    P, F, T = 2, 300, 1100
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 7500, device=dev)
    want = run(x, dev, tile=xc.XC_TILE_AUTO)
    out = torch.full(want.shape, -7, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    st = xc.xc_correlate_noalloc(N, P, F, T, xc.XC_CI8, x.data_ptr(), out.data_ptr(), status.data_ptr(),
                                 torch.cuda.current_stream(dev).cuda_stream)
    assert st == xc.XC_OK, xc.xc_last_error_message()
    torch.cuda.synchronize(dev)
    assert int(status.item()) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), want)


FP8_CASES = [(4, 2, 9, 300), (8, 2, 5, 1000), (16, 2, 7, 1025), (32, 2, 3, 70), (16, 1, 4, 2500),
             (64, 2, 3, 1000), (128, 1, 2, 300)]


@pytest.mark.parametrize("N,P,F,T", FP8_CASES, ids=["N%d_P%d_F%d_T%d" % c for c in FP8_CASES])
def test_small_engine_fp8_4bit_exact(N, P, F, T, dev):
    """e4m3 operands (XC_PREC_FP8) on the small-array engine: 4-bit-class
    data (|x| <= 16, full range of it) stays bit-exact against the oracle."""
    x = synth.uniform_int8((T, F, N, P, 2), -16, 16, 7600 + N + F + T)
    eng = xc.Correlator(N, P, F, T, "int8", tile=xc.XC_TILE_SMALL, precision=xc.XC_PREC_FP8)
    try:
        out = eng.correlate(x.to(dev))
        st = xc.xc_synchronize(eng.h, torch.cuda.current_stream().cuda_stream)
        got = out.cpu().numpy()
    finally:
        eng.close()
    assert st == xc.XC_OK, xc.status_string(st)
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


@pytest.mark.parametrize("N", [16, 64])
def test_small_engine_fp8_reports_out_of_range(N, dev):
    P, F, T = 2, 3, 200
    x = synth.uniform_int8((T, F, N, P, 2), -7, 7, 7700 + N)
    x[150, 2, N - 1, 1, 0] = -17
    eng = xc.Correlator(N, P, F, T, "int8", tile=xc.XC_TILE_SMALL, precision=xc.XC_PREC_FP8)
    try:
        eng.correlate(x.to(dev))
        st = xc.xc_synchronize(eng.h, torch.cuda.current_stream().cuda_stream)
    finally:
        eng.close()
    assert st == xc.XC_ERR_OVERFLOW_RISK, xc.status_string(st)
