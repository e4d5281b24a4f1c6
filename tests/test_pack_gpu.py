"""Small arrays on the planar engine: when n = N P <= 64, k consecutive
channels (k the largest divisor of F with k n <= 128) are correlated as one
virtual channel of k N stations.  The input [T][F][n] is the same memory as
[T][F / k][k n]; one 128 x 128 block holds the k channels' own blocks on its
diagonal, and the epilogue stores only those, at the real channel's indices.

Every case is checked against the oracle, which knows nothing of packing:
8-bit input bit for bit (both polarisation counts, odd and prime channel
counts, integrations longer than the exact-fp32 chunk, accumulate mode, the
batched launch), float input with gains in each precision form and with FP64
block sums within the precision tests' tolerances."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc
from tests.test_parity_gpu import frob_and_maxnorm

pytestmark = pytest.mark.gpu

FROB_TOL = {"fp16": 1e-3, "hilo": 2e-6, "fp8": 3e-2}
PRECS = {"fp16": xc.XC_PREC_FP16, "hilo": xc.XC_PREC_HILO, "fp8": xc.XC_PREC_FP8}


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def pack_of(N, P, F):
    """The packing the engine chooses (restated here only to label cases)."""
    n = N * P
    if n > 64:
        return 1
    for c in range(128 // n, 1, -1):
        if F % c == 0:
            return c
    return 1


# (N, P, F, T): pack 4 (n = 32), pack 6 (n = 20, n' = 120), P = 1 with pack 10,
# prime F = 7 with pack 7, pack 2 (n = 64) over two exact chunks (T > 1024),
# n = 48 with F = 9 (no divisor <= 2: unpacked), F = 1 (unpacked), N = 1.
INT_CASES = [(16, 2, 12, 300), (10, 2, 12, 130), (7, 1, 10, 200), (5, 2, 7, 64),
             (32, 2, 6, 1100), (24, 2, 9, 100), (16, 2, 1, 64), (1, 2, 16, 70), (3, 1, 40, 65)]


@pytest.mark.parametrize("N,P,F,T", INT_CASES,
                         ids=["N%d_P%d_F%d_T%d_k%d" % (c + (pack_of(c[0], c[1], c[2]),)) for c in INT_CASES])
def test_packed_int8_bit_exact(N, P, F, T, dev):
    x = synth.uniform_int8((T, F, N, P, 2), -128, 127, 900 + N * F + T)
    # XC_TILE_128: sizes the small-array engine serves would leave the planar
    # engine (and its packing) under XC_TILE_AUTO.
    eng = xc.Correlator(N, P, F, T, "int8", tile=xc.XC_TILE_128)
    try:
        got = eng.correlate(x.to(dev), sync=True).cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


def test_packed_int8_accumulate(dev):
    N, P, F, T = 12, 2, 20, 256  # n = 24: pack 5
    xa = synth.uniform_int8((T, F, N, P, 2), -128, 127, 911)
    xb = synth.uniform_int8((T, F, N, P, 2), -128, 127, 912)
    eng = xc.Correlator(N, P, F, T, "int8", accumulate=True, tile=xc.XC_TILE_128)
    try:
        out = eng.new_output()
        out.zero_()
        eng.correlate(xa.to(dev), out=out)
        eng.correlate(xb.to(dev), out=out, sync=True)
        got = out.cpu().numpy()
    finally:
        eng.close()
    want = oracle.correlate_i8(xa.numpy()) + oracle.correlate_i8(xb.numpy())
    np.testing.assert_array_equal(got, want)


def test_packed_fp8_4bit_exact(dev):
    N, P, F, T = 16, 2, 8, 512
    x = synth.uniform_int8((T, F, N, P, 2), -16, 16, 913)
    eng = xc.Correlator(N, P, F, T, "int8", precision=xc.XC_PREC_FP8)
    try:
        got = eng.correlate(x.to(dev), sync=True).cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_packed_float_with_gains(prec, dtype, dev):
    T, F, N, P = 256, 10, 12, 2  # n = 24: pack 5, two virtual channels
    x = synth.sky_voltages(T, F, N, P, noise_sigma=0.8, nsrc=2, src_amp=1.0, seed=914,
                           dtype=getattr(torch, dtype))
    g = synth.complex_gains(N, P, 914)
    want = oracle.correlate_f64(x.double().numpy(), gains=g)
    eng = xc.Correlator(N, P, F, T, dtype, precision=PRECS[prec])
    try:
        eng.set_gains(torch.from_numpy(g).float().to(dev))
        got = eng.correlate(x.to(dev), sync=True).cpu().double().numpy()
    finally:
        eng.close()
    frob, mx = frob_and_maxnorm(got, want, N, P)
    print(f"\npacked {prec} {dtype}: frobenius {frob:.3e} max-norm {mx:.3e}")
    assert frob <= FROB_TOL[prec], frob


def test_packed_float_direct_loads_and_fp64_blocks(dev):
    # n = 9 (P = 1, odd): rows are not 16-byte strided, so the converter loads
    # directly; pack 12 of F = 24; FP64 block sums over 128-sample blocks.
    T, F, N, P = 700, 24, 9, 1
    x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=1.0, seed=915)
    g = synth.complex_gains(N, P, 915)
    want = oracle.correlate_f64(x.double().numpy(), gains=g)
    eng = xc.Correlator(N, P, F, T, "float32", fp64_block=128)
    try:
        eng.set_gains(torch.from_numpy(g).float().to(dev))
        got = eng.correlate(x.to(dev), sync=True).cpu().double().numpy()
    finally:
        eng.close()
    frob, _ = frob_and_maxnorm(got, want, N, P)
    assert frob <= 1e-3, frob


def test_packed_batch_subarrays(dev):
    subs = [(8, 16, 128), (16, 12, 200), (300, 2, 64), (4, 30, 96)]
    xs = [synth.uniform_int8((T, F, N, 2, 2), -128, 127, 916 + i) for i, (N, F, T) in enumerate(subs)]
    bc = xc.BatchCorrelator(subs, npol=2)
    try:
        outs = bc.correlate([x.to(dev) for x in xs], sync=True)
        for x, o in zip(xs, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.correlate_i8(x.numpy()))
    finally:
        bc.close()
