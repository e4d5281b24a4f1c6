"""GPU checks of the float precision forms (FP16, split hi/lo FP16, FP8 e4m3),
the per-(channel, input) power-of-two scales and the FP64 block sums, all
against the FP64 oracle on the unquantised voltages (gains applied in FP64).

Error metrics (per channel, worst channel reported): Frobenius relative error
||dV||_F / ||V||_F and max |dV_ab| / sqrt(V_aa V_bb).  Tolerances: FP16 1e-3
(both), FP8 3e-2 Frobenius, HI/LO 2e-6 Frobenius.  The hi/lo bound is set by
the tensor-core accumulator: with exactly representable products, an fp32
TMEM accumulation still loses about 1e-8 per accumulated sample (relative,
growing linearly with the block length), so the hi/lo kernel restarts its
accumulator every 64 samples and sums the blocks in round-to-nearest fp32.
Measured values are printed (pytest -s)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc
from tests.test_parity_gpu import frob_and_maxnorm

pytestmark = pytest.mark.gpu

PRECS = {"fp16": xc.XC_PREC_FP16, "hilo": xc.XC_PREC_HILO, "fp8": xc.XC_PREC_FP8}
FROB_TOL = {"fp16": 1e-3, "hilo": 2e-6, "fp8": 3e-2}
HILO_BLOCK = 64


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def run(x, N, P, F, T, dtype, gains=None, **kw):
    eng = xc.Correlator(N, P, F, T, dtype, **kw)
    try:
        if gains is not None:
            eng.set_gains(torch.from_numpy(gains).float().to(x.device))
        return eng.correlate(x, sync=True).cpu().double().numpy()
    finally:
        eng.close()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_precision_forms_vs_fp64(prec, dtype, dev):
    # Ragged sizes: 72 inputs (one partial block), T not a multiple of 64.
    T, F, N, P = 700, 3, 36, 2
    x = synth.sky_voltages(T, F, N, P, noise_sigma=0.7, nsrc=4, src_amp=1.0, seed=71,
                           dtype=getattr(torch, dtype))
    g = synth.complex_gains(N, P, 71)
    want = oracle.correlate_f64(x.double().numpy(), gains=g)
    got = run(x.to(dev), N, P, F, T, dtype, gains=g, precision=PRECS[prec])
    frob, mx = frob_and_maxnorm(got, want, N, P)
    print(f"\n{prec} {dtype}: frobenius {frob:.3e} max-norm {mx:.3e}")
    assert frob <= FROB_TOL[prec], frob
    if prec == "fp16":
        assert mx <= 1e-3, mx


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_precision_forms_direct_load_converter(prec, dtype, dev):
    """n = 37 (P = 1): rows are not 16-byte strided, so the converter loads
    the input directly instead of through TMA boxes."""
    T, F, N, P = 300, 2, 37, 1
    x = synth.sky_voltages(T, F, N, P, noise_sigma=0.7, nsrc=2, src_amp=1.0, seed=72,
                           dtype=getattr(torch, dtype))
    g = synth.complex_gains(N, P, 72)
    want = oracle.correlate_f64(x.double().numpy(), gains=g)
    got = run(x.to(dev), N, P, F, T, dtype, gains=g, precision=PRECS[prec])
    frob, mx = frob_and_maxnorm(got, want, N, P)
    print(f"\n{prec} {dtype} direct: frobenius {frob:.3e} max-norm {mx:.3e}")
    assert frob <= FROB_TOL[prec], frob


@pytest.mark.parametrize("prec", list(PRECS))
def test_scales_cover_fp32_range(prec, dev):
    """Inputs far outside the fp16 / e4m3 range (and far below it) keep the
    same relative error: the power-of-two scales follow each input."""
    T, F, N, P = 256, 2, 8, 2
    x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=1.0, seed=73)
    mag = torch.tensor([1e9, 1e-9, 3e4, 1.0, 7e-3, 2e6, 1e-5, 5e2], dtype=torch.float32)
    x = (x * mag[None, None, :, None, None]).contiguous()
    want = oracle.correlate_f64(x.double().numpy())
    got = run(x.to(dev), N, P, F, T, "float32", precision=PRECS[prec])
    frob, mx = frob_and_maxnorm(got, want, N, P)
    print(f"\n{prec} wide range: frobenius {frob:.3e} max-norm {mx:.3e}")
    assert np.isfinite(got).all()
    assert mx <= {"fp16": 2e-3, "hilo": 1e-5, "fp8": 1e-1}[prec], mx


def test_hilo_beats_fp16(dev):
    T, F, N, P = 512, 2, 24, 2
    x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=3, src_amp=1.0, seed=75)
    want = oracle.correlate_f64(x.double().numpy())
    xd = x.to(dev)
    e16, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float32"), want, N, P)
    ehl, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float32", precision=xc.XC_PREC_HILO),
                              want, N, P)
    ehb, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float32", precision=xc.XC_PREC_HILO,
                                  fp64_block=HILO_BLOCK), want, N, P)
    print(f"\nfp16 {e16:.3e} hilo {ehl:.3e} hilo+fp64/{HILO_BLOCK} {ehb:.3e}")
    assert ehl < e16 / 30
    assert ehb < e16 / 30


def test_fp64_block_sums_long_integration(dev):
    """fp16-valued input without gains: every product is exact, so the error
    left is the fp32 accumulation, which FP64 block sums shorten to T_blk."""
    T, F, N, P = 32768, 2, 8, 2
    x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=2.0, seed=77,
                           dtype=torch.float16)
    want = oracle.correlate_f64(x.double().numpy())
    xd = x.to(dev)
    e32, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float16"), want, N, P)
    e512, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float16", fp64_block=512), want, N, P)
    e64, _ = frob_and_maxnorm(run(xd, N, P, F, T, "float16", fp64_block=64), want, N, P)
    print(f"\nT={T}: fp32 accumulation {e32:.3e}, FP64 block sums /512 {e512:.3e} /64 {e64:.3e}")
    assert e64 <= 1e-6
    assert e512 < e32 / 30 and e64 < e512


@pytest.mark.parametrize("nblocks", [1, 2, 3, 4], ids=["one_block", "one_pair", "pair_plus_one", "two_pairs"])
@pytest.mark.parametrize("P", [2, 1])
def test_fp64_block_sums_overwrite_each_call(nblocks, P, dev):
    """Without ACCUMULATE every call's result replaces `out`: the same handle
    called twice into an output prefilled with garbage gives one
    integration's visibilities.  Covers a single fp32 chunk, one chunk pair
    (summed in TMEM and stored directly), a pair plus a single chunk and two
    pairs (float64 running sum), both polarisation counts."""
    blk, F, N = 128, 3, 40
    T = blk * nblocks
    x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=1.0, seed=81 + nblocks)
    want = oracle.correlate_f64(x.double().numpy())
    eng = xc.Correlator(N, P, F, T, "float32", fp64_block=blk)
    try:
        out = eng.new_output()
        out.fill_(7.0)
        xd = x.to(dev)
        for _ in range(2):
            eng.correlate(xd, out=out)
        eng.synchronize()
        got = out.cpu().double().numpy()
    finally:
        eng.close()
    frob, mx = frob_and_maxnorm(got, want, N, P)
    assert frob <= FROB_TOL["fp16"] and mx <= 1e-3, (frob, mx)


def test_fp64_block_sums_accumulate_across_calls(dev):
    """ACCUMULATE with FP64 block sums continues the handle's float64 running
    sum: three calls equal one integration over the concatenated samples."""
    T, F, N, P = 640, 2, 12, 1
    parts = [synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=1.0, seed=79 + i)
             for i in range(3)]
    want = oracle.correlate_f64(torch.cat(parts).double().numpy())
    eng = xc.Correlator(N, P, F, T, "float32", accumulate=True, precision=xc.XC_PREC_HILO,
                        fp64_block=HILO_BLOCK)
    try:
        out = eng.new_output()
        for x in parts:
            eng.correlate(x.to(dev), out=out)
        eng.synchronize()
        got = out.cpu().double().numpy()
    finally:
        eng.close()
    frob, _ = frob_and_maxnorm(got, want, N, P)
    print(f"\naccumulated hilo+fp64: frobenius {frob:.3e}")
    assert frob <= FROB_TOL["hilo"]


def test_precision_options_validated(dev):
    eng = xc.Correlator(8, 2, 2, 64, "int8")
    try:
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_PRECISION, xc.XC_PREC_HILO)
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_FP64_BLOCK, 128)
        eng.set_option(xc.XC_OPT_PRECISION, xc.XC_PREC_FP8)  # exact for |x| <= 16
    finally:
        eng.close()
    eng = xc.Correlator(8, 2, 2, 64, "float32")
    try:
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_PRECISION, 7)
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_FP64_BLOCK, 100)
        eng.set_option(xc.XC_OPT_PRECISION, xc.XC_PREC_FP8)
        eng.set_option(xc.XC_OPT_ENGINE, xc.XC_ENGINE_FP32)
        x = torch.zeros(eng.in_shape, device=dev)
        with pytest.raises(xc.XcError):
            eng.correlate(x)
    finally:
        eng.close()


@pytest.fixture(scope="module")
def precision_workload(dev):
    """Precision workload at full size (N=512 x 2 pols, F=480, T=2048, fp16
    input, random gains) and the FP64 oracle on 32 seeded channels."""
    w = synth.PRECISION
    x, g = synth.precision_input(w, device=dev)
    x16 = x.to(torch.float16)
    del x
    rng = np.random.default_rng(w.seed + 3)
    chans = sorted(rng.choice(w.nfreq, size=32, replace=False).tolist())
    want = oracle.correlate_f64(x16[:, chans].cpu().double().numpy(), gains=g)
    return w, x16, g, chans, want


@pytest.mark.parametrize("prec,fp64_block", [("fp16", 0), ("hilo", 0), ("fp8", 0), ("fp16", 1024)],
                         ids=["fp16", "hilo", "fp8", "fp16_fp64_blocks"])
def test_precision_workload_sampled(prec, fp64_block, precision_workload, dev):
    """Each precision form on the full precision workload, in the launch the
    benchmark times: errors of 32 seeded channels against the FP64 oracle."""
    w, x16, g, chans, want = precision_workload
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "float16", precision=PRECS[prec],
                        fp64_block=fp64_block)
    try:
        eng.set_gains(torch.from_numpy(g).float().to(dev))
        out = eng.correlate(x16, sync=True)
        got = out[chans].cpu().double().numpy()
    finally:
        eng.close()
    frob, mx = frob_and_maxnorm(got, want, w.nstation, w.npol)
    print(f"\nprecision workload {prec} (fp64 blocks {fp64_block}): frobenius {frob:.3e} max-norm {mx:.3e}")
    assert frob <= FROB_TOL[prec], frob
    if prec == "fp16":
        assert mx <= 1e-3, mx
