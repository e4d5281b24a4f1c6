"""Failure detection without a GPU fault.

Device side: the converters of the planar engine are told (test hook
XC_OPT_TEST_NO_PUBLISH) never to publish a converted unit, and those of the
small-array engine never to mark a converted tile full, so every wait of the
kernel's consumers runs out after XC_OPT_TIMEOUT_MS.  The kernel must then
finish its in-flight copies and MMAs, free its tensor memory and return; the
host reads XC_ERR_TIMEOUT from xc_synchronize, and the same handle must give
exact results on its next call.  Host side: allocation failure and bad
arguments come back as status codes."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


# 8-bit (TMA converter) and fp16 with n % 4 == 0 (TMA float converter) at
# N = 256 x 2 pols, where 40 channels exceed the ring's 29 slots, so the
# converters' slot claims run out too; fp32 with n odd (direct-load converter);
# 8-bit at N = 16 and N = 64 x 2 pols (the small-array engine, one tile and
# two tiles per channel).
CASES = [("int8", 256, 2, 40, 128), ("float16", 256, 2, 40, 128), ("float32", 33, 1, 40, 130),
         ("int8", 16, 2, 40, 128), ("int8", 64, 2, 8, 300)]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,N,P,F,T", CASES, ids=["%s_N%d" % (c[0], c[1]) for c in CASES])
def test_waits_run_out_and_handle_recovers(dtype, N, P, F, T, dev):
    if dtype == "int8":
        x = synth.uniform_int8((T, F, N, P, 2), -20, 20, 811)
        want = oracle.correlate_i8(x.numpy())
    else:
        x = synth.sky_voltages(T, F, N, P, noise_sigma=0.7, nsrc=2, src_amp=1.0, seed=812,
                               dtype=getattr(torch, dtype))
        want = oracle.correlate_f64(x.double().numpy())
    xd = x.to(dev)
    eng = xc.Correlator(N, P, F, T, dtype, timeout_ms=200)
    try:
        eng.set_option(xc.XC_OPT_TEST_NO_PUBLISH, 1)
        out = eng.new_output()
        t0 = time.perf_counter()
        eng.correlate(xd, out=out)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        st = xc.xc_synchronize(eng.h, torch.cuda.current_stream().cuda_stream)
        assert st == xc.XC_ERR_TIMEOUT, xc.status_string(st)
        assert waited < 10.0, waited  # every wait is bounded
        # The status word was cleared and the context is usable: a normal call is exact.
        eng.set_option(xc.XC_OPT_TEST_NO_PUBLISH, 0)
        got = eng.correlate(xd, out=out, sync=True).cpu().numpy()
    finally:
        eng.close()
    if dtype == "int8":
        np.testing.assert_array_equal(got, want)
    else:
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert rel < 1e-3, rel


@pytest.mark.gpu
def test_allocation_failure_is_reported(dev):
    # Operand ring of terabytes: cudaMalloc fails and xc_create reports it.
    with pytest.raises(xc.XcError) as err:
        xc.xc_create(65536, 2, 64, 4_000_000, xc.XC_CF32)
    assert "XC_ERR_OOM" in str(err.value)
    # The device is still usable.
    eng = xc.Correlator(4, 2, 2, 64, "int8")
    try:
        x = synth.uniform_int8((64, 2, 4, 2, 2), -7, 7, 813)
        got = eng.correlate(x.to(dev), sync=True).cpu().numpy()
    finally:
        eng.close()
    np.testing.assert_array_equal(got, oracle.correlate_i8(x.numpy()))


@pytest.mark.gpu
def test_test_hook_option_validated(dev):
    eng = xc.Correlator(4, 2, 2, 64, "int8")
    try:
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_TEST_NO_PUBLISH, 2)
        with pytest.raises(xc.XcError):
            eng.set_option(xc.XC_OPT_TIMEOUT_MS, 0)
    finally:
        eng.close()


def test_null_handles_are_safe():
    lib = xc.load()
    lib.xc_destroy(None)  # NULL-safe
    assert lib.xc_set_option(None, xc.XC_OPT_TEST_NO_PUBLISH, 1) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_synchronize(None, None) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_batch_correlate(None, None, None, None) == xc.XC_ERR_INVALID_ARG
