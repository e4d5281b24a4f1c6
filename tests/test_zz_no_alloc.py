"""The no-allocation entry point, xc_correlate_noalloc.

It serves callers that may not allocate device memory (a real-time loop
whose memory was reserved at start-up, an application whose memory belongs
to another allocator, a plug-in that must not allocate in its callback):
they cannot create a handle, because xc_create allocates a workspace.  The
call keeps its scratch in the library's static device array instead and runs
the same kernel as xc_correlate.

These tests call it through the C ABI and compare its visibilities with the
handle-based xc_correlate, bit for bit (the same kernel, so float results are
identical too), over two calls in a row with different sizes and inputs, so
the second call also shows that what the first left in the shared scratch
does not leak into its result.  Float inputs far from unit amplitude (1e5 and
1e-6) are also checked against the FP64 oracle: the per-input scaling keeps
them inside fp16's range.  The file is named to be collected last."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc

pytestmark = pytest.mark.gpu

CODES = {"int8": xc.XC_CI8, "float16": xc.XC_CF16, "float32": xc.XC_CF32}


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def reference_output(x, dtype):
    T, F, N, P, _ = x.shape
    eng = xc.Correlator(N, P, F, T, dtype)
    try:
        return eng.correlate(x, sync=True).clone()
    finally:
        eng.close()


def noalloc_output(x, dtype, dev):
    T, F, N, P, _ = x.shape
    out = torch.full((F, N * (N + 1) // 2, P * P, 2), -7,
                     dtype=torch.int32 if dtype == "int8" else torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = xc.xc_correlate_noalloc(N, P, F, T, CODES[dtype], x.data_ptr(), out.data_ptr(),
                                 status.data_ptr(), stream.cuda_stream)
    assert st == xc.XC_OK, xc.xc_last_error_message()
    torch.cuda.synchronize(dev)
    assert int(status.item()) == 0, "a bounded wait gave up"
    return out


def test_noalloc_matches_xc_correlate_two_calls(dev):
    # Call 1: Large-N geometry with 80 channels (2 MiB of operands per
    # channel: the ring of the static scratch wraps twice).  Call 2: a
    # different geometry (ragged N, T beyond one exact chunk) over the scratch
    # call 1 filled.
    w = synth.Workload("noalloc call 1", 256, 2, 80, 1000, 5151)
    x1 = synth.int8_sky(w, device=dev)
    x2 = synth.uniform_int8((1500, 5, 70, 2, 2), -128, 127, 5252, device=dev)
    for x in (x1, x2):
        want = reference_output(x, "int8")
        got = noalloc_output(x, "int8", dev)
        assert torch.equal(got, want)


def test_noalloc_single_pol_and_fp16(dev):
    """npol = 1 over several 128-input blocks, and fp16 input (the 32-bit
    TMA converter), each twice in a row."""
    x1 = synth.uniform_int8((300, 7, 200, 1, 2), -128, 127, 5454, device=dev)
    x2 = synth.sky_voltages(260, 6, 100, 2, noise_sigma=0.8, nsrc=2, src_amp=1.0, seed=5455,
                            device=dev).to(torch.float16)
    for x, dt in ((x1, "int8"), (x2, "float16"), (x1, "int8"), (x2, "float16")):
        want = reference_output(x, dt)
        got = noalloc_output(x, dt, dev)
        assert torch.equal(got, want), dt


@pytest.mark.parametrize("amplitude", [1.0, 1e5, 1e-6], ids=["unit", "1e5", "1e-6"])
def test_noalloc_float_input(amplitude, dev):
    """Float input: identical to xc_correlate on two calls in a row, and
    within the parity tests' float tolerance of the FP64 oracle at any
    amplitude (fp16 alone would overflow at 1e5 and underflow at 1e-6)."""
    from tests.test_parity_gpu import frob_and_maxnorm
    N, P = 40, 2
    x = synth.sky_voltages(300, 6, N, P, noise_sigma=0.7, nsrc=2, src_amp=1.0, seed=5353) * amplitude
    xd = x.to(dev)
    want_dev = reference_output(xd, "float32")
    for _ in range(2):
        got = noalloc_output(xd, "float32", dev)
        assert torch.equal(got, want_dev)
    want = oracle.correlate_f64(x.double().numpy())
    frob, mx = frob_and_maxnorm(got.cpu().double().numpy(), want, N, P)
    assert frob <= 1e-3 and mx <= 1e-3, (frob, mx)


def test_noalloc_rejects_sizes_beyond_its_scratch(dev):
    # N=1024 x 2 pols at T=8256: one channel slot is 2048 inputs x 8256 -> 8320
    # samples x 2 planes x 2 B = 68 MB, more than the 64 MiB scratch.
    x = torch.zeros(16, dtype=torch.int8, device=dev)
    out = torch.zeros(16, dtype=torch.int32, device=dev)
    st = xc.xc_correlate_noalloc(1024, 2, 1, 8256, xc.XC_CI8, x.data_ptr(), out.data_ptr(), 0, 0)
    assert st == xc.XC_ERR_UNSUPPORTED
    assert "static scratch" in xc.xc_last_error_message()
