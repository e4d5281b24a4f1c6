"""GPU parity: every engine (fused tcgen05 planar complex form, the fused
interleaved form on single CTAs and on CTA pairs, the two-pass tensor-core
form and the FP32 CUDA-core form) against the CPU oracle through the C ABI.

Integer input must match bit for bit.  Cases span several 128-row tiles,
ragged station counts (partial tiles), single polarisation, sample counts
that are not multiples of the 64-sample K-block, integrations longer than
the 1024-sample exact-fp32 chunk of the tensor path, full-range int8
(including -128), accumulate mode, the integrated host pipeline (Algorithm 1
of Sec. 5) and, at the full Large-N size, sampled channels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc

pytestmark = pytest.mark.gpu

# (name, engine, tile shape of the planar tensor-core engine)
ENGINES = [("tensor", xc.XC_ENGINE_TENSOR, xc.XC_TILE_AUTO),
           ("tensor_128", xc.XC_ENGINE_TENSOR, xc.XC_TILE_128),
           ("tensor_pair", xc.XC_ENGINE_TENSOR, xc.XC_TILE_PAIR),
           ("tensor_wide", xc.XC_ENGINE_TENSOR, xc.XC_TILE_WIDE),
           ("fp32", xc.XC_ENGINE_FP32, xc.XC_TILE_AUTO),
           ("tensor_2pass", xc.XC_ENGINE_TENSOR_2PASS, xc.XC_TILE_AUTO),
           ("interleaved_1cta", xc.XC_ENGINE_TENSOR_1CTA, xc.XC_TILE_AUTO),
           ("interleaved_pair", xc.XC_ENGINE_TENSOR_PAIR, xc.XC_TILE_AUTO)]


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def run_engine(x_cpu, engine, dev, dtype="int8", accumulate=False, out=None, tile=xc.XC_TILE_AUTO):
    T, F, N, P, _ = x_cpu.shape
    eng = xc.Correlator(N, P, F, T, dtype, engine=engine, accumulate=accumulate, tile=tile)
    try:
        res = eng.correlate(x_cpu.to(dev).contiguous(), out=out, sync=True)
        return res.cpu()
    finally:
        eng.close()


def int_case(name, N, P, F, T, seed, lo=-7, hi=7, fill=None):
    if fill is not None:
        x = torch.full((T, F, N, P, 2), fill, dtype=torch.int8)
    else:
        x = synth.uniform_int8((T, F, N, P, 2), lo, hi, seed)
    return pytest.param(x, id=name)


INT_CASES = [
    int_case("tiny_N16_F8_T256", 16, 2, 8, 256, 1107),
    int_case("one_tile_N32_T1024", 32, 2, 4, 1024, 1),
    int_case("ragged_N200_F3_T77", 200, 2, 3, 77, 2, -128, 127),
    int_case("P1_N37_F2_T100", 37, 1, 2, 100, 3, -128, 127),
    int_case("P1_N130_F2_T64", 130, 1, 2, 64, 4, -128, 127),
    int_case("single_station_T5", 1, 2, 1, 5, 5, -128, 127),
    int_case("T1_N70", 70, 2, 2, 1, 6, -128, 127),
    int_case("drain_T3000_full_range", 40, 2, 2, 3000, 7, -128, 127),
    int_case("drain_T1025", 64, 2, 2, 1025, 8, -128, 127),
    int_case("all_minus128_T4096", 33, 2, 1, 4096, 0, fill=-128),
    int_case("all_127_T2048", 33, 2, 1, 2048, 0, fill=127),
    # many channels: the fused engine's operand ring wraps several times
    int_case("ring_wrap_N64_F100_T200", 64, 2, 100, 200, 9, -128, 127),
    int_case("ring_wrap_N160_F40_T1100", 160, 2, 40, 1100, 10, -128, 127),
]


@pytest.mark.parametrize("engine_name,engine,tile", ENGINES, ids=[e[0] for e in ENGINES])
@pytest.mark.parametrize("x", INT_CASES)
def test_int8_bit_exact(x, engine_name, engine, tile, dev):
    want = oracle.correlate_i8(x.numpy())
    got = run_engine(x, engine, dev, tile=tile).numpy().astype(np.int64)
    assert got.shape == want.shape
    mism = np.argwhere(got != want)
    assert mism.size == 0, "first mismatches %s: got %s want %s" % (
        mism[:4].tolist(), got[tuple(mism[0])], want[tuple(mism[0])])


def test_adversarial_sign_pattern(dev):
    """+-127 / -128 checkerboards over time and inputs, T = 2 chunks + tail."""
    T, F, N, P = 2100, 1, 64, 2
    t = torch.arange(T).view(T, 1, 1, 1, 1)
    a = torch.arange(N * P * 2).view(1, 1, N, P, 2)
    x = torch.where(((t // 3 + a) % 2) == 0, torch.tensor(127), torch.tensor(-128)).to(torch.int8)
    x = x.expand(T, F, N, P, 2).contiguous()
    want = oracle.correlate_i8(x.numpy())
    for _, engine, tile in ENGINES:
        got = run_engine(x, engine, dev, tile=tile).numpy().astype(np.int64)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("engine_name,engine,tile", ENGINES, ids=[e[0] for e in ENGINES])
def test_accumulate_mode(engine_name, engine, tile, dev):
    x1 = synth.uniform_int8((300, 3, 50, 2, 2), -128, 127, 21)
    x2 = synth.uniform_int8((300, 3, 50, 2, 2), -128, 127, 22)
    want = oracle.correlate_i8(x1.numpy()) + oracle.correlate_i8(x2.numpy())
    eng = xc.Correlator(50, 2, 3, 300, "int8", engine=engine, accumulate=True, tile=tile)
    try:
        out = eng.new_output(device=dev)
        eng.correlate(x1.to(dev), out=out)
        eng.correlate(x2.to(dev), out=out, sync=True)
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), want)
    finally:
        eng.close()


@pytest.mark.parametrize("N,F", [(48, 4), (16, 8)], ids=["N48", "N16_packed"])
def test_integrated_pipeline_matches_direct(N, F, dev):
    """Algorithm 1 (Sec. 5): integrations streamed from pinned host memory
    through two device buffers give the same visibilities as direct calls,
    in dump mode (one output per integration) and accumulate mode (N=16:
    four channels packed per tensor-core block)."""
    T, P, nint = 200, 2, 5
    xs = torch.stack([synth.uniform_int8((T, F, N, P, 2), -128, 127, 100 + i) for i in range(nint)])
    host = xs.pin_memory()
    want = [oracle.correlate_i8(xs[i].numpy()) for i in range(nint)]
    eng = xc.Correlator(N, P, F, T, "int8")
    try:
        out = eng.new_output(nint, device=dev)
        hout = torch.zeros((nint,) + eng.out_shape, dtype=torch.int32).pin_memory()
        eng.correlate_stream(host, nint, out, host_out=hout)
        eng.synchronize()
        for i in range(nint):
            np.testing.assert_array_equal(out[i].cpu().numpy().astype(np.int64), want[i])
            np.testing.assert_array_equal(hout[i].numpy().astype(np.int64), want[i])
        eng.set_option(xc.XC_OPT_ACCUMULATE, 1)
        acc = eng.new_output(device=dev)
        eng.correlate_stream(host, nint, acc)
        eng.synchronize()
        np.testing.assert_array_equal(acc.cpu().numpy().astype(np.int64), sum(want))
    finally:
        eng.close()


def test_large_n_sampled_channels(dev):
    """Full Large-N integration (N=256 x 2 pols, F=1024, T=1000) through the
    launch configuration the benchmark times; the oracle recomputes 6 sampled
    channels (first, last and 4 seeded) bit-exactly."""
    w = synth.LARGE_N
    x = synth.large_n_input(w, 0, device=dev)
    rng = np.random.default_rng(w.seed)
    chans = sorted(set([0, w.nfreq - 1] + rng.choice(w.nfreq, 4, replace=False).tolist()))
    xs = x[:, chans].cpu().numpy()
    want = oracle.correlate_i8(xs)
    for _, engine, tile in ENGINES:
        eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8", engine=engine, tile=tile)
        try:
            out = eng.correlate(x, sync=True)
            got = out[chans].cpu().numpy().astype(np.int64)
        finally:
            eng.close()
        np.testing.assert_array_equal(got, want)
        # properties that hold everywhere: autocorrelations real and non-negative
        auto = out[:, [s * (s + 1) // 2 + s for s in range(w.nstation)]]
        assert (auto[:, :, 0, 1] == 0).all() and (auto[:, :, 0, 0] >= 0).all()
        assert (auto[:, :, 3, 1] == 0).all() and (auto[:, :, 3, 0] >= 0).all()
        del out


def test_large_n_streamed_depth(dev):
    """The benchmark's workload as a user runs it: 10 Large-N integrations
    (N=256 x 2 pols, F=1024, T=1000) streamed from pinned host memory through
    xc_correlate_stream (Algorithm 1 of Sec. 5, dump mode: one output per
    integration, each copied back to pinned host memory).  The operand ring
    wraps 34 times per integration.  Checked bit-exactly against the oracle:
    every channel of integration 0 and 64 seeded channels of each of
    integrations 1..9 (1600 channels, 1.7e12 useful ops on the host), and
    the device outputs equal the copies that came back."""
    w = synth.LARGE_N
    nint = 10
    host_in = torch.empty((nint,) + w.shape, dtype=torch.int8, pin_memory=True)
    for i in range(nint):
        host_in[i].copy_(synth.large_n_input(w, i, device=dev))
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8")
    try:
        out = eng.new_output(nint, device=dev)
        host_out = torch.empty((nint,) + w.out_shape, dtype=torch.int32, pin_memory=True)
        eng.correlate_stream(host_in, nint, out, host_out=host_out)
        eng.synchronize()
        for i in (0, nint - 1):
            assert torch.equal(out[i].cpu(), host_out[i])
    finally:
        eng.close()
    del out
    x0 = host_in[0].numpy()
    for c0 in range(0, w.nfreq, 128):
        want = oracle.correlate_i8(np.ascontiguousarray(x0[:, c0:c0 + 128]))
        got = host_out[0, c0:c0 + 128].numpy().astype(np.int64)
        assert np.array_equal(got, want), "integration 0, channels %d..%d" % (c0, c0 + 127)
    rng = np.random.default_rng(w.seed + 99)
    for i in range(1, nint):
        chans = sorted(rng.choice(w.nfreq, size=64, replace=False).tolist())
        want = oracle.correlate_i8(np.ascontiguousarray(host_in[i].numpy()[:, chans]))
        got = host_out[i].numpy()[chans].astype(np.int64)
        assert np.array_equal(got, want), "integration %d" % i


def frob_and_maxnorm(got, want, N, P):
    """Per-channel Frobenius relative error and max |dV_ab| / sqrt(V_aa V_bb)."""
    g = got[..., 0] + 1j * got[..., 1]
    w = want[..., 0] + 1j * want[..., 1]
    frob = np.sqrt((np.abs(g - w) ** 2).sum(axis=(1, 2)) / (np.abs(w) ** 2).sum(axis=(1, 2)))
    diag = [s * (s + 1) // 2 + s for s in range(N)]
    auto = np.stack([w[:, diag, p * P + p].real for p in range(P)], axis=-1)  # [F][N][P]
    s1, s2 = np.tril_indices(N)
    worst = 0.0
    for p1 in range(P):
        for p2 in range(P):
            den = np.sqrt(auto[:, s1, p1] * auto[:, s2, p2])
            worst = max(worst, float((np.abs(g - w)[:, :, p1 * P + p2] / den).max()))
    return float(frob.max()), worst


# Float shapes: n = N P = 140 takes the TMA-staged converter for both input
# types; n = 70 takes it only for fp32 (fp16 rows need n % 4 == 0); n = 37
# (P = 1) takes the direct-load converter for both.
@pytest.mark.parametrize("N,P", [(70, 2), (35, 2), (37, 1)], ids=["n140", "n70", "n37"])
@pytest.mark.parametrize("dtype", ["float32", "float16"])
@pytest.mark.parametrize("engine_name,engine,tile", ENGINES, ids=[e[0] for e in ENGINES])
def test_float_input_within_tolerance(dtype, engine_name, engine, tile, N, P, dev):
    T, F = 700, 3
    x = synth.sky_voltages(T, F, N, P, noise_sigma=0.7, nsrc=3, src_amp=1.0, seed=31)
    xt = x.to(torch.float16 if dtype == "float16" else torch.float32)
    want = oracle.correlate_f64(xt.to(torch.float64).numpy())
    got = run_engine(xt, engine, dev, dtype=dtype, tile=tile).numpy().astype(np.float64)
    frob, mx = frob_and_maxnorm(got, want, N, P)
    # fp16 operands (tensor path, unit round-off 2^-11) / fp32 accumulation
    assert frob <= 1e-3, frob
    assert mx <= 1e-3, mx


def test_bad_pointer_alignment(dev):
    eng = xc.Correlator(16, 2, 8, 256, "int8")
    try:
        x = torch.zeros(eng.in_shape, dtype=torch.int8, device=dev)
        out = eng.new_output(device=dev)
        st = xc.xc_correlate(eng.h, x.data_ptr() + 1, out.data_ptr(), 0)
        assert st == xc.XC_ERR_ALIGNMENT
        st = xc.xc_correlate(eng.h, x.data_ptr(), out.data_ptr() + 4, 0)
        assert st == xc.XC_ERR_ALIGNMENT
    finally:
        eng.close()


@pytest.mark.parametrize("dtype", ["int8", "float32"])
def test_repeat_runs_bitwise_identical(dtype, dev):
    """Races would show as run-to-run differences: the planar kernel's result
    is bitwise reproducible (fixed MMA order, one owner per output element)."""
    T, F, N, P = 300, 30, 96, 2  # more channels than ring slots
    if dtype == "int8":
        x = synth.uniform_int8((T, F, N, P, 2), -127, 127, 901)
    else:
        x = synth.sky_voltages(T, F, N, P, noise_sigma=1.0, nsrc=2, src_amp=1.0, seed=901)
    eng = xc.Correlator(N, P, F, T, dtype)
    try:
        xd = x.to(dev)
        outs = [eng.correlate(xd, sync=True).clone() for _ in range(3)]
    finally:
        eng.close()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
