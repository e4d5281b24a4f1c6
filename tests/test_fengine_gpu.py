"""GPU parity of the F-engine (Sec. 2): xc_channelize against the oracle's
DFT definition, through the C ABI.

Cases span every pass structure of the radix-16 kernel (log2 nchan = 4 .. 12:
radix-16 passes only, or with a radix-2/4/8 last pass), station counts below,
at and above the transforms one CTA holds (8192 / nchan), both polarisation
counts, every input type and both output types.  fp32 output must agree with
the FP64 oracle to 2e-6 (Frobenius, relative) and 1e-5 of the largest bin;
fp16 output to 1e-3 (its rounding is 2^-11 relative).  At the Large-N size
(N=256 x 2 pols, 1024 channels, 1000 blocks) sampled (block, channel)
outputs are checked one by one.  The FX chain (F-engine into the X-engine)
is checked against the oracle's F-engine followed by its X-engine.  Output
requantised to 8 bits must equal the oracle's requantisation except at
rounding boundaries (within 1e-3 of x.5), where the fp32 kernel may round
one code the other way; the 8-bit FX chain is then bit-exact on those codes.
The polyphase front end (random taps, 1 to 8 of them) is checked the same
way against the oracle's tap-weighted DFT."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc

pytestmark = pytest.mark.gpu

TORCH_DT = {"int8": torch.int8, "float16": torch.float16, "float32": torch.float32}


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def streams(N, P, L, dtype, seed):
    """Station-major complex streams [N][P][L][2]: uniform int8 in [-128, 127],
    or Gaussian float (sigma 3) rounded to the storage type."""
    if dtype == "int8":
        return synth.uniform_int8((N, P, L, 2), -128, 127, seed)
    g = torch.Generator().manual_seed(seed)
    return (3.0 * torch.randn((N, P, L, 2), generator=g)).to(TORCH_DT[dtype])


def rel_errors(got, want):
    d = got - want
    frob = np.linalg.norm(d) / np.linalg.norm(want)
    return frob, np.abs(d).max() / np.abs(want).max()


# (N, P, nchan, nblock, input type, output type)
CASES = [
    (3, 2, 16, 5, "int8", "float32"),
    (5, 1, 32, 3, "float32", "float32"),
    (70, 2, 64, 2, "float16", "float32"),
    (33, 2, 128, 2, "int8", "float16"),
    (17, 2, 256, 3, "float32", "float16"),
    (9, 2, 512, 2, "int8", "float32"),
    (9, 2, 1024, 2, "float32", "float32"),
    (3, 1, 2048, 2, "float16", "float16"),
    (4, 2, 4096, 2, "int8", "float32"),
    (1, 1, 2048, 3, "float32", "float32"),
]


@pytest.mark.parametrize("N,P,F,T,idt,odt", CASES,
                         ids=["N%d_P%d_F%d_T%d_%s_%s" % c for c in CASES])
def test_channelize_matches_oracle(N, P, F, T, idt, odt, dev):
    x = streams(N, P, T * F, idt, 70 + N + F)
    scale = 1.0 / np.sqrt(F)
    got = xc.channelize(x.to(dev), F, scale, odt).cpu().double().numpy()
    want = oracle.channelize_f64(x.double().numpy(), F, scale)
    frob, mx = rel_errors(got, want)
    print(f"\nF={F} {idt}->{odt}: frobenius {frob:.2e} max {mx:.2e}")
    if odt == "float32":
        assert frob <= 2e-6 and mx <= 1e-5, (frob, mx)
    else:
        assert frob <= 1e-3 and mx <= 1e-3, (frob, mx)


def test_channelize_tone_lands_in_one_bin(dev):
    N, P, F, T, k0 = 4, 2, 1024, 3, 37
    tau = torch.arange(T * F, dtype=torch.float64)
    ph = 2 * np.pi * k0 * tau / F
    amp = torch.arange(1, N * P + 1, dtype=torch.float64).reshape(N, P, 1)
    x = torch.stack([amp * torch.cos(ph), amp * torch.sin(ph)], dim=-1).float().contiguous()
    X = xc.channelize(x.to(dev), F, 1.0, "float32").cpu().double().numpy()
    mag = np.hypot(X[..., 0], X[..., 1])                       # [T][F][N][P]
    np.testing.assert_allclose(mag[:, k0], np.broadcast_to(F * amp.numpy()[None, :, :, 0], mag[:, k0].shape),
                               rtol=2e-6)
    others = np.delete(mag, k0, axis=1)
    assert others.max() < 1e-5 * mag[:, k0].max()


def test_channelize_large_n_sampled(dev):
    N, P, F, T = 256, 2, 1024, 1000
    x = synth.uniform_int8((N, P, T * F, 2), -128, 127, 71, device=dev)
    scale = 1.0 / np.sqrt(F)
    X = xc.channelize(x, F, scale, "float16")
    torch.cuda.synchronize()
    rng = np.random.default_rng(72)
    for t in (0, 517, T - 1):
        chans = sorted(set(rng.integers(0, F, 6).tolist()) | {0, F - 1})
        xt = x[:, :, t * F:(t + 1) * F].cpu().double().numpy()
        want = oracle.channelize_f64(xt, F, scale, sel=[(0, f) for f in chans])
        got = X[t, chans].cpu().double().numpy()
        frob, mx = rel_errors(got, want)
        assert frob <= 1e-3 and mx <= 1e-3, (t, frob, mx)


def test_fx_chain_matches_oracle(dev):
    """F-engine then X-engine on the GPU against the oracle's F-engine then
    its X-engine: sky-like streams (common sources plus noise per station)."""
    N, P, F, T = 24, 2, 64, 40
    g = torch.Generator().manual_seed(73)
    common = torch.randn((T * F, 2), generator=g)
    x = (torch.randn((N, P, T * F, 2), generator=g) + 0.5 * common).mul(4).round().clamp(-127, 127)
    x = x.to(torch.int8).contiguous()
    scale = 1.0 / np.sqrt(F)
    eng = xc.Correlator(N, P, F, T, "float16")
    try:
        X = xc.channelize(x.to(dev), F, scale, "float16")
        got = eng.correlate(X, sync=True).cpu().double().numpy()
    finally:
        eng.close()
    Xo = oracle.channelize_f64(x.double().numpy(), F, scale)
    want = oracle.correlate_f64(Xo)
    frob, _ = rel_errors(got, want)
    assert frob <= 2e-3, frob


def check_requantised(got, Xs, tol=1e-3):
    """Codes equal the oracle's requantisation of the exact values, except
    where an exact value lies within tol of a rounding boundary (x.5), where
    the fp32 kernel may round the other way by one."""
    want = oracle.requantise_i8(Xs)
    diff = got.astype(np.int64) - want.astype(np.int64)
    frac = np.abs(np.abs(Xs - np.floor(Xs)) - 0.5)
    bad = (diff != 0) & ~((np.abs(diff) == 1) & (frac < tol))
    assert not bad.any(), (int(bad.sum()), Xs[bad][:5], got[bad][:5], want[bad][:5])
    return int((diff != 0).sum())


# N*P a multiple of 8 takes the 16-byte store path; N*P = 5 and nchan = 4096
# (4 transforms per CTA) take the per-code stores.
@pytest.mark.parametrize("F,idt,N,P", [(256, "int8", 8, 2), (1024, "float32", 8, 2),
                                       (64, "float16", 8, 2), (128, "int8", 5, 1),
                                       (4096, "int8", 4, 2), (2048, "float32", 12, 2)],
                         ids=["F256_n16", "F1024_n16", "F64_n16", "F128_n5", "F4096_n8", "F2048_n24"])
def test_channelize_requantised_int8(F, idt, N, P, dev):
    T = 6
    x = streams(N, P, T * F, idt, 80 + F)
    scale = 0.5 / np.sqrt(F)  # output rms about 37 for int8 input: some components saturate
    if idt != "int8":
        scale *= 74.0 / 3.0
    got = xc.channelize(x.to(dev), F, scale, "int8").cpu().numpy()
    Xs = oracle.channelize_f64(x.double().numpy(), F, scale)
    flips = check_requantised(got, Xs)
    assert np.abs(Xs).max() > 127  # saturation exercised
    print(f"\nF={F} {idt}->int8: {flips} boundary flips of {got.size}")


def test_fx_chain_int8_is_exact_on_the_codes(dev):
    """F-engine requantised to 8 bits, then the exact 8-bit X-engine: the
    visibilities equal the oracle's X-engine on the same codes bit for bit,
    and the codes are the oracle's requantisation up to boundary flips."""
    N, P, F, T = 20, 2, 128, 30
    g = torch.Generator().manual_seed(81)
    common = torch.randn((T * F, 2), generator=g)
    x = (torch.randn((N, P, T * F, 2), generator=g) + 0.5 * common).mul(4).round().clamp(-127, 127)
    x = x.to(torch.int8).contiguous()
    scale = 2.0 / np.sqrt(F)
    eng = xc.Correlator(N, P, F, T, "int8")
    try:
        codes = xc.channelize(x.to(dev), F, scale, "int8")
        vis = eng.correlate(codes, sync=True).cpu().numpy()
    finally:
        eng.close()
    codes = codes.cpu().numpy()
    np.testing.assert_array_equal(vis, oracle.correlate_i8(codes))
    check_requantised(codes, oracle.channelize_f64(x.double().numpy(), F, scale))


# (N, P, nchan, input blocks, ntaps, input type, output type)
PFB_CASES = [
    (5, 2, 64, 9, 4, "int8", "float32"),
    (9, 2, 1024, 6, 3, "float32", "float32"),
    (33, 2, 256, 5, 1, "float16", "float16"),
    (8, 1, 2048, 4, 4, "float32", "float32"),
    (8, 2, 1024, 10, 8, "int8", "int8"),
]


@pytest.mark.parametrize("N,P,F,T,ntaps,idt,odt", PFB_CASES,
                         ids=["N%d_P%d_F%d_T%d_taps%d_%s_%s" % c for c in PFB_CASES])
def test_polyphase_matches_oracle(N, P, F, T, ntaps, idt, odt, dev):
    x = streams(N, P, T * F, idt, 90 + F + ntaps)
    g = torch.Generator().manual_seed(91 + ntaps)
    taps = torch.randn((ntaps, F), generator=g)
    sx = 74.0 if idt == "int8" else 3.0
    scale = 37.0 / (sx * np.sqrt(ntaps * F))  # output rms about 37
    got = xc.channelize(x.to(dev), F, scale, odt, taps=taps.to(dev)).cpu()
    want = oracle.channelize_pfb_f64(x.double().numpy(), taps.double().numpy(), scale)
    assert tuple(got.shape) == want.shape == (T - ntaps + 1, F, N, P, 2)
    if odt == "int8":
        check_requantised(got.numpy(), want)
        return
    frob, mx = rel_errors(got.double().numpy(), want)
    print(f"\npfb F={F} taps={ntaps} {idt}->{odt}: frobenius {frob:.2e} max {mx:.2e}")
    if odt == "float32":
        assert frob <= 2e-6 and mx <= 1e-5, (frob, mx)
    else:
        assert frob <= 1e-3 and mx <= 1e-3, (frob, mx)


def test_polyphase_argument_errors(dev):
    x = torch.zeros((2, 2, 64 * 4, 2), dtype=torch.int8, device=dev)
    taps = torch.ones((5, 64), device=dev)
    with pytest.raises(xc.XcError) as e:
        xc.channelize(x, 64, taps=taps)  # 5 taps over 4 blocks
    assert "XC_ERR_INVALID_ARG" in str(e.value)
    out = torch.empty((1, 64, 2, 2, 2), dtype=torch.float32, device=dev)
    assert xc.xc_channelize_pfb(x.data_ptr(), xc.XC_CI8, 2, 2, 64, 4, 0, 4, 1.0, out.data_ptr(),
                                xc.XC_CF32, 0) == xc.XC_ERR_INVALID_ARG


def test_channelize_argument_errors(dev):
    x = torch.zeros((2, 2, 96, 2), dtype=torch.int8, device=dev)
    with pytest.raises(xc.XcError) as e:
        xc.channelize(x, 48)  # not a power of two
    assert "XC_ERR_UNSUPPORTED" in str(e.value)
    out = torch.empty((1, 16 * 6 + 1), dtype=torch.float32, device=dev)
    st = xc.xc_channelize(x.data_ptr(), xc.XC_CI8, 2, 2, 16, 6, 1.0, out.data_ptr() + 4,
                          xc.XC_CF32, 0)
    assert st == xc.XC_ERR_ALIGNMENT
    assert xc.xc_channelize(x.data_ptr(), xc.XC_CI8, 0, 2, 16, 6, 1.0, out.data_ptr(),
                            xc.XC_CF32, 0) == xc.XC_ERR_INVALID_ARG
