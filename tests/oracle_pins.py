"""Pins that tie the CPU oracle to facts other than itself.

Each pin takes an oracle library handle (``oracle.load()`` or a deliberately
broken copy built by the mutation tests) and raises AssertionError when the
oracle disagrees with:

* brute force in numpy complex128 on tiny inputs (an independent evaluation
  of Eq. (outer) of Sec. 2.1 and of the lower-triangle packing);
* invariants the definition fixes: real non-negative autocorrelations equal
  to sum |x|^2, Hermitian symmetry of the diagonal baselines' cross-pol
  products, identical signals giving identical visibilities, the closed form
  of a scaled common signal, quadratic scaling, the cross-term expansion of
  a sum of signals;
* the statistical expectation for injected point sources (this fixes the
  conjugation convention: the phase of V_ab is phi_a - phi_b);
* the int32 range argument of the 8-bit path (Sec. 5 input, int64 oracle);
* central finite differences of the FP64 forward for the adjoint;
* for the F-engine (Sec. 2): numpy's FFT on random blocks (the library
  special case), the closed form of a pure tone, Parseval's identity, a
  delta's phase ramp in the corner-turned position, and the FX closed form of
  a tone shared by all stations.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1107_4264_gb300 import synth


def _cx(x: np.ndarray) -> np.ndarray:
    """[..., 2] real pairs -> complex128."""
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0] + 1j * x[..., 1]


def brute_force(x: np.ndarray, gains=None) -> np.ndarray:
    """Independent evaluation with numpy: V_f = Y_f^T conj(Y_f) over time,
    then the lower triangle of station pairs in row-major order."""
    T, F, N, P, _ = x.shape
    X = _cx(x).reshape(T, F, N * P)
    if gains is not None:
        X = X * _cx(gains).reshape(1, 1, N * P)
    V = np.einsum("tfa,tfb->fab", X, X.conj())
    rows, cols = np.tril_indices(N)
    out = np.zeros((F, len(rows), P * P, 2))
    for p1 in range(P):
        for p2 in range(P):
            v = V[:, rows * P + p1, cols * P + p2]
            out[:, :, p1 * P + p2, 0] = v.real
            out[:, :, p1 * P + p2, 1] = v.imag
    return out


def pin_brute_force_int(lib):
    rng = np.random.default_rng(11)
    for (T, F, N, P) in [(37, 3, 5, 2), (1, 1, 1, 1), (8, 2, 7, 1), (0, 2, 3, 2)]:
        x = rng.integers(-128, 128, (T, F, N, P, 2)).astype(np.int8)
        got = oracle.correlate_i8(x, lib=lib)
        want = brute_force(x)
        assert got.dtype == np.int64
        np.testing.assert_array_equal(got, np.rint(want).astype(np.int64))
    # channel subset selects channels
    x = rng.integers(-128, 128, (9, 4, 3, 2, 2)).astype(np.int8)
    np.testing.assert_array_equal(oracle.correlate_i8(x, chans=[3, 1], lib=lib),
                                  oracle.correlate_i8(x, lib=lib)[[3, 1]])


def pin_brute_force_float(lib):
    rng = np.random.default_rng(12)
    for (T, F, N, P) in [(23, 2, 4, 2), (5, 3, 3, 1)]:
        x = rng.standard_normal((T, F, N, P, 2))
        g = rng.standard_normal((N, P, 2))
        np.testing.assert_allclose(oracle.correlate_f64(x, lib=lib), brute_force(x),
                                   rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(oracle.correlate_f64(x, gains=g, lib=lib),
                                   brute_force(x, gains=g), rtol=1e-12, atol=1e-12)


def _diag_k(N):
    return [s * (s + 1) // 2 + s for s in range(N)]


def pin_autocorrelations(lib):
    x = synth.tiny_input(synth.TINY).numpy()
    T, F, N, P, _ = x.shape
    out = oracle.correlate_i8(x, lib=lib)
    xs = x.astype(np.int64)
    power = (xs[..., 0] ** 2 + xs[..., 1] ** 2).sum(axis=0)  # [F][N][P]
    for s, k in enumerate(_diag_k(N)):
        for p in range(P):
            v = out[:, k, p * P + p]
            assert (v[:, 1] == 0).all(), "autocorrelation must be real"
            assert (v[:, 0] >= 0).all()
            np.testing.assert_array_equal(v[:, 0], power[:, s, p])


def pin_hermitian_diagonal(lib):
    x = synth.tiny_input(synth.TINY).numpy()
    N, P = x.shape[2], x.shape[3]
    out = oracle.correlate_i8(x, lib=lib)
    for k in _diag_k(N):
        xy, yx = out[:, k, 0 * P + 1], out[:, k, 1 * P + 0]
        np.testing.assert_array_equal(xy[:, 0], yx[:, 0])
        np.testing.assert_array_equal(xy[:, 1], -yx[:, 1])


def pin_identical_signals(lib):
    rng = np.random.default_rng(13)
    T, F, N, P = 50, 2, 6, 2
    s = rng.integers(-100, 101, (T, F, 1, 1, 2)).astype(np.int8)
    x = np.broadcast_to(s, (T, F, N, P, 2)).copy()
    out = oracle.correlate_i8(x, lib=lib)
    pw = (s.astype(np.int64) ** 2).sum(axis=(0, 2, 3, 4))  # [F]
    for f in range(F):
        assert (out[f, :, :, 0] == pw[f]).all()
        assert (out[f, :, :, 1] == 0).all()


def pin_closed_form(lib):
    """x_a(t) = c_a s(t) with integer complex c_a: V_ab = c_a conj(c_b) sum|s|^2."""
    rng = np.random.default_rng(14)
    T, F, N, P = 40, 3, 5, 2
    s = rng.integers(-5, 6, (T, F, 2))
    c = rng.integers(-4, 5, (N, P, 2))
    x = np.zeros((T, F, N, P, 2), dtype=np.int64)
    x[..., 0] = s[:, :, None, None, 0] * c[None, None, :, :, 0] - s[:, :, None, None, 1] * c[None, None, :, :, 1]
    x[..., 1] = s[:, :, None, None, 0] * c[None, None, :, :, 1] + s[:, :, None, None, 1] * c[None, None, :, :, 0]
    out = oracle.correlate_i8(x.astype(np.int8), lib=lib)
    S = (s ** 2).sum(axis=(0, 2))  # [F]
    for s1 in range(N):
        for s2 in range(s1 + 1):
            k = s1 * (s1 + 1) // 2 + s2
            for p1 in range(P):
                for p2 in range(P):
                    ar, ai = c[s1, p1]
                    br, bi = c[s2, p2]
                    re = ar * br + ai * bi  # c_a conj(c_b)
                    im = ai * br - ar * bi
                    np.testing.assert_array_equal(out[:, k, p1 * P + p2, 0], re * S)
                    np.testing.assert_array_equal(out[:, k, p1 * P + p2, 1], im * S)


def pin_scaling_and_cross_terms(lib):
    rng = np.random.default_rng(15)
    T, F, N, P = 30, 2, 4, 2
    x = rng.integers(-20, 21, (T, F, N, P, 2))
    y = rng.integers(-20, 21, (T, F, N, P, 2))
    Vx = oracle.correlate_i8(x.astype(np.int8), lib=lib)
    # V(alpha x) = |alpha|^2 V(x), alpha = 2 - 3i
    ax = np.empty_like(x)
    ax[..., 0] = 2 * x[..., 0] + 3 * x[..., 1]
    ax[..., 1] = 2 * x[..., 1] - 3 * x[..., 0]
    np.testing.assert_array_equal(oracle.correlate_i8(ax.astype(np.int8), lib=lib), 13 * Vx)
    # V(x + y) = V(x) + V(y) + [x y^H + y x^H] (cross terms by numpy)
    Vy = oracle.correlate_i8(y.astype(np.int8), lib=lib)
    Vxy = oracle.correlate_i8((x + y).astype(np.int8), lib=lib)
    X, Y = _cx(x).reshape(T, F, N * P), _cx(y).reshape(T, F, N * P)
    C = np.einsum("tfa,tfb->fab", X, Y.conj()) + np.einsum("tfa,tfb->fab", Y, X.conj())
    rows, cols = np.tril_indices(N)
    for p1 in range(P):
        for p2 in range(P):
            cv = C[:, rows * P + p1, cols * P + p2]
            d = Vxy[:, :, p1 * P + p2] - Vx[:, :, p1 * P + p2] - Vy[:, :, p1 * P + p2]
            np.testing.assert_array_equal(d[..., 0], np.rint(cv.real).astype(np.int64))
            np.testing.assert_array_equal(d[..., 1], np.rint(cv.imag).astype(np.int64))


def pin_point_source_statistics(lib):
    """E[V_ab^{pq}]/T = delta_pq [sigma_c^2 delta_ab + sum_k A^2 e^{i(phi_ka - phi_kb)}]."""
    T, F, N, P, K, A, sig = 20000, 2, 4, 2, 2, 1.0, 0.5
    seed = 4242
    x = synth.sky_voltages(T, F, N, P, noise_sigma=sig, nsrc=K, src_amp=A, seed=seed,
                           dtype=torch_float64()).numpy()
    out = oracle.correlate_f64(x, lib=lib) / T
    phi = synth.steering_phases(N, F, K, seed)  # [K][F][N]
    noise_pow = 2 * sig ** 2
    for f in range(F):
        for s1 in range(N):
            for s2 in range(s1 + 1):
                k = s1 * (s1 + 1) // 2 + s2
                for p1 in range(P):
                    for p2 in range(P):
                        e = 0j
                        if p1 == p2:
                            e = (noise_pow if s1 == s2 else 0.0) + A ** 2 * np.exp(
                                1j * (phi[:, f, s1] - phi[:, f, s2])).sum()
                        got = complex(*out[f, k, p1 * P + p2])
                        # per-sample power <= noise + K A^2; std of the mean ~ power/sqrt(T)
                        tol = 6.0 * (noise_pow + K * A ** 2) / np.sqrt(T)
                        assert abs(got - e) < tol, (f, s1, s2, p1, p2, got, e)


def torch_float64():
    import torch
    return torch.float64


INT32_MAX = 2 ** 31 - 1
T_MAX_FULL_RANGE = 66572  # largest T with T * 2 * 127^2 < 2^31


def pin_int32_bound(lib):
    for T, fits in [(T_MAX_FULL_RANGE, True), (T_MAX_FULL_RANGE + 1, False)]:
        x = np.full((T, 1, 1, 1, 2), 127, dtype=np.int8)
        out = oracle.correlate_i8(x, lib=lib)
        assert out[0, 0, 0, 0] == T * 2 * 127 * 127
        assert (out[0, 0, 0, 0] <= INT32_MAX) == fits


def _loss_and_grad_out(V, M, W):
    d = V - M
    L = float((W[..., None] * d * d).sum())
    return L, 2.0 * W[..., None] * d


def pin_adjoint_finite_differences(lib):
    rng = np.random.default_rng(16)
    T, F, N, P = 5, 2, 3, 2
    x = rng.standard_normal((T, F, N, P, 2))
    g = rng.standard_normal((N, P, 2))
    M = rng.standard_normal((F, N * (N + 1) // 2, P * P, 2))
    W = rng.uniform(0, 1, (F, N * (N + 1) // 2, P * P))

    def loss(xx, gg):
        V = oracle.correlate_f64(xx, gains=gg, lib=lib)
        return _loss_and_grad_out(V, M, W)[0]

    V = oracle.correlate_f64(x, gains=g, lib=lib)
    _, go = _loss_and_grad_out(V, M, W)
    gx, gg = oracle.backward_f64(x, go, gains=g, lib=lib)
    h = 1e-5
    idx = [tuple(rng.integers(0, s) for s in x.shape) for _ in range(24)]
    for i in idx:
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (loss(xp, g) - loss(xm, g)) / (2 * h)
        assert abs(fd - gx[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gx[i])
    for i in np.ndindex(g.shape):
        gp, gm = g.copy(), g.copy()
        gp[i] += h
        gm[i] -= h
        fd = (loss(x, gp) - loss(x, gm)) / (2 * h)
        assert abs(fd - gg[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gg[i])


def _fx(x):
    """[N][P][L][2] complex streams -> complex128 [N][P][L]."""
    return _cx(x)


def pin_fengine_numpy_fft(lib):
    """Random blocks, several channel counts (not only powers of two):
    X[t][f][s][p] = scale * fft(x[s][p][t F : (t + 1) F])[f]."""
    rng = np.random.default_rng(31)
    for N, P, F, T in ((2, 2, 16, 3), (3, 1, 12, 2), (1, 2, 64, 2), (2, 2, 5, 4)):
        x = rng.standard_normal((N, P, T * F, 2))
        got = _cx(oracle.channelize_f64(x, F, 0.75, lib=lib))
        ref = np.fft.fft(_fx(x).reshape(N, P, T, F), axis=-1) * 0.75
        np.testing.assert_allclose(got, np.transpose(ref, (2, 3, 0, 1)), rtol=0, atol=1e-11)


def pin_fengine_tone(lib):
    """x(tau) = A_sp exp(2 pi i k0 tau / F): every block gives scale * F * A_sp
    in channel k0 and nothing elsewhere."""
    rng = np.random.default_rng(32)
    N, P, F, T, k0, scale = 3, 2, 32, 3, 5, 0.5
    A = rng.standard_normal((N, P)) + 1j * rng.standard_normal((N, P))
    tau = np.arange(T * F)
    z = A[:, :, None] * np.exp(2j * np.pi * k0 * tau / F)[None, None, :]
    x = np.stack([z.real, z.imag], axis=-1)
    got = _cx(oracle.channelize_f64(x, F, scale, lib=lib))
    want = np.zeros((T, F, N, P), dtype=np.complex128)
    want[:, k0] = scale * F * A[None]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def pin_fengine_parseval(lib):
    """sum_f |X_t(f)|^2 = F sum_m |x(t F + m)|^2 for each block, station, pol."""
    rng = np.random.default_rng(33)
    N, P, F, T = 2, 2, 24, 3
    x = rng.standard_normal((N, P, T * F, 2))
    X = _cx(oracle.channelize_f64(x, F, 1.0, lib=lib))          # [T][F][N][P]
    e_out = (np.abs(X) ** 2).sum(axis=1)                           # [T][N][P]
    e_in = (np.abs(_fx(x).reshape(N, P, T, F)) ** 2).sum(axis=-1)  # [N][P][T]
    np.testing.assert_allclose(e_out, F * np.transpose(e_in, (2, 0, 1)), rtol=1e-12)


def pin_fengine_delta_layout(lib):
    """A unit sample at (s0, p0, tau0) lands in block tau0 // F of station s0,
    pol p0 only, as the phase ramp scale * exp(-2 pi i f (tau0 mod F) / F)."""
    N, P, F, T, scale = 3, 2, 16, 4, 2.0
    s0, p0, tau0 = 2, 1, 2 * 16 + 7
    x = np.zeros((N, P, T * F, 2))
    x[s0, p0, tau0, 0] = 1.0
    got = _cx(oracle.channelize_f64(x, F, scale, lib=lib))
    want = np.zeros((T, F, N, P), dtype=np.complex128)
    want[tau0 // F, :, s0, p0] = scale * np.exp(-2j * np.pi * np.arange(F) * (tau0 % F) / F)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def pin_fengine_fx_tone(lib):
    """FX: stations seeing one tone A_a exp(2 pi i k0 tau / F) give, after the
    F-engine and the X-engine, V_ab = T (scale F)^2 A_a conj(A_b) in channel k0
    and zero in every other channel."""
    rng = np.random.default_rng(34)
    N, P, F, T, k0, scale = 3, 2, 16, 5, 3, 0.25
    A = rng.standard_normal((N, P)) + 1j * rng.standard_normal((N, P))
    tau = np.arange(T * F)
    z = A[:, :, None] * np.exp(2j * np.pi * k0 * tau / F)[None, None, :]
    X = oracle.channelize_f64(np.stack([z.real, z.imag], axis=-1), F, scale, lib=lib)
    V = _cx(oracle.correlate_f64(X, lib=lib))                     # [F][NB][P*P]
    for s1 in range(N):
        for s2 in range(s1 + 1):
            k = s1 * (s1 + 1) // 2 + s2
            for p1 in range(P):
                for p2 in range(P):
                    want = T * (scale * F) ** 2 * A[s1, p1] * np.conj(A[s2, p2])
                    np.testing.assert_allclose(V[k0, k, p1 * P + p2], want, rtol=1e-9)
    mask = np.ones(F, dtype=bool)
    mask[k0] = False
    assert np.abs(V[mask]).max() < 1e-8 * np.abs(V[k0]).max()


def pin_requantise_truth_table(lib):
    """8-bit requantisation: nearest integer with ties to even, saturated at
    +-127 (both signs), on hand-picked values."""
    x = np.array([-0.5, 0.5, 1.5, 2.5, -1.5, 126.5, 127.49, 127.5, 200.0, -127.5, -128.0, -300.0,
                  3.2, -3.7])
    want = np.array([0, 0, 2, 2, -2, 126, 127, 127, 127, -127, -127, -127, 3, -4], dtype=np.int8)
    got = oracle.requantise_i8(x)
    assert got.dtype == np.int8
    np.testing.assert_array_equal(got, want)


def pin_pfb_single_unit_tap_is_dft(lib):
    """One tap of ones: the polyphase F-engine is the plain blockwise DFT."""
    rng = np.random.default_rng(35)
    N, P, F, T = 2, 2, 16, 3
    x = rng.standard_normal((N, P, T * F, 2))
    got = oracle.channelize_pfb_f64(x, np.ones((1, F)), 0.5, lib=lib)
    ref = np.fft.fft(_fx(x).reshape(N, P, T, F), axis=-1) * 0.5
    np.testing.assert_allclose(_cx(got), np.transpose(ref, (2, 3, 0, 1)), rtol=0, atol=1e-11)


def pin_pfb_delta_taps(lib):
    """A unit sample at tau0 = b0 F + m0 reaches output block t = b0 - p through
    tap p only: X_t(f) = scale h[p][m0] exp(-2 pi i f m0 / F), every other
    block, station and pol zero."""
    rng = np.random.default_rng(36)
    N, P, F, T, ntaps, scale = 2, 2, 8, 6, 3, 1.5
    h = rng.standard_normal((ntaps, F))
    s0, p0, b0, m0 = 1, 0, 3, 5
    x = np.zeros((N, P, T * F, 2))
    x[s0, p0, b0 * F + m0, 0] = 1.0
    got = _cx(oracle.channelize_pfb_f64(x, h, scale, lib=lib))  # [T-ntaps+1][F][N][P]
    want = np.zeros_like(got)
    ramp = np.exp(-2j * np.pi * np.arange(F) * m0 / F)
    for p in range(ntaps):
        t = b0 - p
        if 0 <= t < T - ntaps + 1:
            want[t, :, s0, p0] = scale * h[p, m0] * ramp
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def pin_pfb_tone_response(lib):
    """A bin-centred tone exp(2 pi i k0 tau / F) through taps h gives, in every
    output block, scale * DFT(H)[f - k0] with H[m] = sum_p h[p][m] (numpy FFT)."""
    rng = np.random.default_rng(37)
    N, P, F, T, ntaps, k0, scale = 1, 2, 32, 7, 4, 9, 0.25
    h = rng.standard_normal((ntaps, F))
    tau = np.arange(T * F)
    z = np.broadcast_to(np.exp(2j * np.pi * k0 * tau / F), (N, P, T * F))
    x = np.stack([z.real, z.imag], axis=-1)
    got = _cx(oracle.channelize_pfb_f64(x, h, scale, lib=lib))
    Hf = np.fft.fft(h.sum(axis=0))
    want = scale * Hf[(np.arange(F) - k0) % F]
    np.testing.assert_allclose(got, np.broadcast_to(want[None, :, None, None], got.shape),
                               rtol=0, atol=1e-10)


ALL_PINS = [
    pin_brute_force_int,
    pin_brute_force_float,
    pin_autocorrelations,
    pin_hermitian_diagonal,
    pin_identical_signals,
    pin_closed_form,
    pin_scaling_and_cross_terms,
    pin_point_source_statistics,
    pin_int32_bound,
    pin_adjoint_finite_differences,
    pin_fengine_numpy_fft,
    pin_fengine_tone,
    pin_fengine_parseval,
    pin_fengine_delta_layout,
    pin_fengine_fx_tone,
    pin_requantise_truth_table,
    pin_pfb_single_unit_tap_is_dft,
    pin_pfb_delta_taps,
    pin_pfb_tone_response,
]
