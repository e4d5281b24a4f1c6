"""Seeded synthetic station voltages for the X-engine.

This module only draws inputs; it contains none of the correlator's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper measures on no dataset: its workloads are sized by station count N,
channel count F and integration length I (Sec. 6), with 8-bit samples
(Sec. 5).  The generators here stand in for "Large-N" array data
(MWA-like): a station layout drawn uniformly in a 1.5 km-radius disk,
channel frequencies spread linearly over 100-200 MHz, and unpolarised point
sources within 10 degrees of zenith whose per-station geometric phase is
exp(i 2 pi b_s . s_k / lambda_f), on top of independent receiver noise.

Layout of every voltage tensor: ``[T][F][N][P][2]`` = (time, channel,
station, polarisation, re/im), station fastest after the complex pair, as in
the corner-turned ordering of Sec. 4.1.

Random streams: small host-side parameters (geometry, source directions,
gains) come from ``numpy.random.Generator(PCG64(seed))``; bulk samples come
from a ``torch.Generator`` on the requested device seeded with the same seed,
so large workloads can be drawn directly in device memory.  A given
(seed, device) pair always gives the same tensor.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

SEED_BASE = 1107
C_LIGHT = 299_792_458.0


def _np_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _torch_gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def station_positions(nstation: int, seed: int, radius_m: float = 1500.0) -> np.ndarray:
    """East/north station coordinates (metres), uniform in a disk."""
    rng = _np_rng(seed)
    r = radius_m * np.sqrt(rng.uniform(0.0, 1.0, nstation))
    th = rng.uniform(0.0, 2.0 * np.pi, nstation)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def channel_wavelengths(nfreq: int, f_lo: float = 100e6, f_hi: float = 200e6) -> np.ndarray:
    """Wavelength (metres) of each channel, frequencies linear over [f_lo, f_hi]."""
    if nfreq == 1:
        nu = np.array([0.5 * (f_lo + f_hi)])
    else:
        nu = np.linspace(f_lo, f_hi, nfreq)
    return C_LIGHT / nu


def source_directions(nsrc: int, seed: int, max_zenith_deg: float = 10.0) -> np.ndarray:
    """Direction cosines (l, m) of point sources within max_zenith_deg of zenith."""
    rng = _np_rng(seed + 7919)
    za = np.deg2rad(max_zenith_deg) * np.sqrt(rng.uniform(0.0, 1.0, nsrc))
    az = rng.uniform(0.0, 2.0 * np.pi, nsrc)
    return np.stack([np.sin(za) * np.cos(az), np.sin(za) * np.sin(az)], axis=1)


def steering_phases(nstation: int, nfreq: int, nsrc: int, seed: int) -> np.ndarray:
    """Geometric phase phi[k][f][s] = 2 pi b_s . (l_k, m_k) / lambda_f."""
    b = station_positions(nstation, seed)
    lam = channel_wavelengths(nfreq)
    lm = source_directions(nsrc, seed)
    proj = lm @ b.T  # [K][N] metres
    return 2.0 * np.pi * proj[:, None, :] / lam[None, :, None]


def complex_gains(nstation: int, npol: int, seed: int, amp_lo: float = 0.5,
                  amp_hi: float = 2.0) -> np.ndarray:
    """Per-(station, pol) complex gains, |g| ~ U[amp_lo, amp_hi], arg ~ U[0, 2 pi).
    Returned as float64 ``[N][P][2]``."""
    rng = _np_rng(seed + 104729)
    amp = rng.uniform(amp_lo, amp_hi, (nstation, npol))
    ph = rng.uniform(0.0, 2.0 * np.pi, (nstation, npol))
    return np.stack([amp * np.cos(ph), amp * np.sin(ph)], axis=-1)


def sky_voltages(T: int, F: int, N: int, P: int, *, noise_sigma: float, nsrc: int,
                 src_amp: float, seed: int, device="cpu", t_chunk: int = 0,
                 out: Optional[torch.Tensor] = None, quantise_int8: bool = False,
                 dtype: torch.dtype = torch.float32) -> torch.Tensor:
    """Noise plus point sources, shape ``[T][F][N][P][2]``.

    noise: re and im each N(0, noise_sigma^2), independent per sample.
    source k: src_amp * s_k(t, f, p) * exp(i phi[k][f][s]) with s_k a unit
    complex Gaussian (re, im ~ N(0, 1/2)), independent per polarisation
    (unpolarised).  With ``quantise_int8`` the sum is rounded to the nearest
    integer and clipped to [-127, 127].
    Generated in time chunks so device memory stays bounded.
    """
    dev = torch.device(device)
    gen = _torch_gen(seed, dev)
    if out is None:
        out = torch.empty((T, F, N, P, 2), dtype=torch.int8 if quantise_int8 else dtype, device=dev)
    phi = torch.from_numpy(steering_phases(N, F, max(nsrc, 0), seed)).to(dev, torch.float32)
    steer = torch.polar(torch.ones_like(phi), phi) if nsrc > 0 else None  # [K][F][N] complex64
    if t_chunk <= 0:
        per_t = F * N * P * 2 * 4 * 3
        t_chunk = max(1, min(T, (256 << 20) // max(per_t, 1)))
    for t0 in range(0, T, t_chunk):
        tc = min(t_chunk, T - t0)
        v = torch.randn((tc, F, N, P, 2), generator=gen, device=dev, dtype=torch.float32)
        v.mul_(noise_sigma)
        if nsrc > 0:
            s = torch.randn((tc, F, nsrc, P, 2), generator=gen, device=dev, dtype=torch.float32)
            s = torch.view_as_complex(s.mul_(math.sqrt(0.5) * src_amp).contiguous())
            add = torch.einsum("tfkp,kfs->tfsp", s, steer)
            v += torch.view_as_real(add.contiguous())
        if quantise_int8:
            out[t0:t0 + tc] = v.round_().clamp_(-127, 127).to(torch.int8)
        else:
            out[t0:t0 + tc] = v.to(out.dtype)
    return out


# ---------------------------------------------------------------- workloads


@dataclass(frozen=True)
class Workload:
    name: str
    nstation: int
    npol: int
    nfreq: int
    ntime: int
    seed: int

    @property
    def shape(self) -> Tuple[int, int, int, int, int]:
        return (self.ntime, self.nfreq, self.nstation, self.npol, 2)

    @property
    def nbaseline(self) -> int:
        return self.nstation * (self.nstation + 1) // 2

    @property
    def out_shape(self) -> Tuple[int, int, int, int]:
        return (self.nfreq, self.nbaseline, self.npol * self.npol, 2)

    @property
    def useful_ops(self) -> int:
        """8 real ops per complex MAC, one CMAC per stored (baseline, pol
        product) per sample (Sec. 2.1, Eq. flops convention applied to the
        stored products)."""
        return 8 * self.nfreq * self.ntime * self.npol * self.npol * self.nbaseline


TINY = Workload("tiny int8 N=16 P=2 F=8 T=256", 16, 2, 8, 256, SEED_BASE + 0)
LARGE_N = Workload("large-N int8 N=256 P=2 F=1024 T=1000 x10 integrations", 256, 2, 1024, 1000,
                   SEED_BASE + 1)
LARGE_N_INTEGRATIONS = 10
PRECISION = Workload("precision float N=512 P=2 F=480 T=2048", 512, 2, 480, 2048, SEED_BASE + 2)
BATCHED = [Workload("batched sub%d" % i, n, 2, f, t, SEED_BASE + 3 + 100 * i) for i, (n, f, t) in
           enumerate(zip((32, 64, 128, 200, 384, 1024), (64, 128, 256, 256, 512, 96),
                         (256, 1024, 4096, 512, 2048, 8192)))]
DIFF = Workload("differentiable float N=256 P=2 F=64 T=4096", 256, 2, 64, 4096, SEED_BASE + 4)


def uniform_int8(shape: Sequence[int], lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """Independent uniform integers in [lo, hi] as int8."""
    gen = _torch_gen(seed, device)
    return torch.randint(lo, hi + 1, tuple(shape), generator=gen, device=torch.device(device),
                         dtype=torch.int16).to(torch.int8)


def tiny_input(w: Workload = TINY, device="cpu", lo: int = -7, hi: int = 7) -> torch.Tensor:
    """Tiny workload: re, im uniform integers in [-7, 7]."""
    return uniform_int8(w.shape, lo, hi, w.seed, device)


def large_n_input(w: Workload = LARGE_N, integration: int = 0, device="cpu",
                  out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Large-N int8 workload, one integration: N(0, 3^2) per component plus 3
    sources of amplitude 0.5 sigma, rounded and clipped to +-127."""
    return sky_voltages(w.ntime, w.nfreq, w.nstation, w.npol, noise_sigma=3.0, nsrc=3,
                        src_amp=1.5, seed=w.seed + 1000 * integration, device=device, out=out,
                        quantise_int8=True)


def int8_sky(w: Workload, device="cpu", integration: int = 0) -> torch.Tensor:
    """Generic int8 sky at the Large-N recipe (sigma 3, 3 sources)."""
    return large_n_input(w, integration, device)


def precision_input(w: Workload = PRECISION, device="cpu"):
    """Float voltages: complex Gaussian with unit variance per complex sample
    (re, im ~ N(0, 1/2)) plus 5 sources; returns (x, gains) where the gains
    [N][P][2] (|g| in [0.5, 2]) are applied by the engine."""
    x = sky_voltages(w.ntime, w.nfreq, w.nstation, w.npol, noise_sigma=math.sqrt(0.5), nsrc=5,
                     src_amp=1.0, seed=w.seed, device=device)
    return x, complex_gains(w.nstation, w.npol, w.seed)


def diff_inputs(w: Workload = DIFF, device="cpu"):
    """Differentiable workload: (x, gains, target_gains, weights).

    x: FP32 Gaussian voltages plus 4 sources; gains: learnable start point;
    target_gains: the second seeded gain set (seed + 1000) that generates the
    target visibilities; weights W ~ U[0, 1] over the output layout."""
    x = sky_voltages(w.ntime, w.nfreq, w.nstation, w.npol, noise_sigma=math.sqrt(0.5), nsrc=4,
                     src_amp=1.0, seed=w.seed, device=device)
    g = complex_gains(w.nstation, w.npol, w.seed)
    g_t = complex_gains(w.nstation, w.npol, w.seed + 1000)
    gen = _torch_gen(w.seed + 77, device)
    W = torch.rand(w.out_shape[:3], generator=gen, device=torch.device(device),
                   dtype=torch.float32)
    return x, g, g_t, W


def workload_by_name(name: str) -> Workload:
    table = {"tiny": TINY, "large_n": LARGE_N, "precision": PRECISION, "diff": DIFF}
    return table[name]


def batched_inputs(device="cpu", subs: Optional[List[Workload]] = None) -> List[torch.Tensor]:
    return [int8_sky(w, device) for w in (subs or BATCHED)]
