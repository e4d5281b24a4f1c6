#!/usr/bin/env python
"""X-engine benchmark: Large-N 8-bit workload on GB300.

Workload (one step): 10 integrations of N=256 dual-polarisation stations,
F=1024 channels, T=1000 samples per integration, complex int8 input
[T][F][N][P][2] (noise sigma 3 plus 3 point sources, rounded and clipped),
int32 visibilities of the N(N+1)/2 baselines x 4 polarisation products.

Metric: X-engine TOPS at 8 real ops per complex multiply-accumulate, one CMAC
per stored (baseline, polarisation product) per sample (the Eq. flops
convention of Sec. 2.1 applied to the stored products), with the tensor-core
fraction of peak and the speedup over the plain FP32 CUDA-core form of the
same X-engine on the same GPU.

  value   device-resident inputs (HBM), timed with CUDA events over K steps.
  e2e     the same work through xc_correlate_stream: inputs in pinned host
          memory, H2D copies overlapped with compute (Algorithm 1 of Sec. 5)
          and every visibility copied back to pinned host memory.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xc|reference]
Under torchrun (N > 1) every rank correlates its own 10 integrations (weak
scaling, no data-path collective; barrier and max-over-ranks timing only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "X-engine TOPS (8 ops/CMAC) & % tensor peak vs plain FP32 CUDA-core X-engine"
UNIT = "TOPS"
N_INTEGRATIONS = 10
PROFILE_DIR = os.path.join(ROOT, "profiles")
TRAFFIC_FILE = os.path.join(PROFILE_DIR, "traffic.json")
MAIN_KERNEL_SOURCES = ["paper_1107_4264_gb300/csrc/xc_planar.cu", "paper_1107_4264_gb300/csrc/xc_planar_kernel.cuh",
                       "paper_1107_4264_gb300/csrc/xc_ptx.cuh"]
# Channels of one Large-N integration that the CPU oracle is timed on, in the
# cpu_baseline leg and in every step of the reference arm alike (64 channels:
# 64 MB of 8-bit input, 6.9e10 useful ops).
CPU_SAMPLE_CHANNELS = 64


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["xc", "reference"], default="xc")
    ap.add_argument("--comparator-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-channels", type=int, default=0,
                    help="channels of one integration in the CPU oracle's sample, for cpu_baseline and "
                         "every reference step alike (default %d)" % CPU_SAMPLE_CHANNELS)
    ap.add_argument("--nfreq", type=int, default=0,
                    help="channels per integration (default 1024; smaller only for profiling captures)")
    ap.add_argument("--integrations", type=int, default=N_INTEGRATIONS,
                    help="integrations per step (default 10)")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip measuring the fp16 / fp8 / FP32 / H2D peaks in this run")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision, batched and differentiable workloads")
    ap.add_argument("--form-steps", type=int, default=5)
    ap.add_argument("--fengine", action="store_true",
                    help="instead of the bench line: the F-engine alone at the Large-N shape "
                         "(N=256 x 2 pols, 1024 channels), fp16, fp32 and 8-bit output, one JSON object")
    ap.add_argument("--fengine-blocks", type=int, default=1000,
                    help="blocks (samples per stream / 1024) for --fengine (smaller for profiling)")
    ap.add_argument("--tile", choices=["auto", "128", "pair", "wide"], default="auto",
                    help="tile shape of the tensor-core engine (default: the library's choice)")
    ap.add_argument("--smalln", type=int, default=0,
                    help="time the small-array engine and the packed planar engine at this N "
                         "(P=2, T=1000, F from --nfreq or the N sweep's choice) and exit")
    ap.add_argument("--fp8-4bit", action="store_true",
                    help="time the Large-N geometry with samples clipped to +-7 on the FP8 path "
                         "(F from --nfreq) and exit")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the bench line: kernel TOPS over N (fixed work) and over T at "
                         "fixed F*T (output traffic), one JSON object")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def planar_pack(N, P, F):
    """Channels the planar engine packs into one virtual channel (asked of the
    library: the largest divisor k of F with k N P <= 128 when N P <= 64)."""
    from paper_1107_4264_gb300 import xc
    return xc.load().xc_channels_packed(N, P, F)


def executed_ops(N, P, F, T, steps_per_block=1):
    """Real operations the planar engine's MMAs execute: for every lower
    128 x 128 block of the (virtual, packed) channel, 128 rows times the
    block's columns trimmed to a multiple of 16, over T padded to 64."""
    n = N * P
    k = planar_pack(N, P, F)
    nv, fv = k * n, F // k
    nb = (nv + 127) // 128
    macs = 0
    for by in range(nb):
        for bx in range(by + 1):
            macs += 128 * ((min(128, nv - 128 * bx) + 15) // 16 * 16)
    return 8 * macs * ((T + 63) // 64 * 64) * fv * steps_per_block


def small_executed_ops(N, P, F, T):
    """Real operations the small-array engine's MMAs execute: per channel
    group (m = 128 / W channels, or one channel of two tiles at W = 2 N P =
    256) and sample, one 128 x 128 MMA step (three at W = 256: the lower tile
    blocks), over T padded to 64."""
    from paper_1107_4264_gb300 import xc
    m = xc.load().xc_small_engine_channels(N, P)
    blocks = 3 if 2 * N * P == 256 else 1
    return 2 * 128 * 128 * blocks * ((T + 63) // 64 * 64) * ((F + m - 1) // m)


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it still
    describes the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != source_sha(MAIN_KERNEL_SOURCES):
        return None
    return e.get("bytes_per_launch")


def measure_peaks(torch, xc, dev, stream, sustained_s=4.0):
    """Dense tensor peaks (torch fp16 matmul and torch._scaled_mm e4m3,
    8192^3, best of 10 and back to back for a few seconds), the FP32
    CUDA-core peak (the library's FFMA probe) and the pinned host-to-device
    copy rate, measured in this run on this GPU.  Missing pieces are reported
    as unavailable."""
    res = {}

    def ev_time(fn, reps):
        best, tot = 1e30, 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best, tot = min(best, t), tot + t
        return best, tot / reps

    def gemm_peak(fn, flops):
        for _ in range(3):
            fn()
        best, _ = ev_time(fn, 10)
        t0 = time.perf_counter()
        n, e0 = 0, torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        while time.perf_counter() - t0 < sustained_s:
            for _ in range(20):
                fn()
            n += 20
            e1.record(stream)
            e1.synchronize()
        sus = e0.elapsed_time(e1) / n
        return {"burst": flops / (best * 1e-3) / 1e12, "sustained": flops / (sus * 1e-3) / 1e12,
                "sustained_s": round(time.perf_counter() - t0, 2)}

    n = 8192
    flops = 2.0 * n ** 3

    def fp16():
        a = torch.randn(n, n, device=dev, dtype=torch.float16)
        b = torch.randn(n, n, device=dev, dtype=torch.float16)
        c = torch.empty(n, n, device=dev, dtype=torch.float16)
        r = gemm_peak(lambda: torch.matmul(a, b, out=c), flops)
        r["how"] = "torch.matmul fp16 8192^3"
        return r

    def fp8():
        a8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        one = torch.ones((), device=dev, dtype=torch.float32)
        r = gemm_peak(lambda: torch._scaled_mm(a8, b8.t(), one, one, out_dtype=torch.bfloat16), flops)
        r["how"] = "torch._scaled_mm e4m3 x e4m3 -> bf16, 8192^3"
        return r

    with torch.cuda.stream(stream):
        for key, fn in (("fp16_dense_tflops", fp16), ("fp8_e4m3_dense_tflops", fp8)):
            try:
                res[key] = fn()
            except Exception as e:  # noqa: BLE001
                res[key] = {"unavailable": str(e)[:200]}
            torch.cuda.empty_cache()
        try:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            sink = torch.zeros(4 * sms, device=dev)
            s_ptr = stream.cuda_stream
            fl = xc.xc_fp32_peak_probe(20000, sink.data_ptr(), s_ptr)
            best, _ = ev_time(lambda: xc.xc_fp32_peak_probe(20000, sink.data_ptr(), s_ptr), 5)
            sampler = ClockSampler(gpu_uuid(torch, dev))
            sampler.start()
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 1.0:
                xc.xc_fp32_peak_probe(20000, sink.data_ptr(), s_ptr)
                torch.cuda.synchronize(dev)
            clk = sampler.stop()
            res["fp32_ffma_tflops"] = {"value": fl / (best * 1e-3) / 1e12, "sm_mhz": clk.get("sm_mhz"),
                                       "nominal_at_that_clock": sms * 128 * 2 * (clk.get("sm_mhz") or 0) / 1e6,
                                       "how": "xc_fp32_peak_probe: 8 FFMA chains per thread, 16 warps per SM"}
        except Exception as e:  # noqa: BLE001
            res["fp32_ffma_tflops"] = {"unavailable": str(e)[:200]}
        try:
            nbytes = 1 << 30
            h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            best, _ = ev_time(lambda: d.copy_(h, non_blocking=True), 5)
            res["h2d_pinned_gbs"] = {"value": nbytes / (best * 1e-3) / 1e9, "how": "1 GiB pinned -> device copy, best of 5"}
            del h, d
        except Exception as e:  # noqa: BLE001
            res["h2d_pinned_gbs"] = {"unavailable": str(e)[:200]}
    torch.cuda.empty_cache()
    return res


def frob_and_maxnorm(got, want, N, P):
    """Worst per-channel Frobenius relative error ||dV||_F / ||V||_F and worst
    max |dV_ab| / sqrt(V_aa V_bb) over stored entries, for outputs
    [F][N(N+1)/2][P*P][2]."""
    import numpy as np
    g = got[..., 0] + 1j * got[..., 1]
    w = want[..., 0] + 1j * want[..., 1]
    frob = np.sqrt((np.abs(g - w) ** 2).sum(axis=(1, 2)) / (np.abs(w) ** 2).sum(axis=(1, 2)))
    diag = [s * (s + 1) // 2 + s for s in range(N)]
    auto = np.stack([w[:, diag, p * P + p].real for p in range(P)], axis=-1)
    s1, s2 = np.tril_indices(N)
    worst = 0.0
    for p1 in range(P):
        for p2 in range(P):
            den = np.sqrt(auto[:, s1, p1] * auto[:, s2, p2])
            worst = max(worst, float((np.abs(g - w)[:, :, p1 * P + p2] / den).max()))
    return float(frob.max()), worst


def peak_of(peaks, measured, kind, long_region):
    """Peak in TFLOP/s for a tensor path of `kind` ("fp16" or "fp8"): the
    pool's measured dense bf16 figure (MEASURED_PEAKS.json; burst, or for a
    timed region over a second the sustained one) times the nominal
    kind/bf16 ratio (1 for fp16, 2 for fp8).  The same kind's own rate
    measured in this run is returned beside it, as context."""
    ratio = 2.0 if kind == "fp8" else 1.0
    key = "sustained" if long_region else "burst"
    base = peaks["bf16_tflops_sustained" if long_region else "bf16_tflops"]
    m = measured.get("%s_dense_tflops" % ("fp8_e4m3" if kind == "fp8" else "fp16"), {})
    return base * ratio, "bf16 %s of MEASURED_PEAKS.json x nominal %s/bf16 ratio %.0f" % (key, kind, ratio), m.get(key)


# ------------------------------------------------------------- multi-rank
# One process per GPU (torchrun): every rank correlates its own integrations
# (channels and integrations are independent; no data-path collective), the
# timed region is bracketed by barriers and the slowest rank's time counts.


def rank_integrations(rank: int, per_rank: int):
    """Integration indices (generator seeds) of one rank: disjoint across ranks."""
    return [rank * per_rank + i for i in range(per_rank)]


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (identity without a process group)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_tops(world: int, steps: int, per_rank: int, ops_per_unit: float, ms: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * steps * per_rank * ops_per_unit / (ms * 1e-3) / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9], float(parts[3])))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[3] for r in rows), "samples": len(rows), "reasons": reasons}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return "0"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_sample(x_cpu_chans, w, channels, threads=None):
    """Time the CPU oracle, as it stands, on `channels` channels of one
    integration, on `threads` threads (default: every host core).  Returns
    (seconds, ops, threads used)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    oracle.set_num_threads(threads)
    t0 = time.perf_counter()
    oracle.correlate_i8(x_cpu_chans)
    dt = time.perf_counter() - t0
    ops = w.useful_ops // w.nfreq * channels
    return dt, ops, oracle.num_threads()


# --------------------------------------------------------------- reference


def run_reference(args):
    """Reference arm: the CPU oracle on the host cores, same workload, metric
    and unit; each step is a bounded sample of channels of one integration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import oracle
    from paper_1107_4264_gb300 import synth

    oracle.build()
    w = synth.LARGE_N
    cores = os.cpu_count() or 1
    nchan = args.cpu_channels or CPU_SAMPLE_CHANNELS
    x = synth.large_n_input(w, 0, device="cpu")
    chans = list(range(nchan))
    xs = x[:, chans].contiguous().numpy()
    for _ in range(args.warmup):
        cpu_oracle_sample(xs, w, nchan)
    t_tot, ops_tot, thr = 0.0, 0, 1
    for _ in range(args.steps):
        dt, ops, thr = cpu_oracle_sample(xs, w, nchan)
        t_tot += dt
        ops_tot += ops
    value = ops_tot / t_tot / 1e12
    sample = "%d of %d channels of one integration per step (N=256 x 2 pols, T=1000)" % (nchan, w.nfreq)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": w.name, "nstation": w.nstation, "npol": w.npol, "nfreq": w.nfreq,
                   "ntime": w.ntime, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- ours


def measure_forms(args, torch, xc, synth, dev, stream, timed, peaks, measured):
    """Throughput of the other workloads (one line each in the result):
    precision forms (fp16 input, gains), the batched six-subarray launch and
    the differentiable workload's forward and adjoint."""
    res = {}
    k = args.form_steps

    def executed_planar(w, steps_per_block):
        return executed_ops(w.nstation, w.npol, w.nfreq, w.ntime, steps_per_block)

    # Precision workload: N=512 x 2 pols, F=480, T=2048, fp16 input, gains.
    w = synth.PRECISION
    x, g = synth.precision_input(w, device=dev)
    x16 = x.to(torch.float16)
    del x
    gains = torch.from_numpy(g).float().to(dev)
    prec = {}
    # Sampled channels of every form's output, kept for the error check
    # against the FP64 oracle that the CPU-baseline leg runs (outside the
    # timed region, on the same fp16 input and gains).
    import numpy as np
    rng = np.random.default_rng(w.seed + 7)
    err_chans = sorted(set([0, w.nfreq - 1] + rng.choice(w.nfreq, 2, replace=False).tolist()))
    samples = {"chans": err_chans, "x": x16[:, err_chans].double().cpu().numpy(), "gains": g,
               "N": w.nstation, "P": w.npol, "outs": {}}
    for name, form, blk, steps, peak_ratio in (("fp16", xc.XC_PREC_FP16, 0, 1, 1.0),
                                               ("hilo", xc.XC_PREC_HILO, 0, 3, 1.0),
                                               ("fp8_e4m3", xc.XC_PREC_FP8, 0, 1, 2.0),
                                               ("fp16_fp64_blocks_1024", xc.XC_PREC_FP16, 1024, 1, 1.0)):
        eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "float16", precision=form,
                            fp64_block=blk)
        eng.set_gains(gains)
        out = eng.new_output()
        eng.correlate(x16, out=out, stream=stream)
        eng.synchronize(stream)
        eng.set_option(xc.XC_OPT_PROFILE, 1)
        ms = timed(lambda: eng.correlate(x16, out=out, stream=stream), k) / k
        eng.synchronize(stream)
        (_, kms), (_, nk) = eng.kernel_times(reset=True)
        kms /= max(nk, 1)
        ex = executed_planar(w, steps)
        peak, peak_src, peak_run = peak_of(peaks, measured, "fp8" if peak_ratio == 2.0 else "fp16", False)
        samples["outs"][name] = out[err_chans].double().cpu().numpy()
        prec[name] = {"tops": w.useful_ops / (ms * 1e-3) / 1e12, "ms": ms,
                      "fp64_block": blk,
                      "kernel_ms_incl_scale_pass": kms,
                      "executed_tflops": ex / (kms * 1e-3) / 1e12,
                      "frac_of_peak": ex / (kms * 1e-3) / 1e12 / peak,
                      "peak": peak, "peak_source": peak_src, "peak_measured_this_run": peak_run}
        if blk:
            prec[name]["note"] = ("fp32 blocks of %d samples summed in float64 in device memory "
                                  "(long-integration mode; 2 drains per 2048-sample integration)" % blk)
        eng.close()
    del x16
    res["_precision_samples"] = samples
    res["precision"] = {"workload": w.name, "useful_ops": w.useful_ops, "forms": prec,
                        "errors": "per form: worst per-channel Frobenius and max |dV_ab|/sqrt(V_aa V_bb) "
                                  "over the sampled channels, against the FP64 oracle"}

    # Large-N workload re-quantised to 4 bits (sigma 3 clipped to +-7, as a
    # 4-bit digitiser delivers it) on the FP8 tensor path: exact for |x| <= 16.
    w = synth.LARGE_N
    x4 = synth.large_n_input(w, 0, device=dev).clamp_(-7, 7)
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8", precision=xc.XC_PREC_FP8)
    out = eng.new_output()
    eng.correlate(x4, out=out, stream=stream)
    eng.synchronize(stream)
    eng.set_option(xc.XC_OPT_PROFILE, 1)
    ms = timed(lambda: eng.correlate(x4, out=out, stream=stream), k) / k
    eng.synchronize(stream)  # raises on a range report
    (_, kms), (_, nk) = eng.kernel_times(reset=True)
    kms /= max(nk, 1)
    ex = executed_planar(w, 1)
    res["large_n_4bit_fp8"] = {
        "workload": "large-N int8 N=256 P=2 F=1024 T=1000, one integration per call, "
                    "samples clipped to +-7", "useful_ops": w.useful_ops,
        "tops": w.useful_ops / (ms * 1e-3) / 1e12, "ms": ms, "kernel_ms": kms,
        "executed_tflops": ex / (kms * 1e-3) / 1e12,
        "frac_of_peak": ex / (kms * 1e-3) / 1e12 / peak_of(peaks, measured, "fp8", False)[0],
        "peak": peak_of(peaks, measured, "fp8", False)[0], "peak_source": peak_of(peaks, measured, "fp8", False)[1],
        "peak_measured_this_run": peak_of(peaks, measured, "fp8", False)[2],
        "exact": "bit-exact vs the int64 oracle: tests/test_fp8_int8_gpu.py"}
    eng.close()
    del x4, out

    # F-engine (Sec. 2) at the Large-N shape: 8-bit station streams
    # [N][P][T F] -> fp16 channels already in the X-engine's layout, then the
    # FX chain (F-engine + fp16 X-engine).  The 1 GB of Large-N int8 sky data
    # is read as the streams (the transform's cost does not depend on values).
    w = synth.LARGE_N
    F = w.nfreq
    xs8 = synth.large_n_input(w, 0, device=dev).view(w.nstation, w.npol, w.ntime * F, 2)
    X16 = torch.empty((w.ntime, F, w.nstation, w.npol, 2), dtype=torch.float16, device=dev)
    scale = 1.0 / F ** 0.5
    xc.channelize(xs8, F, scale, "float16", out=X16, stream=stream)
    ms_f = timed(lambda: xc.channelize(xs8, F, scale, "float16", out=X16, stream=stream), k) / k
    nbytes = xs8.numel() * xs8.element_size() + X16.numel() * X16.element_size()
    ntrans = w.nstation * w.npol * w.ntime
    eng = xc.Correlator(w.nstation, w.npol, F, w.ntime, "float16")
    out = eng.new_output()
    eng.correlate(X16, out=out, stream=stream)
    eng.synchronize(stream)

    def fx():
        xc.channelize(xs8, F, scale, "float16", out=X16, stream=stream)
        eng.correlate(X16, out=out, stream=stream)

    ms_fx = timed(fx, k) / k
    eng.synchronize(stream)
    eng.close()
    # The same chain with the F-engine output requantised to 8 bits (scale
    # 2/sqrt(F): rms about 6 codes on this data) into the exact 8-bit X-engine.
    del X16
    X8 = torch.empty((w.ntime, F, w.nstation, w.npol, 2), dtype=torch.int8, device=dev)
    eng8 = xc.Correlator(w.nstation, w.npol, F, w.ntime, "int8")
    out8 = eng8.new_output()
    scale8 = 2.0 / F ** 0.5

    def fx8():
        xc.channelize(xs8, F, scale8, "int8", out=X8, stream=stream)
        eng8.correlate(X8, out=out8, stream=stream)

    fx8()
    eng8.synchronize(stream)
    ms_f8 = timed(lambda: xc.channelize(xs8, F, scale8, "int8", out=X8, stream=stream), k) / k
    ms_fx8 = timed(fx8, k) / k
    eng8.synchronize(stream)
    eng8.close()
    del X8, out8
    res["fengine"] = {
        "workload": "F-engine: N=256 x 2 pols, 8-bit streams of 1000 blocks x 1024 samples -> "
                    "fp16 [T][F][N][P] (corner-turned), scale 1/sqrt(F)",
        "ms": ms_f, "bytes": nbytes, "gbs": nbytes / (ms_f * 1e-3) / 1e9,
        "frac_of_hbm": nbytes / (ms_f * 1e-3) / 1e9 / peaks["hbm_gbs"],
        "peak": "%s GB/s (measured HBM copy)" % peaks["hbm_gbs"],
        "fft_gflops": 5.0 * F * (F.bit_length() - 1) * ntrans / (ms_f * 1e-3) / 1e9,
        "fx_chain": {"ms": ms_fx, "x_engine": "planar fp16 (float16 input)",
                     "useful_tops": w.useful_ops / (ms_fx * 1e-3) / 1e12},
        "fengine_int8_out_ms": ms_f8,
        "fx_chain_int8": {"ms": ms_fx8, "x_engine": "planar int8 (exact), F-engine requantised to 8 bits",
                          "useful_tops": w.useful_ops / (ms_fx8 * 1e-3) / 1e12}}
    del xs8, out

    # Batched workload: six subarrays in one persistent launch (graph replay).
    subs = [(b.nstation, b.nfreq, b.ntime) for b in synth.BATCHED]
    xs = [synth.int8_sky(b, device=dev) for b in synth.BATCHED]
    bc = xc.BatchCorrelator(subs, npol=2)
    outs = bc.new_outputs()
    cand_ms, best = bc.tune(xs, outs, reps=2, stream=stream)
    bc.correlate(xs, outs, stream=stream)
    bc.synchronize(stream)
    ms = timed(lambda: bc.correlate(xs, outs, stream=stream), k) / k
    bc.synchronize(stream)
    useful = sum(b.useful_ops for b in synth.BATCHED)
    res["batched"] = {"subarrays": [b.name for b in synth.BATCHED], "useful_ops": useful,
                      "tops": useful / (ms * 1e-3) / 1e12, "ms": ms,
                      "tuner_candidate_ms": cand_ms, "tuner_best": best, "launches_per_call": 1}
    bc.close()
    del xs, outs

    # Differentiable workload: forward with gains, adjoint (grad_x, grad_g).
    w = synth.DIFF
    x, g, _, _ = synth.diff_inputs(w, device=dev)
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "float32")
    eng.set_gains(torch.from_numpy(g).float().to(dev))
    out = eng.new_output()
    go = torch.randn(out.shape, device=dev)
    gx = torch.empty_like(x)
    eng.correlate(x, out=out, stream=stream)
    eng.correlate_backward(go, x, grad_in=gx, stream=stream)
    eng.synchronize(stream)
    fms = timed(lambda: eng.correlate(x, out=out, stream=stream), k) / k
    bms = timed(lambda: eng.correlate_backward(go, x, grad_in=gx, stream=stream), k) / k
    eng.synchronize(stream)
    n = w.npol * w.nstation
    bwd_ops = 8 * w.nfreq * n * n * w.ntime
    res["differentiable"] = {"workload": w.name, "forward_tops": w.useful_ops / (fms * 1e-3) / 1e12,
                             "forward_ms": fms, "backward_tops": bwd_ops / (bms * 1e-3) / 1e12,
                             "backward_ms": bms, "backward_ops": bwd_ops,
                             "backward_arithmetic": "tcgen05 complex GEMM (H_f diag(g)) x, fp16 hi/lo operands, fp32 accumulation"}
    eng.close()
    del x, out, go, gx

    # Small arrays (Sec. 6.1's small-N regime) at the N sweep's sizes, T = 1000:
    # the small-array engine (XC_TILE_AUTO picks it) against the planar
    # engine's packed channels (XC_TILE_128) on the same int8 sky data.  The
    # small engine is bound by its single input read: in_gbs is that stream.
    small = {}
    for N, F in ((8, 65528), (16, 65528), (32, 65104), (64, 16520)):
        T = 1000
        xs = synth.sky_voltages(T, F, N, 2, noise_sigma=3.0, nsrc=3, src_amp=1.5, seed=4242 + N + T,
                                device=dev, quantise_int8=True)
        useful = 8 * F * T * 4 * N * (N + 1) // 2
        entry = {"F": F, "T": T, "useful_ops": useful}
        for name, tile in (("small_engine", xc.XC_TILE_AUTO), ("planar_packed", xc.XC_TILE_128)):
            eng = xc.Correlator(N, 2, F, T, "int8", tile=tile)
            out = eng.new_output()
            eng.correlate(xs, out=out, stream=stream)
            eng.synchronize(stream)
            eng.set_option(xc.XC_OPT_PROFILE, 1)
            ms = timed(lambda: eng.correlate(xs, out=out, stream=stream), k) / k
            eng.synchronize(stream)
            (_, kms), (_, nk) = eng.kernel_times(reset=True)
            kms /= max(nk, 1)
            in_gbs = T * F * N * 4 / (kms * 1e-3) / 1e9
            entry[name] = {"tops": useful / (ms * 1e-3) / 1e12, "ms": ms, "kernel_ms": kms,
                           "in_gbs": in_gbs, "in_frac_of_hbm": in_gbs / peaks["hbm_gbs"]}
            eng.close()
            del out
        small["N=%d" % N] = entry
        del xs
    res["small_n"] = {"workload": "int8 sky data, P=2, T=1000, F sized as in the N sweep", "points": small,
                      "engine": "small_kernel<W> (W = 2 N P real rows per channel); planar_kernel for comparison"}
    return res


def run_sweep(args):
    """Kernel throughput of the 8-bit tensor-core engine over the station count
    N (F chosen for ~1.1e12 useful ops per integration, T = 1000; Sec. 6's
    dependence on N) and over the integration length T at fixed F*T = 1024000
    with N = 256 (the output is written once per integration, so short
    integrations are bound by output traffic)."""
    import torch

    from paper_1107_4264_gb300 import build as engine_build
    from paper_1107_4264_gb300 import synth, xc

    engine_build.build()
    xc.load()
    dev = torch.device("cuda")

    def measure(N, F, T, reps=10, tile=xc.XC_TILE_AUTO):
        x = synth.sky_voltages(T, F, N, 2, noise_sigma=3.0, nsrc=3, src_amp=1.5, seed=4242 + N + T,
                               device=dev, quantise_int8=True)
        small = tile == xc.XC_TILE_AUTO and xc.load().xc_small_engine_channels(N, 2) > 0
        eng = xc.Correlator(N, 2, F, T, "int8", tile=tile)
        out = eng.new_output()
        for _ in range(2):
            eng.correlate(x, out=out)
        eng.synchronize()
        eng.set_option(xc.XC_OPT_PROFILE, 1)
        eng.kernel_times(reset=True)
        for _ in range(reps):
            eng.correlate(x, out=out)
        eng.synchronize()
        (_, kms), (_, nk) = eng.kernel_times(reset=True)
        eng.close()
        ms = kms / max(nk, 1)
        useful = 8 * F * T * 4 * N * (N + 1) // 2
        executed = small_executed_ops(N, 2, F, T) if small else executed_ops(N, 2, F, T)
        in_b, out_b = T * F * N * 4, F * N * (N + 1) // 2 * 4 * 8
        return {"N": N, "F": F, "T": T, "engine": "small" if small else "planar",
                "channels_per_tile": xc.load().xc_small_engine_channels(N, 2) if small
                else planar_pack(N, 2, F),
                "kernel_ms": ms, "tops": useful / ms / 1e9,
                "executed_tflops": executed / ms / 1e9, "useful_fraction": useful / executed,
                "hbm_gbs_algorithmic": (in_b + out_b) / ms / 1e6}

    by_n = []
    for N in (4, 8, 16, 32, 64, 128, 256, 512, 1024):
        # Channel counts are multiples of 8, as channelised data usually is.
        F = max(8, min(65528, int(round(1.1e12 / (8 * 1000 * 4 * N * (N + 1) / 2))) // 8 * 8))
        by_n.append(measure(N, F, 1000))
        if by_n[-1]["engine"] == "small":  # the planar engine on the same sizes
            by_n.append(measure(N, F, 1000, tile=xc.XC_TILE_128))
    by_t = []
    for T in (125, 250, 500, 1000, 2000, 4000, 8000):
        by_t.append(measure(256, 1024000 // T, T))
    print(json.dumps({"sweep": "small_kernel / planar_kernel <int8>, GB300, 1 GPU", "by_nstation": by_n,
                      "by_ntime_fixed_FT": by_t}))
    return 0


def run_single(args):
    """One engine on one workload, kernel time from live CUDA events (used
    for the profiles' ncu captures of the small-array and FP8 kernels)."""
    import torch

    from paper_1107_4264_gb300 import build as engine_build
    from paper_1107_4264_gb300 import synth, xc

    engine_build.build()
    xc.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    runs = []
    if args.smalln:
        N, T = args.smalln, 1000
        F = args.nfreq or max(8, min(65528, int(round(1.1e12 / (8 * T * 4 * N * (N + 1) / 2))) // 8 * 8))
        x = synth.sky_voltages(T, F, N, 2, noise_sigma=3.0, nsrc=3, src_amp=1.5, seed=4242 + N + T,
                               device=dev, quantise_int8=True)
        useful = 8 * F * T * 4 * N * (N + 1) // 2
        for name, tile, prec in (("small_engine", xc.XC_TILE_AUTO, xc.XC_PREC_FP16),
                                 ("planar_packed", xc.XC_TILE_128, xc.XC_PREC_FP16)):
            runs.append((name, xc.Correlator(N, 2, F, T, "int8", tile=tile, precision=prec), x, useful))
        what = {"N": N, "P": 2, "F": F, "T": T}
    else:
        w = synth.LARGE_N
        if args.nfreq:
            w = synth.Workload(w.name, w.nstation, w.npol, args.nfreq, w.ntime, w.seed)
        x = synth.large_n_input(w, 0, device=dev).clamp_(-7, 7)
        runs.append(("fp8_4bit", xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8",
                                               precision=xc.XC_PREC_FP8), x, w.useful_ops))
        runs.append(("fp16", xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8"), x, w.useful_ops))
        what = {"N": w.nstation, "P": w.npol, "F": w.nfreq, "T": w.ntime, "samples": "clipped to +-7"}
    res = {"mode": "single", "workload": what}
    for name, eng, xx, useful in runs:
        out = eng.new_output()
        for _ in range(max(1, args.warmup)):
            eng.correlate(xx, out=out, stream=stream)
        eng.synchronize(stream)
        eng.set_option(xc.XC_OPT_PROFILE, 1)
        eng.kernel_times(reset=True)
        for _ in range(args.steps):
            eng.correlate(xx, out=out, stream=stream)
        eng.synchronize(stream)
        (_, kms), (_, nk) = eng.kernel_times(reset=True)
        kms /= max(nk, 1)
        res[name] = {"kernel_ms": kms, "useful_tops": useful / (kms * 1e-3) / 1e12}
        eng.close()
        del out
    print(json.dumps(res))
    return 0


def run_xc(args):
    import torch

    from paper_1107_4264_gb300 import build as engine_build
    from paper_1107_4264_gb300 import synth, xc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        engine_build.build()
    if dist:
        dist.barrier()
    xc.load()

    w = synth.LARGE_N
    if args.nfreq:
        w = synth.Workload(w.name.replace("F=1024", "F=%d" % args.nfreq), w.nstation, w.npol,
                           args.nfreq, w.ntime, w.seed)
    nint = args.integrations
    peaks, peaks_kind = load_peaks()

    # Inputs resident in HBM: this rank's 10 integrations (1.05 GB each).
    xs = torch.empty((nint,) + w.shape, dtype=torch.int8, device=dev)
    for i, seed_index in enumerate(rank_integrations(rank, nint)):
        synth.large_n_input(w, integration=seed_index, device=dev, out=xs[i])
    outs = torch.empty((nint,) + w.out_shape, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    tile = {"auto": xc.XC_TILE_AUTO, "128": xc.XC_TILE_128, "pair": xc.XC_TILE_PAIR,
            "wide": xc.XC_TILE_WIDE}[args.tile]
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "int8", engine=xc.XC_ENGINE_TENSOR,
                        tile=tile)
    eng.set_option(xc.XC_OPT_PROFILE, 1)

    def step():
        for i in range(nint):
            eng.correlate(xs[i], out=outs[i], stream=stream)

    def timed(fn, k):
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    for _ in range(args.warmup):
        step()
    eng.synchronize(stream)
    eng.kernel_times(reset=True)

    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    ms = timed(step, args.steps)
    clocks = sampler.stop()
    eng.synchronize(stream)
    (form_ms, main_ms), (n_form, n_main) = eng.kernel_times(reset=True)

    ops_int = w.useful_ops  # per integration
    value = aggregate_tops(world, args.steps, nint, ops_int, ms)
    ms_step = ms / args.steps

    # Peaks measured in this run (after the timed region, so they do not heat
    # the GPU before it), then the roofline of the dominant kernel (the
    # tensor-core X-engine) from its live launch events.
    measured = {} if args.no_peaks else measure_peaks(torch, xc, dev, stream)
    main_s = main_ms * 1e-3 / max(n_main, 1)
    form_s = form_ms * 1e-3 / max(n_form, 1)
    achieved = ops_int / main_s / 1e12
    long_region = ms * 1e-3 > 1.0
    peak, peak_note, peak_run = peak_of(peaks, measured, "fp16", long_region)
    peak_note += " (%s)" % peaks_kind
    executed = executed_ops(w.nstation, w.npol, w.nfreq, w.ntime)
    roofline = {
        "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak, "traffic": traffic_for("planar_kernel"),
        "kernel": "planar_kernel<int8> (fused: operand formation + tcgen05 kind::f16 planar complex 128x128 lower blocks + epilogue)",
        "peak_source": peak_note,
        "kernel_ms": main_s * 1e3, "launches": n_main,
        "executed_tflops": executed / main_s / 1e12,
        "algorithmic_ops_per_launch": ops_int,
        "fp16_peak_measured_this_run": peak_run,
        "frac_of_fp16_measured_this_run": achieved / peak_run if peak_run else None,
    }
    gpu_launches = n_form + n_main
    if n_form:
        roofline["form_kernel_ms"] = form_s * 1e3

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic",
        "config": {
            "workload": w.name, "nstation": w.nstation, "npol": w.npol, "nfreq": w.nfreq,
            "ntime": w.ntime, "integrations_per_step": nint, "input": "complex int8 [T][F][N][P][2]",
            "output": "int32 [F][N(N+1)/2][4][2], bit-exact",
            "arithmetic": "planar complex: int8 exact in fp16, tcgen05 fp32 accumulation in chunks with 2*max|x|^2*S <= 2^24 (exact), int32 output",
            "l2": "inputs larger than L2 (%.2f GB per integration, %.1f GB per step)"
                  % (w.ntime * w.nfreq * w.nstation * w.npol * 2 / 1e9,
                     nint * w.ntime * w.nfreq * w.nstation * w.npol * 2 / 1e9),
            "ops_convention": "8 ops per CMAC, one CMAC per stored (baseline, pol product) per sample",
            "eq_flops_tops": value * (2 * w.nstation + 1) / (2 * (w.nstation + 1)),
            "parallelism": "replicas (each rank its own integrations)" if world > 1 else "1 GPU",
        },
        "roofline": roofline,
        "peaks_measured": measured,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }

    # Same-GPU comparator: plain FP32 CUDA-core X-engine on the same inputs.
    if not args.no_comparator:
        eng.set_option(xc.XC_OPT_ENGINE, xc.XC_ENGINE_FP32)
        step()
        eng.synchronize(stream)
        eng.kernel_times(reset=True)
        cms = timed(step, args.comparator_steps)
        eng.synchronize(stream)
        (_, fp32_ms), (_, n_fp32) = eng.kernel_times(reset=True)
        eng.set_option(xc.XC_OPT_ENGINE, xc.XC_ENGINE_TENSOR)
        cvalue = world * args.comparator_steps * nint * ops_int / (cms * 1e-3) / 1e12
        props = torch.cuda.get_device_properties(dev)
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        nominal = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
        ffma = measured.get("fp32_ffma_tflops", {}).get("value")
        fp32_peak = ffma or nominal
        result["comparator_fp32"] = {
            "value": cvalue, "unit": UNIT, "kernel_ms": fp32_ms / max(n_fp32, 1),
            "fp32_peak_tflops": fp32_peak,
            "fp32_peak_source": ("measured FFMA probe, this run" if ffma else
                                 "nominal SMs x 128 lanes x 2 x sampled clock"),
            "fp32_nominal_tflops_at_sampled_clock": nominal,
            "frac_of_fp32_peak": cvalue / fp32_peak,
            "tensor_speedup": value / cvalue,
        }
        result["gpu_launches_comparator"] = n_fp32

    # End to end through the public streamed call: pinned host in and out.
    if not args.no_e2e:
        host_in = torch.empty((nint,) + w.shape, dtype=torch.int8, pin_memory=True)
        host_in.copy_(xs)
        host_out = torch.empty((nint,) + w.out_shape, dtype=torch.int32, pin_memory=True)
        torch.cuda.synchronize(dev)

        def e2e_step():
            eng.correlate_stream(host_in, nint, outs, host_out=host_out, stream=stream)

        e2e_step()
        eng.synchronize(stream)
        ems = timed(e2e_step, args.e2e_steps)
        eng.synchronize(stream)
        eng.kernel_times(reset=True)
        result["e2e"] = {
            "value": world * args.e2e_steps * nint * ops_int / (ems * 1e-3) / 1e12, "unit": UNIT,
            "h2d_bytes_per_step": host_in.numel(), "d2h_bytes_per_step": host_out.numel() * 4,
            "ms_per_step": ems / args.e2e_steps,
            "h2d_gbs": host_in.numel() * args.e2e_steps / (ems * 1e-3) / 1e9,
            "mode": "every integration's visibilities copied back (dump)",
        }
        # The paper's own pipeline (Algorithm 1): the integrations of a step
        # accumulate into one matrix, copied back once.
        host_acc = torch.empty(w.out_shape, dtype=torch.int32, pin_memory=True)
        eng.set_option(xc.XC_OPT_ACCUMULATE, 1)

        def alg1_step():
            eng.correlate_stream(host_in, nint, outs[0], host_out=host_acc, stream=stream)

        alg1_step()
        eng.synchronize(stream)
        ams = timed(alg1_step, args.e2e_steps)
        eng.synchronize(stream)
        eng.kernel_times(reset=True)
        eng.set_option(xc.XC_OPT_ACCUMULATE, 0)
        result["e2e_algorithm1"] = {
            "value": world * args.e2e_steps * nint * ops_int / (ams * 1e-3) / 1e12, "unit": UNIT,
            "h2d_bytes_per_step": host_in.numel(), "d2h_bytes_per_step": host_acc.numel() * 4,
            "ms_per_step": ams / args.e2e_steps,
            "mode": "ACCUMULATE: 10 integrations summed into one matrix, copied back once per step",
        }
        del host_in, host_out, host_acc

    if not args.no_forms and world == 1:
        result["workloads"] = measure_forms(args, torch, xc, synth, dev, stream, timed, peaks, measured)

    samples = result.get("workloads", {}).pop("_precision_samples", None)
    # CPU baseline: the oracle as it stands, bounded sample, rank 0 at N=1.
    if not args.no_cpu_baseline and world == 1 and rank == 0:
        if samples:
            # The precision forms' errors against the FP64 oracle on their
            # sampled channels (the oracle recomputes them on the host).
            import oracle
            want = oracle.correlate_f64(samples["x"], gains=samples["gains"])
            for name, got in samples["outs"].items():
                frob, mx = frob_and_maxnorm(got, want, samples["N"], samples["P"])
                result["workloads"]["precision"]["forms"][name]["error_vs_fp64_oracle"] = {
                    "frobenius": frob, "max_normalised": mx, "channels": samples["chans"]}
        cores = os.cpu_count() or 1
        nchan = min(args.cpu_channels or CPU_SAMPLE_CHANNELS, w.nfreq)
        xs_cpu = xs[0][:, :nchan].contiguous().cpu().numpy()
        # The same sample as every reference-arm step, repeated until about
        # 10 s of host work.
        dt, ops, reps = 0.0, 0, 0
        while dt < 10.0 or reps < 2:
            d, o, thr = cpu_oracle_sample(xs_cpu, w, nchan)
            dt, ops, reps = dt + d, ops + o, reps + 1
        dt1, ops1, _ = cpu_oracle_sample(xs_cpu[:, :1].copy(), w, 1, threads=1)
        result["cpu_baseline"] = {
            "value": ops / dt / 1e12, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": "%d of %d channels of integration 0 (N=256 x 2 pols, T=1000), %d times, %.1f s"
                      % (nchan, w.nfreq, reps, dt),
            "cpu": cpu_model(),
            "single_thread": {"value": ops1 / dt1 / 1e12, "unit": UNIT,
                              "sample": "1 channel on 1 thread, %.2f s" % dt1},
        }

    eng.close()
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_fengine(args):
    """F-engine alone: N=256 x 2 pols of 8-bit station streams, 1024 channels,
    --fengine-blocks blocks, into fp16, fp32 and 8-bit codes (corner-turned), timed
    with CUDA events over --steps calls after --warmup."""
    import torch

    from paper_1107_4264_gb300 import build as engine_build
    from paper_1107_4264_gb300 import synth, xc

    engine_build.build()
    xc.load()
    dev = torch.device("cuda")
    N, P, F, T = 256, 2, 1024, args.fengine_blocks
    x = synth.uniform_int8((N, P, T * F, 2), -128, 127, 4242, device=dev)
    peaks, kind = load_peaks()
    res = {"fengine": "N=%d x %d pols, %d channels, %d blocks, 8-bit streams" % (N, P, F, T)}
    for odt in ("float16", "float32", "int8"):
        out = torch.empty((T, F, N, P, 2), dtype=getattr(torch, odt), device=dev)
        for _ in range(max(args.warmup, 1)):
            xc.channelize(x, F, 1.0 / 32, odt, out=out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            xc.channelize(x, F, 1.0 / 32, odt, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nbytes = x.numel() + out.numel() * out.element_size()
        res[odt] = {"ms": ms, "gbs": nbytes / ms / 1e6,
                    "frac_of_hbm": nbytes / ms / 1e6 / peaks["hbm_gbs"], "peak_kind": kind}
        del out
    # Polyphase front end, 4 taps (T - 3 output blocks), fp16 out.
    taps = torch.ones((4, F), device=dev)
    out = torch.empty((T - 3, F, N, P, 2), dtype=torch.float16, device=dev)
    for _ in range(max(args.warmup, 1)):
        xc.channelize(x, F, 1.0 / 64, "float16", out=out, taps=taps)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        xc.channelize(x, F, 1.0 / 64, "float16", out=out, taps=taps)
    e1.record()
    torch.cuda.synchronize()
    res["polyphase_4_taps_float16"] = {"ms": e0.elapsed_time(e1) / args.steps,
                                       "output_blocks": T - 3}
    print(json.dumps(res))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.smalln or args.fp8_4bit:
        return run_single(args)
    if args.fengine:
        return run_fengine(args)
    return run_xc(args)


if __name__ == "__main__":
    sys.exit(main())
