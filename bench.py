#!/usr/bin/env python3
"""Benchmark of the MWAX FX correlator hot path on one B300 (or N independent replicas).

Workload (full-array plain form): 256 tiles x 2 pols = 512 signal paths, one coarse
channel, one 8 s sub-observation at 1.28 MS/s (10.24 M int8 complex samples per path,
seeded noise sigma=16 plus a common point source with linear per-tile delays, sky
frequency 139.52 MHz), 128-point FFT (10 kHz), 0.5 s integrations (16 per call),
averaged to 40 kHz (fscrunch 4), FP32.  One step = one mwax_correlate call over the
whole sub-observation (F-step + X-step + averaging/ordering for all 16 integrations).

metric: real-time 256-tile coarse channels per B300 = 8 s / (device time per
sub-observation), summed over GPUs.  Inputs (10.5 GB) exceed the 126 MB L2, so no flush
is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SUBOBS_S = 8.0
FS = 1_280_000.0
WORKLOAD = dict(name="full-array plain FX, 256 tiles, 8 s sub-observation, N=128, 0.5 s, fscrunch 4",
                n_tiles=256, fft_len=128, fine_avg=4, int_time_s=0.5, samples=10_240_000, seed=0x4D574159,
                sky_freq_hz=139.52e6)
# one 0.5 s integration of the same array: the small case used for ncu captures
SMALL = dict(WORKLOAD, name="full-array plain FX, 256 tiles, one 0.5 s integration, N=128, fscrunch 4",
             samples=640_000)
METRIC = "real-time 256-tile coarse channels per B300"
# Plan workspace of the timed forms: 48 GiB holds the operands of all 16 integrations of
# the sub-observation at once (FP32: 43 GB), so the F-step and the X-step each run as one
# launch over the whole call (B300 has 275 GB of HBM).
WORKSPACE = 48 << 30

# DRAM bytes (read + write) per integration slot of the dominant kernel, from an ncu
# capture of the one-integration case (profiles/).  Reported only while the kernel's
# source is byte-identical to the one captured (sha1 prefix of its .cu file).
TRAFFIC = {"xstep_simt_kernel": ("paper_2303_11557_b300/csrc/xstep_simt.cu", "4aed89a75fb5", 6.595614e9 + 0.098705e9)}


def traffic_per_slot(kernel: str):
    import hashlib
    if kernel not in TRAFFIC:
        return None
    path, sha, per_slot = TRAFFIC[kernel]
    try:
        h = hashlib.sha1(open(os.path.join(ROOT, path), "rb").read()).hexdigest()
    except OSError:
        return None
    return per_slot if h.startswith(sha) else None
FP32_LANES_PER_SM = 128


def sm_count(torch, dev: int = 0) -> int:
    return torch.cuda.get_device_properties(dev).multi_processor_count


def measure_peaks(mw, torch, dev: int, seconds: float = 2.0):
    """Roofline denominators that MEASURED_PEAKS.json does not hold, measured here with CUDA
    events (no clock or power setting touched), each as a burst (best of several short
    runs) and sustained (back to back for `seconds`), with the SM clock sampled meanwhile:
    - FP32 FMA: the library's FMA probe (16 independent chains per thread, full occupancy);
    - FP8 e4m3 dense tensor: cuBLASLt through torch._scaled_mm at 8192^3, as the bf16 figure
      of MEASURED_PEAKS.json is cuBLAS at 8192^3."""
    res = {"sms": sm_count(torch, dev)}
    clocks = ClockSampler(dev)
    clocks.start()
    stream = torch.cuda.current_stream()

    def rate(fn, work, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return work * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12

    blocks = res["sms"] * 8
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    iters = 4096
    fmas = mw.mwax_probe_fma(blocks, iters, sink)
    torch.cuda.synchronize()
    one = rate(lambda: mw.mwax_probe_fma(blocks, iters, sink), 2.0 * fmas, 1)
    reps = max(1, int(0.05 / max(2.0 * fmas / (one * 1e12), 1e-6)))   # ~50 ms per burst sample
    burst = max(rate(lambda: mw.mwax_probe_fma(blocks, iters, sink), 2.0 * fmas, reps) for _ in range(5))
    sus_reps = max(1, int(seconds / (2.0 * fmas / (burst * 1e12))))
    sus = rate(lambda: mw.mwax_probe_fma(blocks, iters, sink), 2.0 * fmas, sus_reps)
    res["fp32_fma_tflops"] = burst
    res["fp32_fma_tflops_sustained"] = sus
    res["fp32_fma_probe"] = f"mwax_probe_fma: {blocks} blocks x 256 threads x {iters * 8 * 16} FMA"
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one_s = torch.tensor(1.0, device="cuda")
        mm = lambda: torch._scaled_mm(a, b, scale_a=one_s, scale_b=one_s, out_dtype=torch.bfloat16)
        mm()
        torch.cuda.synchronize()
        flop = 2.0 * n ** 3
        res["fp8_tflops"] = max(rate(mm, flop, 10) for _ in range(3))
        res["fp8_tflops_sustained"] = rate(mm, flop, max(1, int(seconds / (flop / (res["fp8_tflops"] * 1e12)))))
        res["fp8_how"] = "torch._scaled_mm e4m3 x e4m3 -> bf16, 8192^3 (cuBLASLt)"
        del a, b
    except Exception as e:   # no FP8 GEMM in this torch build: the nominal ratio is used instead
        res["fp8_unavailable"] = f"{type(e).__name__}: {str(e)[:120]}"
    res["clocks"] = clocks.stop()
    return res


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
            "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        load = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- inputs
def make_inputs(W, pin: bool):
    import torch
    import synth
    T, S = W["n_tiles"], W["samples"]
    delay = synth.tile_delays_linear(W["seed"], T)
    host = torch.empty(S // 64_000 * 2 * T * 64_000 * 2, dtype=torch.int8, pin_memory=pin)
    synth.voltages(W["seed"], 2 * T, S, tones=synth.point_source_tones(W["seed"]), delay_c01=delay[:, :2],
                   sky_freq_hz=W["sky_freq_hz"], out=host.numpy().reshape(-1, 2 * T, 64_000, 2))
    return host, delay


def used_bins(N: int, F: int, keep_dc: int = 0) -> int:
    """Ultrafine channels that feed at least one output channel (Sec. 2.6 geometry)."""
    M, half = N // F, F // 2
    used = set()
    for j in range(M):
        mid = (j - M // 2) * F
        for u in range(mid - half, mid + half + 1):
            if not -(N // 2) <= u < N - N // 2:
                continue
            if u == 0 and F > 1 and not keep_dc:
                continue
            used.add(u)
    return len(used)


def algorithmic_work(T: int, N: int, F: int, K: int, n_ints: int, prec_bytes: int):
    """Algorithmic work of one call: X flops over the ultrafine bins that feed an output
    (8 real flops per complex multiply-accumulate over the unique pairs p <= q), and
    F-step bytes (2 B of int8 in, two operand planes out per sample and path)."""
    n = 2 * T
    used = used_bins(N, F)
    pairs = n * (n + 1) // 2
    x_flops = 8.0 * pairs * K * used * n_ints
    f_bytes = (2.0 + 2 * prec_bytes) * n * K * N * n_ints
    return x_flops, f_bytes, used


# ------------------------------------------------------------------------- cpu / oracle
def oracle_sample_time(threads_note: dict, Ts: int = 32):
    """Time the FP64 oracle on a bounded sample of the workload: a Ts-tile sub-array, one
    0.5 s integration (5000 frames), same N, F and delays.  Returns (seconds per 8 s
    256-tile sub-observation extrapolated, description, measured seconds)."""
    import oracle
    import synth
    W = WORKLOAD
    N, F = W["fft_len"], W["fine_avg"]
    K = int(W["int_time_s"] * FS) // N
    S = K * N
    d = synth.tile_delays_linear(W["seed"], Ts)
    volt = synth.voltages(W["seed"], 2 * Ts, S, tones=synth.point_source_tones(W["seed"]), delay_c01=d[:, :2],
                          sky_freq_hz=W["sky_freq_hz"])
    desc = oracle.Desc(n_tiles=Ts, fft_len=N, fine_avg=F, int_frames=K, n_samples=S,
                       sky_freq_hz=W["sky_freq_hz"])
    t0 = time.perf_counter()
    for p in range(2 * Ts):
        oracle.spectra(desc, volt, d, p, 0, K)
    t_f = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.correlate(desc, volt, d)
    t_all = time.perf_counter() - t0
    t_x = max(t_all - t_f, 0.0)
    n_s, n_f = 2 * Ts, 2 * W["n_tiles"]
    bp_s, bp_f = Ts * (Ts + 1) // 2, W["n_tiles"] * (W["n_tiles"] + 1) // 2
    n_ints = int(SUBOBS_S / W["int_time_s"])
    est = (t_f * (n_f / n_s) + t_x * (bp_f / bp_s)) * n_ints
    desc_s = (f"{Ts}-tile sub-array, one 0.5 s integration (N=128, F=4): F part x{n_f // n_s} paths, X part "
              f"x{bp_f / bp_s:.1f} baselines, x{n_ints} integrations")
    threads_note["cores"] = int(os.environ.get("OMP_NUM_THREADS", 0)) or len(os.sched_getaffinity(0))
    return est, desc_s, t_all


def oracle_config0_time():
    """Seconds the FP64 oracle takes (all host cores) for the whole parity workload of 16
    tiles, 0.4 s, N = 128, no averaging (not extrapolated: it runs in full)."""
    import oracle
    import synth
    T, N, S = 16, 128, 512_000
    d = synth.tile_delays_fixed(T)
    volt = synth.voltages(0x4D574158, 2 * T, S, tones=synth.point_source_tones(0x4D574158), delay_c01=d[:, :2],
                          sky_freq_hz=WORKLOAD["sky_freq_hz"])
    desc = oracle.Desc(n_tiles=T, fft_len=N, fine_avg=1, int_frames=S // N, n_samples=S,
                       sky_freq_hz=WORKLOAD["sky_freq_hz"], dc_exclude=0)
    t0 = time.perf_counter()
    oracle.correlate(desc, volt, d)
    return time.perf_counter() - t0


def oracle_one_core():
    """The same oracle timing on one host core (a separate process with OMP_NUM_THREADS=1,
    which the oracle's OpenMP runtime reads at start), on a 16-tile sub-array so that it
    stays a bounded sample; extrapolated to the workload the same way."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; n = {}; "
            "e, s, t = bench.oracle_sample_time(n, Ts=16); print(json.dumps([e, s, t]))" % ROOT)
    try:
        res = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                             capture_output=True, text=True, timeout=300)
        est, sample, t = json.loads(res.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError, OSError) as e:
        return {"unavailable": f"one-core oracle run failed: {type(e).__name__}"}
    return {"value": SUBOBS_S / est, "unit": "channels", "cores": 1, "sample": sample, "measured_s": t,
            "extrapolated_s_per_subobs": est}


# ----------------------------------------------------------------------------- arms
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    if rank != 0:
        return
    note = {}
    for _ in range(args.warmup):
        oracle_sample_time(note)
    ests, descs, meas = [], "", []
    for _ in range(args.steps):
        est, descs, t = oracle_sample_time(note)
        ests.append(est)
        meas.append(t)
    est = statistics.median(ests)
    value = SUBOBS_S / est
    line = {"metric": METRIC, "value": value, "unit": "channels", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * est, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded noise + point source)",
            "impl": "reference",
            # each step times a bounded sample (a 32-tile sub-array, one 0.5 s integration) and
            # scales it to the 256-tile 8 s sub-observation: ms_per_step and value are extrapolated
            "extrapolated": True, "measured_sample_s_per_step": statistics.median(meas),
            "config": {"workload": WORKLOAD["name"], "precision": "fp64 oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": "channels", "cores": note.get("cores"), "kind": "oracle",
                             "sample": descs},
            "e2e": {"value": value, "unit": "channels", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------ 24-channel batch and real-time serving
F_CHOICES = {32: [1], 128: [1, 4], 1280: [10, 40], 6400: [50, 200]}


def mixed_channels(seed: int, n: int = 24, int8_share: float = 0.0):
    """Seeded mix of coarse channels: tiles in {128, 256, 512}, FFT length in {32, 128,
    1280, 6400}, fscrunch giving >= 10 kHz channels, integration in {0.25, 0.5, 2, 8} s;
    a share of them in the integer mode (no FFT, 1.28 MHz)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        T = int(rng.choice([128, 256, 512]))
        t = float(rng.choice([0.25, 0.5, 2.0, 8.0]))
        if rng.random() < int8_share:
            out.append(dict(T=T, N=1, F=1, t=t, prec="int8"))
        else:
            N = int(rng.choice([32, 128, 1280, 6400]))
            out.append(dict(T=T, N=N, F=int(rng.choice(F_CHOICES[N])), t=t, prec="fp16"))
    return out


def channel_volt(torch, dev_base, T):
    """Voltages of a T-tile channel: the resident 256-tile 8 s voltage bytes viewed (128 tiles: the
    first half; 256: all; 512: two copies) as [160 blocks][2T paths][64000][2]."""
    need = 160 * 2 * T * 64_000 * 2
    if need <= dev_base.numel():
        return dev_base[:need]
    return torch.cat([dev_base] * (need // dev_base.numel()))


def run_batch24(mw, torch, dev_base, args):
    """24 coarse channels of mixed shapes, one batch call per 8 s sub-observation
    (FP16 X-engine in one persistent launch per round, autotuned, CUDA-graph replayed)."""
    chans = mixed_channels(0x4D57415B)
    plans, vols, outs = [], {}, []
    tuned = {}
    for c in chans:
        d = mw.PlanDesc(n_tiles=c["T"], fft_len=c["N"], fine_avg=c["F"], int_time_s=c["t"],
                        samples_per_call=10_240_000, precision=mw.MWAX_FP16, sky_freq_hz=WORKLOAD["sky_freq_hz"],
                        workspace_limit=4 << 30)
        p = mw.mwax_plan_create_ex(d)
        mw.mwax_plan_set_stream(p)
        if c["T"] not in vols:
            vols[c["T"]] = channel_volt(torch, dev_base, c["T"])
        o = mw.empty_output(p)
        key = (c["T"], c["N"], c["F"], c["t"])
        if key not in tuned:
            tuned[key] = mw.mwax_plan_autotune(p, vols[c["T"]], None, o)
        else:
            mw.mwax_plan_set_tuning(p, tuned[key])
        plans.append(p)
        outs.append(o)
    b = mw.Batch(plans)
    V = [vols[c["T"]] for c in chans]
    b.correlate(V, None, outs)          # eager
    b.correlate(V, None, outs)          # capture + replay
    b.sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    e0.record()
    for _ in range(steps):
        b.correlate(V, None, outs)
    e1.record()
    b.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    flops = 0.0
    for c in chans:
        n = 2 * c["T"]
        flops += 8.0 * n * (n + 1) / 2 * 10_240_000 / c["N"] * used_bins(c["N"], c["F"])
    b.close()
    for p in plans:
        p.close()
    return {"workload": "24 coarse channels, 8 s each, tiles {128,256,512}, N {32,128,1280,6400}, "
                        "int {0.25,0.5,2,8} s (seeded mix), FP16, one batch call",
            "ms_per_batch": ms, "realtime_factor": SUBOBS_S / (ms * 1e-3),
            "channels_realtime": 24 * SUBOBS_S / (ms * 1e-3), "x_tflops_alg": flops / (ms * 1e-3) / 1e12,
            "tunings": {f"T{k[0]} N{k[1]} F{k[2]} t{k[3]}": repr(v) for k, v in tuned.items()},
            "mix": [f"T{c['T']}/N{c['N']}/F{c['F']}/{c['t']}s" for c in chans],
            "input": "the 256-tile 8 s voltage bytes re-tiled per tile count (every channel computed in full)"}


def run_serve(mw, torch, host_base, args, periods: int = 2, counts=(24, 32, 40, 48, 56, 64)):
    """Real-time serving: n coarse channels each delivering an 8 s sub-observation every 8 s
    (seeded offsets within the period), FP16 or integer mode per request (80/20), host
    pinned voltages; the server admits by HBM footprint; deadline = 8 s.  The 24-channel
    load is measured first, then the offered count is raised until a deadline is missed:
    the capacity is the largest count with no miss.  Warm-up requests (one per new shape,
    which create the plans) run before each count's statistics are reset."""
    chans_all = mixed_channels(0x4D57415C, n=max(counts), int8_share=0.2)
    hosts, outs = {}, {}

    def host_volt(T):
        if T not in hosts:
            need = 160 * 2 * T * 64_000 * 2
            if need <= host_base.numel():
                hosts[T] = host_base[:need]
            else:
                h = torch.empty(need, dtype=torch.int8, pin_memory=True)
                for k in range(need // host_base.numel()):
                    h[k * host_base.numel():(k + 1) * host_base.numel()].copy_(host_base)
                hosts[T] = h
        return hosts[T]

    def desc_of(c):
        prec = mw.MWAX_INT8 if c["prec"] == "int8" else mw.MWAX_FP16
        return mw.PlanDesc(n_tiles=c["T"], fft_len=c["N"], fine_avg=c["F"], int_time_s=c["t"],
                           samples_per_call=10_240_000, precision=prec, sky_freq_hz=0.0, workspace_limit=4 << 30)

    def key_of(d):
        return (d.n_tiles, d.fft_len, d.fine_avg, d.int_time_s, d.precision)

    def out_for(d):
        # one pinned result buffer per shape, shared by that shape's requests: the read-back
        # volume is the same, results are not inspected here (the tests compare them)
        k = key_of(d)
        if k not in outs:
            p = mw.mwax_plan_create_ex(d)
            outs[k] = torch.empty(p.output_bytes, dtype=torch.uint8, pin_memory=True)
            p.close()
        return outs[k]

    srv = mw.Server(hbm_budget=160 << 30, n_lanes=4)
    warmed, sweep, first = set(), [], None
    for n in counts:
        chans = chans_all[:n]
        descs = [desc_of(c) for c in chans]
        for d in descs:   # warm-up of the shapes not seen yet (plan creation, module loading)
            if key_of(d) not in warmed:
                warmed.add(key_of(d))
                srv.submit(d, host_volt(d.n_tiles), None, out_for(d))
        srv.drain()
        srv.reset_stats()
        rng = np.random.default_rng(0x5E7E + n)
        offsets = rng.uniform(0, SUBOBS_S, n)
        t0 = time.perf_counter()
        events = sorted((pp * SUBOBS_S + offsets[k], k) for pp in range(periods) for k in range(n))
        for at, k in events:
            while time.perf_counter() - t0 < at:
                time.sleep(0.0005)
            srv.submit(descs[k], host_volt(descs[k].n_tiles), None, out_for(descs[k]), deadline_s=SUBOBS_S)
        srv.drain()
        wall = time.perf_counter() - t0
        st = srv.stats()
        up = sum(160 * 2 * d.n_tiles * 64_000 * 2 for d in descs) / SUBOBS_S / 1e9
        row = {"channels": n, "completed": st["completed"], "deadline_misses": st["deadline_misses"],
               "cold_starts": st["cold_starts"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
               "p50_warm_ms": st["p50_warm_ms"], "p99_warm_ms": st["p99_warm_ms"],
               "throughput_channels": st["completed"] * SUBOBS_S / wall, "wall_s": wall,
               "upload_gb_per_s_offered": up}
        sweep.append(row)
        if first is None:
            first = row
        if st["deadline_misses"] > 0:
            break
    srv.close()
    capacity = max([r["channels"] for r in sweep if r["deadline_misses"] == 0], default=0)
    return {"workload": f"{counts[0]} coarse channels x {periods} sub-observations of 8 s at wall-clock rate, tiles "
                        "{128,256,512}, mixed N/F/int as the 24-channel batch, 20 % integer mode, host pinned voltages",
            "p50_ms": first["p50_ms"], "p99_ms": first["p99_ms"], "max_ms": first["max_ms"],
            "p50_warm_ms": first["p50_warm_ms"], "p99_warm_ms": first["p99_warm_ms"],
            "cold_starts": first["cold_starts"],
            "deadline_ms": 1e3 * SUBOBS_S, "deadline_misses": first["deadline_misses"], "completed": first["completed"],
            "sustained_channels": counts[0] * (first["completed"] - first["deadline_misses"]) / max(1, first["completed"]),
            "capacity_channels": capacity,
            "capacity_note": "largest offered channel count (of the sweep) with no deadline miss over "
                             f"{periods} periods; the sweep stops at the first count that misses",
            "sweep": sweep,
            "latency_note": "warm-up requests (one per new shape) excluded; p50/p99 over every timed request, "
                            "*_warm over those whose lane already held the plan (no plan creation)",
            "lanes": 4, "hbm_budget_gb": 160}


def time_plan(mw, torch, plan, dev_volt, dev_delay, steps, warmup, world, clocks=None):
    """Warm up, then time `steps` calls on the plan's stream with CUDA events (and per-stage
    events inside the library).  Returns (ms per step max over ranks, stage times, output)."""
    stream = torch.cuda.current_stream()
    mw.mwax_plan_set_stream(plan, stream)
    out = mw.empty_output(plan)
    # the clock sampler (nvidia-smi) starts, and the library's stage events are created,
    # before the warm-up: neither start-up happens inside the timed region
    if clocks:
        clocks.start()
        time.sleep(1.0)
    mw.mwax_plan_enable_timing(plan, True)
    for _ in range(warmup):
        mw.mwax_correlate(plan, dev_volt, dev_delay, out)
    mw.mwax_plan_sync(plan)
    mw.mwax_plan_stage_times(plan)          # reset counters
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        mw.mwax_correlate(plan, dev_volt, dev_delay, out)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop() if clocks else None
    mw.mwax_plan_sync(plan)
    stages = mw.mwax_plan_stage_times(plan)
    mw.mwax_plan_enable_timing(plan, False)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
    return ms, stages, out, ck


def _time_calls(torch, fn, steps, warmup):
    """Device milliseconds per call of fn() on torch's current stream (CUDA events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_extensions(mw, torch, W, dev_volt, delay, args, mpk):
    """The roadmap rows on the full 256-tile sub-observation (Sec. 2.4, 4.1-4.5): per-call
    device time of the plain FP16 call beside the same call with zeroing flags +
    normalisation, a 5 ms delay table, de-ripple gains; an oversampled channel (FP16);
    and 8 tied-array beams with detected outputs (FP32), with the beam kernel's rate."""
    import numpy as np
    import synth
    T, S, N = W["n_tiles"], W["samples"], W["fft_len"]
    n = 2 * T
    steps, warm = max(2, min(args.steps, 3)), 1
    res = {}
    desc = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=W["fine_avg"], int_time_s=W["int_time_s"], samples_per_call=S,
                       precision=mw.MWAX_FP16, sky_freq_hz=W["sky_freq_hz"])
    plan = mw.mwax_plan_create_ex(desc)
    mw.mwax_plan_set_stream(plan)
    out = mw.empty_output(plan)
    ddelay = torch.from_numpy(delay).cuda()
    n_blocks = S // 64_000
    flags = torch.from_numpy((np.random.default_rng(W["seed"]).random((n_blocks, n)) < 0.01).astype(np.uint8)).cuda()
    t_mid = (np.arange(S // 6400) + 0.5) * 6400 / synth.FS
    table = torch.from_numpy(np.ascontiguousarray(delay[:, :1] + delay[:, 1:2] * t_mid[None, :])).cuda()
    u = np.arange(N) - N // 2
    gains = (1.0 / ((1 + 0.03 * np.cos(2 * np.pi * u / 21.0)) * (1 - 0.45 * (np.abs(u) / (N / 2)) ** 6)))
    plain = _time_calls(torch, lambda: mw.mwax_correlate(plan, dev_volt, ddelay, out), steps, warm)
    fl = _time_calls(torch, lambda: mw.mwax_correlate_ex(plan, dev_volt, out, delay_poly=ddelay, zero_flags=flags,
                                                         normalise=True), steps, warm)
    tb = _time_calls(torch, lambda: mw.mwax_correlate_ex(plan, dev_volt, out, delay_table=table), steps, warm)
    mw.mwax_plan_set_passband(plan, gains.astype(np.float32))
    pb = _time_calls(torch, lambda: mw.mwax_correlate(plan, dev_volt, ddelay, out), steps, warm)
    plan.close()
    del out
    ch = lambda ms: SUBOBS_S / (ms * 1e-3)
    res["fp16_plain"] = {"ms_per_subobs": plain, "channels": ch(plain)}
    res["zero_flags_normalised"] = {"ms_per_subobs": fl, "channels": ch(fl), "flagged_blocks": "1 % seeded"}
    res["delay_table_5ms"] = {"ms_per_subobs": tb, "channels": ch(tb), "steps_per_path": int(S // 6400)}
    res["passband_deripple"] = {"ms_per_subobs": pb, "channels": ch(pb)}
    # oversampled coarse channel: 32/25 x 1.28 MS/s, the central 100 of 128 bins, 25 channels
    fs = 1.6384e6
    od = mw.PlanDesc(n_tiles=T, fft_len=N, fine_avg=4, int_time_s=1_024_000 / fs, samples_per_call=S,
                     precision=mw.MWAX_FP16, sky_freq_hz=W["sky_freq_hz"], sample_rate_hz=fs, keep_bins=100)
    op = mw.mwax_plan_create_ex(od)
    mw.mwax_plan_set_stream(op)
    oo = mw.empty_output(op)
    os_ms = _time_calls(torch, lambda: mw.mwax_correlate(op, dev_volt, ddelay, oo), steps, warm)
    res["oversampled_32_25"] = {"ms_per_call": os_ms, "seconds_of_data": S / fs, "real_time_factor": S / fs / (os_ms * 1e-3),
                                "n_chan_out": op.info["n_chan_out"]}
    op.close()
    del oo
    # tied-array beams: 8 beams, 5 ms steering tables, 10 ms detected Stokes I + incoherent;
    # both engines (0: tensor cores from FP16 hi/lo pairs, 1: FP32 CUDA cores)
    nb = 8
    rng = np.random.default_rng(W["seed"] + 4)
    btab = torch.from_numpy(delay[None, :, :1] + rng.uniform(-200e-9, 200e-9, (nb, n, 1)) +
                            delay[None, :, 1:2] * t_mid[None, None, :]).cuda()
    flops = 8.0 * nb * n * S
    fp32_peak = mpk["fp32_fma_tflops_sustained"]
    beam = {"n_beams": nb, "work": "8 flop per beam x path x sample (complex MAC); calls include the F-step",
            "fp32_peak_tflops": fp32_peak, "fp32_peak_kind": "measured FMA probe, sustained"}
    for engine, name in ((0, "tensor_cores"), (1, "cuda_cores")):
        bf = mw.Beamformer(T, N, nb, S, sky_freq_hz=W["sky_freq_hz"], int_frames=100, engine=engine)
        bf.set_stream()
        beams = torch.empty(bf.output_bytes(0), dtype=torch.uint8, device="cuda")
        power = torch.empty(bf.output_bytes(1), dtype=torch.uint8, device="cuda").view(torch.float32)
        incoh = torch.empty(bf.output_bytes(2), dtype=torch.uint8, device="cuda").view(torch.float32)
        bms = _time_calls(torch, lambda: bf.form(dev_volt, btab, beams, power, incoh), steps, warm)
        beam[name] = {"ms_per_subobs": bms, "real_time_factor": SUBOBS_S / (bms * 1e-3),
                      "whole_call_tflops": flops / (bms * 1e-3) / 1e12}
        del bf, beams, power, incoh
    beam["cuda_cores"]["whole_call_frac_fp32"] = beam["cuda_cores"]["whole_call_tflops"] / fp32_peak
    # the tensor-core engine issues 12 FP16 products of M 128 x N 16 per 16 tiles, channel, pol
    # and 16 beams over units of at most 128 frames: at 50 frames per 5 ms step and 8 beams,
    # issued / algorithmic = (128 / 50) (16 / 8) x 3 (hi/lo products)
    beam["tensor_cores"]["issued_tflops_fp16"] = beam["tensor_cores"]["whole_call_tflops"] * (128 / 50) * 2 * 3
    bf16_sus = peaks()[0].get("bf16_tflops_sustained", 1400.0)
    beam["tensor_cores"]["issued_frac_of_tensor_peak"] = beam["tensor_cores"]["issued_tflops_fp16"] / bf16_sus
    res["beamformer"] = beam
    return res


def rel_error_vs(mw, torch, plan, out, ref_vis, T):
    """max / median of |V - V_ref| / sqrt(V_ref,pp V_ref,qq) (parallel-pol autos of V_ref)."""
    vis, _ = mw.split_output(plan, out)
    ti = torch.tensor([i for i in range(T) for _ in range(i, T)], device=vis.device)
    tj = torch.tensor([j for i in range(T) for j in range(i, T)], device=vis.device)
    auto_b = ti.new_tensor([i * (2 * T - i + 1) // 2 for i in range(T)])
    mx, meds = 0.0, []
    for w in range(vis.shape[0]):
        r, v = ref_vis[w], vis[w]
        for pol in range(4):
            a, e = pol >> 1, pol & 1
            ap = r[:, :, 3 * a].real.abs()[auto_b[ti]]
            aq = r[:, :, 3 * e].real.abs()[auto_b[tj]]
            err = (v[:, :, pol] - r[:, :, pol]).abs() / torch.sqrt(ap * aq)
            mx = max(mx, float(err.max()))
            meds.append(float(err.median()))
    return mx, statistics.median(meds)


def run_mine(args, world, rank, local):
    import torch
    import paper_2303_11557_b300 as mw

    torch.cuda.set_device(local)
    W = SMALL if args.workload == "small" else WORKLOAD
    if args.fft_len:
        # profiler captures of the other FFT lengths on the small workload only
        if W is not SMALL:
            raise SystemExit("--fft-len applies to --workload small (profiler captures)")
        W = dict(W, fft_len=args.fft_len, fine_avg=args.fine_avg or 1,
                 name=f"{W['name']} (N={args.fft_len}, fscrunch {args.fine_avg or 1})")
    host, delay = make_inputs(W, pin=not args.no_e2e)
    dev_volt = host.cuda(non_blocking=False)
    dev_delay = torch.from_numpy(delay).cuda()
    if args.beam_only:
        # the beamformer alone on this workload (profiler captures): 8 beams, one engine
        import synth
        T, S, N, n = W["n_tiles"], W["samples"], W["fft_len"], 2 * W["n_tiles"]
        nb = 8
        t_mid = (np.arange(S // 6400) + 0.5) * 6400 / synth.FS
        rng = np.random.default_rng(W["seed"] + 4)
        btab = torch.from_numpy(delay[None, :, :1] + rng.uniform(-200e-9, 200e-9, (nb, n, 1)) +
                                delay[None, :, 1:2] * t_mid[None, None, :]).cuda()
        bf = mw.Beamformer(T, N, nb, S, sky_freq_hz=W["sky_freq_hz"], int_frames=100, engine=args.beam_engine)
        bf.set_stream()
        beams = torch.empty(bf.output_bytes(0), dtype=torch.uint8, device="cuda")
        power = torch.empty(bf.output_bytes(1), dtype=torch.uint8, device="cuda").view(torch.float32)
        incoh = torch.empty(bf.output_bytes(2), dtype=torch.uint8, device="cuda").view(torch.float32)
        ms = _time_calls(torch, lambda: bf.form(dev_volt, btab, beams, power, incoh), args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"beam_only": True, "engine": args.beam_engine, "workload": W["name"], "n_beams": nb,
                              "ms_per_call": ms, "tflops_whole_call": 8.0 * nb * n * S / (ms * 1e-3) / 1e12}), flush=True)
        return
    pk, pk_kind = peaks()
    mpk = measure_peaks(mw, torch, local)
    headline = args.precision
    forms = [headline] + ([] if args.no_forms else [f for f in ("fp32", "fp16x3", "fp16", "fp8", "int8")
                                                     if f != headline])
    results, ref_vis, line_parts = {}, None, {}
    for form in forms:
        prec = mw.PRECISIONS[form]
        if form == "int8":
            # integer mode on the same voltages: no FFT (1.28 MHz channels), 1 s integrations
            desc = mw.PlanDesc(n_tiles=W["n_tiles"], fft_len=1, fine_avg=1, int_time_s=1.0 if W is WORKLOAD else 0.5,
                               samples_per_call=W["samples"], precision=prec, workspace_limit=WORKSPACE)
            ddelay = None
        else:
            desc = mw.PlanDesc(n_tiles=W["n_tiles"], fft_len=W["fft_len"], fine_avg=W["fine_avg"],
                               int_time_s=W["int_time_s"], samples_per_call=W["samples"], precision=prec,
                               sky_freq_hz=W["sky_freq_hz"], workspace_limit=WORKSPACE)
            ddelay = dev_delay
        plan = mw.mwax_plan_create_ex(desc)
        # one-off autotune on this workload (F-step variant, run length, tensor-core window),
        # as a user does once per shape; the timed steps below run the chosen tuning
        tuning = (mw.mwax_plan_get_tuning(plan) if args.no_tune
                  else mw.mwax_plan_autotune(plan, dev_volt, ddelay, mw.empty_output(plan)))
        if args.fstep_variant is not None:   # a fixed F-step kernel (profiler captures)
            tuning = mw.Tuning(args.fstep_variant, tuning.run_len, tuning.window, 0.0)
            mw.mwax_plan_set_tuning(plan, tuning)
        torch.cuda.empty_cache()
        clocks = ClockSampler(local) if form == headline else None
        ms, stages, out, ck = time_plan(mw, torch, plan, dev_volt, ddelay, args.steps, args.warmup, world, clocks)
        info = plan.info
        K, n_ints = info["frames_per_int"], info["n_ints"]
        N, F = desc.fft_len, desc.fine_avg
        elem = {"fp32": 4, "fp16": 2, "fp8": 1, "int8": 2, "fp16x3": 4}[form]
        x_flops, f_bytes, used = algorithmic_work(W["n_tiles"], N, F, K, n_ints, elem)
        if form == "fp8" and tuning.fstep_variant == 2:
            # the DFT-product F-steps write FP16: a maxima pass and a quantisation pass follow
            f_bytes += 2.0 * 2 * W["n_tiles"] * K * N * n_ints
        x_ms, x_n = stages["xstep"]
        f_ms, f_n = stages["fstep"]
        x_per_launch = x_flops * args.steps / x_n
        x_avg_ms = x_ms / x_n
        x_achieved = x_per_launch / (x_avg_ms * 1e-3) / 1e12
        nominal = None
        if form == "fp32":
            xkern, bound = "xstep_simt_kernel", "alu"
            x_peak = mpk["fp32_fma_tflops_sustained"]
            nominal = mpk["sms"] * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
            peak_kind = (f"measured FP32 FMA throughput, sustained ({mpk['fp32_fma_probe']}, "
                         f"SM clock median {mpk['clocks'].get('sm_mhz')} MHz); nominal {mpk['sms']} SMs x "
                         f"{FP32_LANES_PER_SM} lanes x 2 x {pk.get('sm_max_mhz')} MHz = {nominal:.1f} TFLOP/s")
        elif form == "fp8" and "fp8_tflops_sustained" in mpk:
            xkern, bound = "xstep_tc_kernel<0> (e4m3)", "tensor"
            x_peak = mpk["fp8_tflops_sustained"]
            peak_kind = f"measured dense e4m3, sustained ({mpk['fp8_how']})"
        else:
            xkern = {"fp16": "xstep_tc_kernel<0> (fp16)", "fp8": "xstep_tc_kernel<0> (e4m3)",
                     "fp16x3": "xstep_tc_kernel<1> (fp16 hi/lo pairs)",
                     "int8": "xstep_tc_kernel<2> (integer mode)"}[form]
            bound = "tensor"
            base = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
            ratio = 2.0 if form == "fp8" else 1.0
            x_peak = base * ratio
            peak_kind = (f"{pk_kind} dense bf16 cuBLAS, sustained" + (" x 2 (fp8 : bf16 nominal 4.5 : 2.25)"
                                                                        if form == "fp8" else " (fp16 = bf16 rate)")
                         + ("; int8 values run exactly as fp16" if form == "int8" else "")
                         + ("; three fp16 products per algorithmic term, so frac <= 1/3 by construction"
                            if form == "fp16x3" else ""))
        tps = traffic_per_slot(xkern) if form == headline else None
        r = {"value": world * SUBOBS_S * (n_ints * desc.int_time_s / SUBOBS_S) / (ms * 1e-3),
             "ms_per_step": ms, "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
             "tuning": repr(tuning),
             "launches_per_step": sum(v[1] for v in stages.values()) / args.steps,
             "roofline": {"bound": bound, "kernel": xkern, "achieved": x_achieved, "peak": x_peak, "unit": "TFLOP/s",
                          "frac": x_achieved / x_peak,
                          "traffic": None if tps is None else tps * n_ints * args.steps / x_n,
                          "peak_kind": peak_kind, "nominal_peak": nominal,
                          "per_launch": f"{x_per_launch:.4g} flop (8 x pairs x frames x {used} used bins)",
                          "avg_launch_ms": x_avg_ms,
                          # what the kernel executes with this tuning: whole tiles (pairs below
                          # the diagonal and past n included), K blocks, shared boundary channels
                          "issued_per_launch": info["x_flop_issued"] * args.steps / x_n,
                          "issued_achieved": info["x_flop_issued"] * args.steps / x_n / (x_avg_ms * 1e-3) / 1e12,
                          "issued_frac": info["x_flop_issued"] * args.steps / x_n / (x_avg_ms * 1e-3) / 1e12
                          * (3.0 if form == "fp16x3" else 1.0) / x_peak,
                          "issued_note": "issued_frac counts the three FP16 products per term of the hi/lo form"
                          if form == "fp16x3" else "issued_frac = issued_achieved / peak"},
             "roofline_fstep": {"bound": "hbm", "achieved": f_bytes / (f_ms / args.steps * 1e-3) / 1e9,
                                "peak": pk["hbm_gbs"], "unit": "GB/s",
                                "frac": f_bytes / (f_ms / args.steps * 1e-3) / 1e9 / pk["hbm_gbs"],
                                "per_step_bytes": f_bytes, "peak_kind": f"{pk_kind} copy bandwidth"},
             "gpu_launches": sum(v[1] for v in stages.values())}
        if form == "fp32" and form != "int8":
            vis32, _ = mw.split_output(plan, out)
            ref_vis = vis32.clone()
        elif form in ("fp16", "fp8", "fp16x3") and ref_vis is not None:
            mx, med = rel_error_vs(mw, torch, plan, out, ref_vis, W["n_tiles"])
            r["error_vs_fp32"] = {"max": mx, "median": med,
                                  "metric": "|V - V_fp32| / sqrt(auto_pp auto_qq), full workload"}
        if form == headline:
            line_parts["clocks"] = ck
            line_parts["info"] = info
            line_parts["plan"] = plan
            line_parts["desc"] = desc
        else:
            plan.close()
            del out
        results[form] = r

    # end to end through the host-memory entry point (pinned buffers), headline precision
    plan, info = line_parts["plan"], line_parts["info"]
    e2e = None
    if not args.no_e2e:
        # End to end from pinned host memory through the streaming host call: every step
        # uploads its 10.5 GB of voltages and reads back its visibilities; the upload of
        # step k + 1 overlaps the correlation of step k, as in a real-time loop.  The
        # synchronous one-call latency (upload, correlate, read back, nothing overlapped
        # across calls) is reported beside it.
        host_outs = [torch.empty(plan.output_bytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        for k in range(2):                                     # warm-up (allocates both staging sets)
            mw.mwax_correlate_host_async(plan, host, delay, host_outs[k])
        mw.mwax_plan_sync(plan)
        # every timed call uploads its own voltages and reads back its result; the first
        # upload overlaps nothing, so more calls amortise that pipeline fill
        reps = max(10, args.steps)
        barrier(world)
        t0 = time.perf_counter()
        for k in range(reps):
            mw.mwax_correlate_host_async(plan, host, delay, host_outs[k % 2])
        mw.mwax_plan_sync(plan)
        t_e2e = max_over_ranks((time.perf_counter() - t0) / reps, world)
        t0 = time.perf_counter()
        mw.mwax_correlate_host(plan, host, delay, host_outs[0])
        t_sync = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * info["n_ints"] * W["int_time_s"] / t_e2e, "unit": "channels",
               "h2d_bytes_per_step": info["input_bytes"] + delay.nbytes, "d2h_bytes_per_step": info["output_bytes"],
               "ms_per_step": 1e3 * t_e2e, "steps": reps,
               "mode": "streaming host call, next upload overlapped with the current correlation",
               "sync_call_ms": 1e3 * t_sync}

    ext = None
    if not args.no_ext and W is WORKLOAD:
        ext = run_extensions(mw, torch, W, dev_volt, delay, args, mpk)

    # 24 batched channels of mixed shapes, then real-time serving
    batch = serve = None
    if not args.no_batch and W is WORKLOAD:
        plan.close()
        batch = run_batch24(mw, torch, dev_volt, args)
    if not args.no_serve and not args.no_e2e and W is WORKLOAD:
        serve = run_serve(mw, torch, host, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        note = {}
        est, sample, _ = oracle_sample_time(note)
        cpu = {"value": SUBOBS_S / est, "unit": "channels", "cores": note["cores"], "kind": "oracle",
               "sample": sample, "extrapolated_s_per_subobs": est}
        cpu["one_core"] = oracle_one_core()
        cpu["config0_whole_run_s"] = oracle_config0_time()

    if rank != 0:
        return
    h = results[headline]
    line = {
        "metric": METRIC, "value": h["value"], "unit": "channels", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "fp8": "e4m3",
                                                          "int8": "s8", "fp16x3": "f16x3"}[headline],
        "data": "synthetic (seeded Gaussian sigma=16 + point source, linear per-tile delays)",
        "config": {"workload": W["name"], "n_tiles": W["n_tiles"], "fft_len": W["fft_len"],
                   "fine_avg": W["fine_avg"], "int_time_s": W["int_time_s"], "subobs_s": SUBOBS_S,
                   "precision": headline, "l2": "inputs 10.5 GB > 126 MB L2, no flush needed",
                   "parallelism": f"replicas x{world} (independent coarse channels)"},
        "roofline": h["roofline"],
        "roofline_fstep": h["roofline_fstep"],
        "stage_ms_per_step": h["stage_ms_per_step"],
        "tuning": h["tuning"],
        "gpu_launches": h["gpu_launches"],
        "clocks": line_parts["clocks"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "precision_forms": {f: {k: v for k, v in r.items() if k != "gpu_launches"} for f, r in results.items()
                            if f != headline},
        "measured_peaks": mpk,
        "batch": batch,
        "serving": serve,
        "extensions": ext,
        "context": {"paper": "1 coarse channel of 256 tiles in real time per NVIDIA A40 (6.2 s per 8 s at "
                             "250 ms / 40 kHz, Table 2)"},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16x3", "fp16", "fp8", "int8"],
                    help="headline precision (the full-array plain form is FP32); the other forms are timed beside it")
    ap.add_argument("--no-forms", action="store_true", help="time the headline precision only")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep each plan's default tuning (no autotune launches; for profiler captures)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-channel batched measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the real-time serving measurement")
    ap.add_argument("--no-ext", action="store_true", help="skip the roadmap extensions and the beamformer")
    ap.add_argument("--fft-len", type=int, default=0,
                    help="with --workload small: another FFT length (for profiler captures of the F-step)")
    ap.add_argument("--fine-avg", type=int, default=0, help="fscrunch with --fft-len")
    ap.add_argument("--workload", default="full", choices=["full", "small"],
                    help="small = one 0.5 s integration (for profiler captures)")
    ap.add_argument("--fstep-variant", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="fix the F-step kernel (0 radix-32 / generic, 1 generic, 2 tensor-core DFT "
                         "products, 3 128-row tensor-core, 4 frames-on-lanes direct DFT) after tuning")
    ap.add_argument("--beam-only", action="store_true", help="time the beamformer alone (profiler captures)")
    ap.add_argument("--beam-engine", type=int, default=0, choices=[0, 1],
                    help="with --beam-only: 0 tensor cores, 1 CUDA cores")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_mine(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
