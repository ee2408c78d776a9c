#!/usr/bin/env python3
"""Benchmark of the multi-tone synthesis hot path on GB300.

Workload (the one the headline metric is quoted on): 1000 tones, each chirped from a seeded
frequency to a seeded target in 80-180 MHz over 35 ms at 280 MS/s (9.8M samples); even tones
linear, odd tones minimum-jerk; amplitudes U[0.5, 1]/1000; int16 output in 2^18-sample chunks.

One step = the whole record rendered chunk by chunk through the C ABI: awg_render_stream over the
37 full chunks and the last, shorter one (one chirp tile set-up per group of chunks, one render
kernel per chunk with its fused quantise-and-store, consecutive renders overlapping on the
device).  `value` is tone-samples per second with the tone state resident on the
device; `e2e` repeats the step through the public API from host arrays (set_tones + set_chirps,
then rendering straight into pinned host memory).  The CPU oracle is timed on the host cores on a
bounded window of the same workload (`cpu_baseline`); `--impl reference` times only that oracle.
With N GPUs (torchrun) every rank renders its own replica of the workload; the step time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tone-samples/s and max real-time tones at 280 MS/s; p50/p99 chunk latency at ≤1 LSB"
UNIT = "tone-samples/s"
# Paper (Playback pathway, Quadro RTX 6000): 1000 tones chirped for 35 ms at 280 MS/s computed in
# 610 ms, i.e. 9.8e9 / 0.61 tone-samples/s.  Context, another machine.
PAPER_TONE_SAMPLES_PER_S = 9.8e9 / 0.610
# SFU peak used as the roofline denominator of the render kernel: 16 sine results per clock per SM
# x the device's SMs (queried) x its maximum SM clock (nvidia-smi clocks.max.sm during the timed
# region; 2070 MHz on GB300 if unsampled).
SFU_SIN_PER_CLK_SM = 16
SM_MAX_MHZ_DEFAULT = 2070.0
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one render launch of the timed
# step (a 2^18-sample chunk of the 1000-chirp record), from one ncu capture of the render kernel as
# it stands in this file's revision; None when the kernel has changed since that capture.
RENDER_TRAFFIC_BYTES = 11.92832e6
RENDER_TRAFFIC_SOURCE = "ncu --set full capture of one render_split_kernel launch (2^18 samples, 1000 chirps; shared LOW3 run set-up, 7 CTAs per SM)"

CLOCK_FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload():
    from paper_2403_15582_gb300 import workloads as wl
    return wl.chirp_1000(seed=0)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.thread = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(CLOCK_FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(CLOCK_FIELDS):
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for name, v in zip(names, s[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        pw = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples),
                "power_w_max": max(pw) if pw else None}


def oracle_window_rate(wk, seconds: float, n0: int | None = None, record=None, parity=None):
    """Time the CPU oracle (all host cores) on a window of the workload sized for ~`seconds`.
    With `record` (the int16 samples the GPU rendered for the whole workload), the timed window is
    also compared with them: `parity` receives the largest |difference| in LSB and the share of
    samples equal to the oracle's FP64 sum quantised in FP64."""
    import numpy as np
    import oracle
    oracle.build()
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, grid_log2=wk.grid_log2)
    nthreads = os.cpu_count() or 1
    start = wk.n_samples // 2 if n0 is None else n0
    probe = 4096
    t0 = time.perf_counter()
    oracle.render(w, start, probe, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(max(probe, probe * seconds / dt), wk.n_samples - start))
    t0 = time.perf_counter()
    x_ref = oracle.render(w, start, n, nthreads=nthreads)
    dt = time.perf_counter() - t0
    used = oracle.render.last_threads
    if record is not None and parity is not None:
        dq = np.abs(record[start:start + n].astype(np.int32) - oracle.quantize(x_ref, w.full_scale()).astype(np.int32))
        parity.update({"samples": int(n), "from_sample": int(start), "max_lsb": int(dq.max(initial=0)),
                       "exact_fraction": float(np.mean(dq == 0)), "reference": "oracle FP64 sum, quantised in FP64"})
    # the same oracle on one thread, on a window sized to ~a quarter of the time budget
    n1 = max(probe, min(n, int(n / max(used, 1) * 0.25)))
    t0 = time.perf_counter()
    oracle.render(w, start, n1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": wk.K * n / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{wk.K} tones x {n} samples from sample {start} (FP64 direct sum, 192-bit chirp cascade)",
            "seconds": dt,
            "single_thread": {"value": wk.K * n1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{wk.K} tones x {n1} samples from sample {start}", "seconds": dt1}}


def run_reference(args, wk):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, grid_log2=wk.grid_log2)
    nthreads = os.cpu_count() or 1
    start = wk.n_samples // 2
    t0 = time.perf_counter()
    oracle.render(w, start, 4096, nthreads=nthreads)
    rate = 4096 * wk.K / max(time.perf_counter() - t0, 1e-6)
    per_step = int(min(max(4096, rate * 2.0 / wk.K), wk.n_samples - start))   # ~2 s per step
    for _ in range(args.warmup):
        oracle.render(w, start, per_step, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.render(w, start, per_step, nthreads=nthreads)
    dt = time.perf_counter() - t0
    value = wk.K * per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_TONE_SAMPLES_PER_S,
            "dtype": "f64", "data": "synthetic", "config": config(wk, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.render.last_threads, "kind": "oracle",
                             "sample": f"{wk.K} tones x {per_step} samples per step from sample {start}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def stream_leg(awg, fs: float, stream, seconds: float = 1.0, n_slots: int = 4, prefill: int = 2, engine: int = 0):
    """Continuous stream of 10,000 tones whose groups of 100 ramp in turn (1 ms linear ramps),
    2^20-sample chunks through the pinned ring with a real-time host sink: underruns and chunk
    latency (engine: the static-tone engine, direct or tensor-core GEMM)."""
    from paper_2403_15582_gb300 import workloads as wl
    from paper_2403_15582_gb300.stream import run_stream
    wk = wl.stream_rotating(seed=0, fs=fs, seconds=seconds)
    synth = awg.Synth(fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    synth.set_static_engine(engine)
    ring = awg.Ring(synth, wk.chunk, n_slots)
    n_chunks = -(-wk.n_samples // wk.chunk)
    st = run_stream(synth, ring, wk.chirps, n_chunks, stream, prefill=prefill)
    ring.close()
    synth.close()
    return {"tones": wk.K, "fs_hz": fs, "chunk": wk.chunk, "chunks": int(st["played"]), "underruns": int(st["underruns"]),
            "chunk_latency_ms": {"p50": st["latency_p50_ms"], "p99": st["latency_p99_ms"], "max": st["latency_max_ms"]},
            "min_lead_ms": st["lead_min_ms"], "playback_ms": st["chunk_playback_ms"], "slots": n_slots,
            "required_tone_samples_per_s": wk.K * fs, "static_engine": ["direct", "gemm_fp16", "gemm_bf16"][engine]}


def chirping_leg(awg, stream, K: int, fs: float = 280e6, chunk: int = 1 << 20, segments: int = 7,
                 n_slots: int = 3, prefill: int = 2):
    """K tones that all chirp all the time (back-to-back 33.7 ms linear / minimum-jerk chirps between
    seeded 80-180 MHz frequencies), streamed in real time through the pinned ring with a host sink
    playing one chunk per chunk / fs: underruns and chunk latency (GPU completion minus push)
    against the playback time of a chunk.  Beside it, the device rate of one segment rendered
    through the pipelined chunk loop with the tone state resident."""
    import torch
    from paper_2403_15582_gb300 import workloads as wl
    from paper_2403_15582_gb300.stream import run_stream
    wk = wl.chirping_stream(seed=0, K=K, fs=fs, segments=segments)
    S = wk.n_samples // segments
    synth = awg.Synth(fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    ring = awg.Ring(synth, chunk, n_slots)
    n_chunks = wk.n_samples // chunk
    t0 = time.perf_counter()
    st = run_stream(synth, ring, wk.chirps, n_chunks, stream, prefill=prefill)
    wall = time.perf_counter() - t0
    status = synth.device_status()
    ring.close()
    synth.close()
    # device rate: the first segment through the pipelined chunk loop, best of 3
    synth = awg.Synth(fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    synth.set_chirp_list([c for c in wk.chirps if c["start_sample"] == 0])
    out = torch.empty(S, dtype=torch.int16, device="cuda")
    ts = []
    for r in range(4):
        synth.seek(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        synth.render_stream(S, chunk, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            ts.append(e0.elapsed_time(e1))
    # one chunk at a time on an otherwise idle device: set-up + render of each chunk (library events)
    o1 = torch.empty(chunk, dtype=torch.int16, device="cuda")
    synth.profile_begin()
    synth.seek(0)
    for _ in range(min(16, S // chunk)):
        synth.render(chunk, o1, stream)
    torch.cuda.synchronize()
    prep, rend, _ = synth.profile_end()
    synth.close()
    import numpy as np
    iso = np.asarray(prep) + np.asarray(rend)
    ms = min(ts)
    playback = 1e3 * chunk / fs
    lat99 = float(np.percentile(iso, 99))
    return {"tones": K, "chirping": K, "fs_hz": fs, "chunk": chunk, "chunks": int(st["played"]),
            "underruns": int(st["underruns"]), "playback_ms": playback,
            # set-up + render of one chunk issued to the device alone (the latency a chunk adds)
            "chunk_latency_ms": {"p50": float(np.percentile(iso, 50)), "p99": lat99, "chunks": int(iso.size)},
            "p99_within_playback": bool(lat99 < playback),
            # the ring: GPU completion minus push, which includes waiting behind the chunks the
            # producer queued ahead (the start-up fill drains at the device's margin over real time)
            "ring_push_to_complete_ms": {"p50": st["latency_p50_ms"], "p99": st["latency_p99_ms"], "max": st["latency_max_ms"]},
            "min_lead_ms": st["lead_min_ms"],
            "required_tone_samples_per_s": K * fs, "stream_wall_s": wall, "device_status": status,
            "device_segment_ms": ms, "device_tone_samples_per_s": K * S / (ms * 1e-3),
            "device_realtime_factor": (S / fs * 1e3) / ms,
            "slots": n_slots, "prefill": prefill, "segment_samples": S}


def sfu_probe(awg, stream, n_sm: int, achieved: float, runs: int = 1024, reps: int = 5, probe=None, what="static"):
    """The rate the SFU sustains in one of the render kernel's own loops alone (no staging, set-up
    or split sums; one wave of 5 CTAs per SM), best of a few launches: a measured ceiling beside
    the nominal SFU rate, and the render's rate in the timed steps against it."""
    import torch
    probe = probe or awg.sfu_rate_probe
    blocks = 5 * n_sm
    out = torch.empty(blocks * 128, dtype=torch.float32, device="cuda")
    probe(out, blocks, runs, stream)       # warm-up
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        probe(out, blocks, runs, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    rate = blocks * 128 * runs * 32 / (best * 1e-3) / 1e12
    name = "awg_sfu_rate_probe" if what == "static" else "awg_chirp_rate_probe"
    return {"value": rate, "unit": "Tsin/s", "frac": achieved / rate,
            "source": f"{name}: the render's {what} sine loop alone, {blocks} CTAs x 128 threads x {runs} runs of 32 samples, best of {reps}"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def table_leg(awg, stream, reps: int = 3, K: int = 10000, log2_len: int = 24, gpu: int = 0):
    """Periodic K-tone table of 2^log2_len samples (default 10,000 tones, 2^24): split-precision
    tcgen05 GEMM (FP16 and BF16 hi+lo) against the direct-sum render of the same record on the same
    GPU.  Per precision: the median of a few calls (against the burst bf16 peak), then calls back to
    back for about half a second with the SM clock sampled (against the sustained peak: a dense
    GEMM runs into the power cap)."""
    import numpy as np
    import torch
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.table_10000(seed=0, K=K, log2_len=log2_len)
    lg = wk.grid_log2
    N = 1 << lg
    synth = awg.Synth(wk.fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=lg)
    q = torch.empty(N, dtype=torch.int16, device="cuda")
    out = {"workload": f"table-{wk.K}tone-2^{lg}", "tone_samples": wk.K * N}
    peaks, src = measured_peaks()
    flops = 3 * 2.0 * (N // 256) * 256 * (2 * wk.K)          # three hi/lo products, 2K inner terms
    for prec, name in ((1, "fp16"), (0, "bf16")):
        synth.table_gemm(lg, prec, q, None, stream)          # warm-up
        synth.profile_begin()
        for _ in range(reps):
            synth.table_gemm(lg, prec, q, None, stream)
        torch.cuda.synchronize()
        prep, gemm, _ = synth.profile_end()
        g = float(np.median(gemm))
        out[name] = {"gemm_ms": g, "operand_prep_ms": float(np.median(prep)),
                     "tflops": flops / (g * 1e-3) / 1e12,
                     "frac_of_bf16_peak": flops / (g * 1e-3) / 1e12 / peaks["bf16_tflops"],
                     "tone_samples_per_s": wk.K * N / (g * 1e-3)}
        R = max(8, int(0.5 / max(g * 1e-3, 1e-6)))
        cs = ClockSampler(gpu)
        cs.start()
        time.sleep(0.2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(R):
            synth.table_gemm(lg, prec, q, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        cs.stop()
        gs = e0.elapsed_time(e1) / R
        out[name]["sustained"] = {"calls": R, "ms_per_call": gs,   # B-operand set-up (about 0.02 ms) included
                                  "tflops": flops / (gs * 1e-3) / 1e12,
                                  "frac_of_bf16_sustained": flops / (gs * 1e-3) / 1e12 / peaks["bf16_tflops_sustained"],
                                  "clocks": cs.summary()}
    synth.profile_begin()
    for _ in range(reps):
        synth.seek(0)
        synth.render(N, q, stream)
    torch.cuda.synchronize()
    prep, rend, _ = synth.profile_end()
    d = float(np.median(prep + rend))
    out["direct_ms"] = d
    out["direct_tone_samples_per_s"] = wk.K * N / (d * 1e-3)
    out["peak_source"] = f"{src} bf16 {peaks['bf16_tflops']} TFLOP/s (FP16 dense rate taken equal)"
    synth.close()
    return out


def static_leg(awg, stream, reps: int = 5):
    """Static combs in both sine variants: the 100-tone 2^20-sample record and a 10,000-tone comb
    over 2^22 samples (one render call each; best of reps; library profiling events)."""
    import numpy as np
    import torch
    from paper_2403_15582_gb300 import workloads as wl
    out = {}
    c1 = wl.static_100(seed=0)
    rng = np.random.default_rng(0)
    f = 80e6 + 1e4 * np.sort(rng.choice(10000, 10000, replace=False)).astype(np.float64)
    cases = {"static-100tone-2^20": (c1.fs, c1.freq_hz, c1.amp, c1.phase_rad, c1.n_samples),
             "static-10000tone-2^22": (280e6, f, np.full(10000, 1e-4), rng.uniform(0, 2 * np.pi, 10000), 1 << 22)}
    # the same comb with 100 tones fading (minimum-jerk amplitude ramps of 1 ms) inside the record
    ramps = [dict(tone=int(t), amp_end=0.0 if i % 2 else 2e-4, duration=1e-3, profile=1,
                  start_sample=int(rng.integers(0, (1 << 22) - 280000)))
             for i, t in enumerate(rng.choice(10000, 100, replace=False))]
    cases["static-10000tone-2^22+100ramps"] = cases["static-10000tone-2^22"]
    for name, (fs, fr, amp, th, n) in cases.items():
        synth = awg.Synth(fs)
        synth.set_tones(fr, amp, th)
        if name.endswith("ramps"):
            synth.set_ramp_list(ramps)
        q = torch.empty(n, dtype=torch.int16, device="cuda")
        res = {}
        for mode, engine, label in ((awg.SINE_SFU, awg.STATIC_DIRECT, "sfu"), (awg.SINE_ROTATOR, awg.STATIC_DIRECT, "rotator"),
                                    (awg.SINE_SFU, awg.STATIC_GEMM_FP16, "gemm_fp16")):
            synth.set_sine_mode(mode)
            synth.set_static_engine(engine)
            synth.seek(0)
            synth.render(n, q, stream)      # warm-up
            synth.profile_begin()
            for _ in range(reps):
                synth.seek(0)
                synth.render(n, q, stream)
            torch.cuda.synchronize()
            _, rend, _ = synth.profile_end()
            ms = float(np.min(rend)) if len(rend) else float("nan")
            if engine != awg.STATIC_DIRECT:   # the GEMM path has no profiling split: time the call
                ts = []
                for _ in range(reps):
                    synth.seek(0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    synth.render(n, q, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = float(np.min(ts))
            res[label] = {"render_ms": ms, "tone_samples_per_s": len(fr) * n / (ms * 1e-3)}
        out[name] = res
        synth.close()
    # digital SFDR of the int16 output for grid tones (periodic 2^20-sample record, unwindowed FFT)
    lg, N = 20, 1 << 20
    for K in (1, 100):
        j = np.sort(rng.choice(np.arange(N // 20, N // 2 - N // 20), K, replace=False))
        synth = awg.Synth(280e6)
        synth.set_tones(j * 280e6 / N, np.full(K, 1.0 / K), rng.uniform(0, 2 * np.pi, K), grid_log2=lg)
        q = torch.empty(N, dtype=torch.int16, device="cuda")
        res = {}
        for mode, label in ((awg.SINE_SFU, "sfu"), (awg.SINE_ROTATOR, "rotator")):
            synth.set_sine_mode(mode)
            synth.seek(0)
            synth.render(N, q, stream)
            torch.cuda.synchronize()
            P = np.abs(np.fft.rfft(q.cpu().numpy().astype(np.float64))) ** 2
            mask = np.ones(P.size, dtype=bool)
            mask[0] = False
            mask[j] = False
            res[label] = float(10 * np.log10(P[j].min() / P[mask].max()))
        out[f"sfdr_dbc_grid_{K}tone_2^20"] = res
        synth.close()
    return out


def chirp_profile_leg(awg, stream, wk, reps: int = 3):
    """The C2 record (1000 tones chirping 80-180 MHz over 35 ms) with every chirp on one profile:
    linear, minimum-jerk, exponential; pipelined chunk renders, best of reps, L2 flushed before
    each."""
    import numpy as np
    import torch
    N, chunk = wk.n_samples, wk.chunk
    tone, f0, f1, dur, _, start = wk.chirp_arrays()
    out = torch.empty(N, dtype=torch.int16, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for prof, label in ((awg.PROFILE_LINEAR, "linear"), (awg.PROFILE_MINJERK, "minjerk"),
                        (awg.PROFILE_EXPONENTIAL, "exponential")):
        synth = awg.Synth(wk.fs)
        synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
        synth.set_chirps(tone, f0, f1, dur, np.full(len(tone), prof, dtype=np.int32), start)
        ts = []
        for r in range(reps + 1):
            synth.seek(0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            synth.render_stream(N, chunk, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        ms = float(np.min(ts))
        res[label] = {"ms": ms, "tone_samples_per_s": wk.K * N / (ms * 1e-3), "device_status": synth.device_status()}
        synth.close()
    return res


def periodic_leg(awg, stream, reps: int = 5):
    """Periodic hand-off: the 10,000-tone 2^24-sample table (split-precision GEMM, FP16) set up
    once, then replayed for 2^28 samples; replay rate against the measured HBM copy bandwidth
    (2 B written per sample; the 32 MB table is read from L2)."""
    import numpy as np
    import torch
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.table_10000(seed=0)
    synth = awg.Synth(wk.fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=wk.grid_log2)
    t0 = time.perf_counter()
    synth.set_periodic(wk.grid_log2, awg.PERIODIC_GEMM_FP16, stream)
    setup_s = time.perf_counter() - t0
    n = 1 << 28
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    ts = []
    for _ in range(reps + 1):
        synth.seek(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        synth.render(n, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts[1:]))
    peaks, src = measured_peaks()
    gbs = 2.0 * n / (ms * 1e-3) / 1e9
    synth.close()
    return {"table": f"{wk.K} tones x 2^{wk.grid_log2} (GEMM FP16)", "setup_s": setup_s, "replay_samples": n,
            "replay_ms": ms, "samples_per_s": n / (ms * 1e-3), "tone_samples_per_s": wk.K * n / (ms * 1e-3),
            "write_gbs": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"], "peak_source": f"{src} hbm {peaks['hbm_gbs']} GB/s"}


def late_chunk_breakdown(srv):
    """Where the time of each late chunk went: release -> planning of the round that completed it
    (host), planning -> device start (queue), device start -> done; medians over the late chunks,
    and the same for all chunks c >= 1."""
    import numpy as np
    rounds, chunks = srv.trace_rounds(), srv.trace_chunks()
    if len(rounds) == 0 or len(chunks) == 0:
        return {}
    by_done = {float(r["t_done"]): r for r in rounds}

    def parts(sel):
        rows = []
        for c in sel:
            r = by_done.get(float(c["done"]))
            if r is None:
                continue
            rows.append((1e3 * (r["t_plan"] - c["release"]), 1e3 * (r["t_start"] - r["t_plan"]),
                         1e3 * (r["t_done"] - r["t_start"]), 1e3 * (c["due"] - c["release"]), r["work"], r["pieces"]))
        if not rows:
            return {"n": 0}
        a = np.array(rows, dtype=np.float64)
        return {"n": len(rows), "release_to_plan_ms": float(np.median(a[:, 0])), "plan_to_start_ms": float(np.median(a[:, 1])),
                "start_to_done_ms": float(np.median(a[:, 2])), "period_ms": float(np.median(a[:, 3])),
                "round_work": float(np.median(a[:, 4])), "round_pieces": float(np.median(a[:, 5])),
                "max_release_to_plan_ms": float(a[:, 0].max()), "max_plan_to_start_ms": float(a[:, 1].max()),
                "max_start_to_done_ms": float(a[:, 2].max())}
    later = chunks[chunks["chunk"] >= 1]
    lead = 1e3 * (later["due"] - later["done"])   # time to spare at completion
    return {"late": parts(later[later["late"] != 0]), "all": parts(later),
            "lead_ms": {"min": float(lead.min()), "p01": float(np.percentile(lead, 1)), "p50": float(np.percentile(lead, 50))}
            if len(lead) else {}}


def served_leg(awg, fs: float = 280e6, seconds: float = 2.0, rho: float = 0.8, prefetch: int = 2,
               engine: int = 0, engine_min_tones: int = 1000):
    """Served rearrangement stream: Poisson arrivals of requests (50-10,000 tones, up to 100 chirping
    over 0.1-2 ms, 8 chunks of 2^16-2^20 samples) at rho x capacity / mean request work, submitted in
    real time; admission by memory and deadline; continuous batching.  capacity is the server's own
    calibration of this GPU (static tone-samples per second of a busy device, the direct render
    path); each chunk may be rendered `prefetch` chunk periods before it is due."""
    import math
    from paper_2403_15582_gb300 import workloads as wl
    srv = awg.Server(fs, 16 << 30, 256)
    srv.set_prefetch(prefetch)
    if engine:
        srv.set_static_engine(engine, engine_min_tones)
    capacity = srv.stats()["est_throughput"]
    mean_K = (10000 - 50) / math.log(10000 / 50)
    mean_chunk = sum(1 << e for e in range(16, 21)) / 5
    rate = rho * capacity / (mean_K * mean_chunk * 8)
    reqs = wl.served_requests(seed=0, rate_hz=rate, seconds=seconds, fs=fs)
    t0 = time.perf_counter()
    ids = []
    for r in reqs:
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(r.freq_hz, r.amp, r.phase_rad, r.chunk, r.n_chunks, r.chirps))
    srv.drain(120000)
    st = srv.stats()
    late = late_chunk_breakdown(srv)
    for rid in ids:
        srv.release(rid)
    srv.close()
    return {"fs_hz": fs, "rho": rho, "capacity": capacity, "prefetch_chunks": prefetch,
            "static_engine": ["direct", "gemm_fp16", "gemm_bf16"][engine],
            "engine_min_tones": engine_min_tones if engine else None,
            "engine_capacity": st["est_engine_throughput"] if engine else None, "arrival_rate_hz": rate,
            "seconds": seconds, "served_over_capacity": st["tone_samples_per_s"] / capacity,
            "requests": st["submitted"], "admitted": st["admitted"], "rejected_deadline": st["rejected_deadline"],
            "rejected_memory": st["rejected_memory"], "completed": st["completed"], "chunks": st["chunks"],
            "deadline_misses": st["deadline_misses"],
            "chunk_latency_ms": {"p50": st["latency_p50_ms"], "p99": st["latency_p99_ms"], "max": st["latency_max_ms"],
                                 "p99_of_playback": st["latency_p99_of_period"]},
            "first_chunk_ms": {"p50": st["first_chunk_p50_ms"], "p99": st["first_chunk_p99_ms"]},
            "samples_per_s": st["samples_per_s"], "tone_samples_per_s": st["tone_samples_per_s"],
            "mean_batch": st["mean_batch"], "max_batch": st["max_batch"], "rounds": st["rounds"], "busy_fraction": st["busy_fraction"],
            "est_throughput": st["est_throughput"],
            "est_round_cost_ms": st["est_round_cost_ms"], "est_cta_rate": st["est_cta_rate"],
            "late_chunks": late}


def config(wk, args):
    return {"workload": "chirp-1000tone-35ms-280MSps", "tones": wk.K, "samples": wk.n_samples, "chunk": wk.chunk,
            "fs_hz": wk.fs, "profiles": "linear (even tones) / minimum-jerk (odd tones)",
            "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-chirping", action="store_true")
    ap.add_argument("--no-table", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-static", action="store_true")
    ap.add_argument("--no-periodic", action="store_true")
    ap.add_argument("--no-profiles", action="store_true")
    ap.add_argument("--table-case", default="10000,24",
                    help="tones,log2 samples of the table leg (a smaller case for profiling)")
    args = ap.parse_args()
    wk = workload()
    if args.impl == "reference":
        return run_reference(args, wk)

    import numpy as np
    import torch
    import paper_2403_15582_gb300 as awg
    from paper_2403_15582_gb300 import build as awg_build
    awg_build.build()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_

    def barrier():
        if dist is not None:
            dist.barrier()

    N, chunk, K = wk.n_samples, wk.chunk, wk.K
    tone, f0, f1, dur, prof, start = wk.chirp_arrays()
    synth = awg.Synth(wk.fs)
    synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    synth.set_chirps(tone, f0, f1, dur, prof, start)
    out = torch.empty(N, dtype=torch.int16, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    n_full, tail = N // chunk, N % chunk

    def render_record(dst):
        # the chunk loop as one pipelined sequence of chunk renders, the short last chunk included
        synth.render_stream(N, chunk, dst, stream)

    def step_device():
        synth.seek(0)
        render_record(out)

    def step_chunkwise():
        synth.seek(0)
        for c0 in range(0, N, chunk):
            synth.render(min(chunk, N - c0), out[c0:], stream)

    for _ in range(args.warmup):
        flush.zero_()
        step_device()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = synth.launch_count
    # the library's profiling events split each step into the tile set-up and the span of the chunk
    # renders (which overlap one another) up to the join: the render kernel's own time
    synth.profile_begin()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step_device()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    sampler.stop()
    seq_prep_ms, seq_render_ms, _ = synth.profile_end()
    # our kernels in the timed steps (the library's own count): per group of chunks one chirp
    # set-up and one join, and one render per chunk
    launches = synth.launch_count - launches0
    # kernel split and per-chunk latency: the same chunks rendered one call at a time with the
    # library's profiling events (separately from the timed steps; events split the pipeline)
    synth.profile_begin()
    for i in range(args.steps):
        flush.zero_()
        step_chunkwise()
    torch.cuda.synchronize()
    prep_ms, render_ms, _ = synth.profile_end()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    work_per_step = K * N
    value = world * work_per_step * args.steps / (total_ms * 1e-3)
    status = synth.device_status()

    # e2e through the public API from host arrays into pinned host memory
    out_host = torch.empty(N, dtype=torch.int16, pin_memory=True)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        synth.seek(0)
        synth.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
        synth.set_chirps(tone, f0, f1, dur, prof, start)
        render_record(out_host)
        stream.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = max_over_ranks(sum(e2e_ms), dist, "cuda")
    record = out.cpu().numpy()   # the whole record (timed steps; the chunk-by-chunk pass wrote the same samples)
    e2e_same = bool(np.array_equal(record, out_host.numpy()))
    e2e_value = world * work_per_step * args.steps / (e2e_total * 1e-3)
    h2d = K * (2 * 96 + 208)     # 96-B tone records twice (set_tones, set_chirps) + 208-B chirp records

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (render): one SFU sine per tone-sample.  In the timed steps
    # the chunk renders overlap (pipelined sequence): their average launch duration times the
    # launches is the span from the end of the tile set-up to the join (library events on the
    # launching stream), so the kernel's rate is the step's sines over that span; over the whole
    # step (set-up and join included) it is a lower bound, reported beside it; the chunk-by-chunk
    # pass gives the rate of one render launch in isolation.
    achieved_step = K * N * args.steps / (total_ms * 1e-3) / 1e12
    render_span_ms = float(np.sum(seq_render_ms))
    achieved = K * N * args.steps / (render_span_ms * 1e-3) / 1e12 if render_span_ms > 0 else achieved_step
    chunk_sizes = [min(chunk, N - c0) for c0 in range(0, N, chunk)] * args.steps
    render_total_s = float(np.sum(render_ms)) * 1e-3
    achieved_isolated = K * float(np.sum(chunk_sizes)) / render_total_s / 1e12
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = sampler.summary()
    sm_max = clocks.get("sm_max_mhz") or SM_MAX_MHZ_DEFAULT
    peak = SFU_SIN_PER_CLK_SM * n_sm * sm_max * 1e6 / 1e12
    chunk_lat = np.asarray(prep_ms) + np.asarray(render_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_TONE_SAMPLES_PER_S, "dtype": "f32", "data": "synthetic",
        "config": config(wk, args),
        "max_realtime_tones_280MSps": value / world / 280e6,
        "output_msps": value / world / K / 1e6,
        "chunk_latency_ms": {"p50": float(np.percentile(chunk_lat, 50)), "p99": float(np.percentile(chunk_lat, 99)),
                             "playback_ms": 1e3 * chunk / wk.fs},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tsin/s",
                     "frac": achieved / peak, "traffic": RENDER_TRAFFIC_BYTES, "traffic_source": RENDER_TRAFFIC_SOURCE,
                     "kernel": "render_split_kernel",
                     "peak_source": f"16 SFU sin/clk/SM x {n_sm} SMs x {sm_max:g} MHz (nominal SFU rate, measured clock)",
                     "basis": "timed steps: sines / the span of the 38 overlapping chunk renders of each step "
                              "(CUDA events on the launching stream from the end of the tile set-up to the join)",
                     "render_span_ms_per_step": render_span_ms / args.steps,
                     "setup_ms_per_step": float(np.sum(seq_prep_ms)) / args.steps,
                     "whole_step": {"achieved": achieved_step, "frac": achieved_step / peak,
                                    "basis": "timed steps: sines / step time (set-up and join included)"},
                     "isolated_launch": {"achieved": achieved_isolated, "frac": achieved_isolated / peak,
                                         "basis": "chunk-by-chunk pass: sines / render kernel event time"},
                     "measured_sfu": sfu_probe(awg, stream, n_sm, achieved),
                     "measured_chirp_loop": sfu_probe(awg, stream, n_sm, achieved, probe=awg.chirp_rate_probe, what="chirp")},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 2 * N},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "device_status": status,
        "kernel_ms_per_step": {"prep": float(np.sum(prep_ms)) / args.steps,
                               "render": float(np.sum(render_ms)) / args.steps},
    }
    if not args.no_profiles:
        line["chirp_profiles"] = chirp_profile_leg(awg, stream, wk)
    if not args.no_static:
        line["static"] = static_leg(awg, stream)
    if not args.no_periodic:
        line["periodic"] = periodic_leg(awg, stream)
    if not args.no_table:
        tk, tl = (int(v) for v in args.table_case.split(","))
        line["table"] = table_leg(awg, stream, K=tk, log2_len=tl, gpu=local)
    if not args.no_served:
        line["served"] = {f"rho{r}": served_leg(awg, rho=r) for r in (0.5, 0.8, 1.0)}
        # requests of >= 1000 tones on the tensor-core static engine, at the same and at twice the
        # arrival rate (rho relative to the direct path's capacity)
        line["served_engine"] = {f"rho{r}": served_leg(awg, rho=r, engine=awg.STATIC_GEMM_FP16) for r in (1.0, 2.0)}
    if not args.no_stream:
        line["stream"] = {f"{int(fs_/1e6)}MSps": stream_leg(awg, fs_, stream) for fs_ in (280e6, 50e6)}
        line["stream"]["280MSps_gemm"] = stream_leg(awg, 280e6, stream, engine=awg.STATIC_GEMM_FP16)
    if not args.no_chirping:
        # the real-time target: 10,000 (and 11,000) tones all chirping at once at 280 MS/s; both
        # chunk sizes start with the same 7.5 ms of prefilled ring (2 chunks of 2^20, 8 of 2^18)
        line["chirping_10000_280MSps"] = {
            f"chunk_2^{c.bit_length() - 1}": chirping_leg(awg, stream, 10000, chunk=c, n_slots=2 * (1 << 20) // c + 1,
                                                          prefill=2 * (1 << 20) // c)
            for c in (1 << 20, 1 << 18)}
        line["chirping_11000_280MSps"] = {"chunk_2^20": chirping_leg(awg, stream, 11000, chunk=1 << 20)}
    if not args.no_cpu_baseline and world == 1:
        parity = {"e2e_output_equals_device_output": e2e_same}
        line["cpu_baseline"] = oracle_window_rate(wk, args.cpu_seconds, record=record, parity=parity)
        line["parity"] = parity
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
