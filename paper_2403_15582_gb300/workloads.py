"""Seeded synthetic inputs for the five workload shapes (tones in Hz, amplitudes, phases, chirps).

This module holds input recipes only: it draws random numbers and lays out parameter lists.
It computes no phase words, no sines and no sums -- both the CUDA library and the CPU oracle
receive exactly these Hz / radian / second values and do their own set-up.

Shapes follow the paper's workloads (Sec. V): AOD-band tone combs with Schroeder-style phases,
chirps along linear or minimum-jerk profiles (Eq. freqchirp), tweezer-rearrangement requests
(Sec. V-B) and groups of tones chirped in turn (Streaming pathway).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LINEAR = 0
MINJERK = 1


@dataclass
class Workload:
    name: str
    fs: float
    freq_hz: np.ndarray
    amp: np.ndarray
    phase_rad: np.ndarray
    chirps: list = field(default_factory=list)   # dicts: tone, f_start, f_end, duration, profile, start_sample
    n_samples: int = 0
    chunk: int = 0
    grid_log2: int | None = None                  # snap static tones to f_s / 2^grid_log2 (Eq. freqapprox)
    full_scale: float | None = None               # None: sum |A|

    @property
    def K(self) -> int:
        return int(self.freq_hz.size)

    def chirp_arrays(self):
        """Chirps as parallel arrays in the order the C ABI takes them."""
        n = len(self.chirps)
        tone = np.array([c["tone"] for c in self.chirps], dtype=np.int32).reshape(n)
        fs0 = np.array([c["f_start"] for c in self.chirps], dtype=np.float64).reshape(n)
        fs1 = np.array([c["f_end"] for c in self.chirps], dtype=np.float64).reshape(n)
        dur = np.array([c["duration"] for c in self.chirps], dtype=np.float64).reshape(n)
        prof = np.array([c["profile"] for c in self.chirps], dtype=np.int32).reshape(n)
        start = np.array([c.get("start_sample", 0) for c in self.chirps], dtype=np.int64).reshape(n)
        return tone, fs0, fs1, dur, prof, start


def schroeder_quadratic(K: int) -> np.ndarray:
    """Quadratic (Schroeder) phases theta_k = -pi k^2 / K for low crest factor (Sec. II cites
    Schroeder for crest-factor control; the formula itself is not printed in the paper)."""
    k = np.arange(K, dtype=np.float64)
    return -math.pi * k * k / K


def static_100(seed: int = 0, n_samples: int = 1 << 20) -> Workload:
    """100 static tones on a 1 MHz grid from 80 to 179 MHz, amplitude 1/100, uniform phases,
    f_s = 280 MS/s, 2^20 samples."""
    rng = np.random.default_rng(seed)
    K = 100
    f = 80e6 + 1e6 * np.arange(K, dtype=np.float64)
    A = np.full(K, 1.0 / K)
    th = rng.uniform(0.0, 2.0 * math.pi, K)
    return Workload("static-100tone-2^20", 280e6, f, A, th, [], n_samples, n_samples)


def chirp_1000(seed: int = 0, K: int = 1000, duration: float = 35e-3, chunk: int = 1 << 18,
               fs: float = 280e6) -> Workload:
    """1000 tones, each ramping from a seeded start frequency to a seeded target in 80-180 MHz
    over 35 ms at 280 MS/s (9.8M samples); even tones linear, odd tones minimum-jerk;
    amplitudes U[0.5, 1]/1000, uniform phases; output in 2^18-sample chunks."""
    rng = np.random.default_rng(seed)
    f0 = rng.uniform(80e6, 180e6, K)
    f1 = rng.uniform(80e6, 180e6, K)
    A = rng.uniform(0.5, 1.0, K) / K
    th = rng.uniform(0.0, 2.0 * math.pi, K)
    chirps = [dict(tone=k, f_start=float(f0[k]), f_end=float(f1[k]), duration=duration,
                   profile=(LINEAR if k % 2 == 0 else MINJERK), start_sample=0) for k in range(K)]
    n = int(round(duration * fs))
    return Workload(f"chirp-{K}tone-{duration*1e3:g}ms", fs, f0.copy(), A, th, chirps, n, chunk)


def table_10000(seed: int = 0, K: int = 10000, log2_len: int = 24) -> Workload:
    """10,000 static tones on a 10 kHz grid in 80-180 MHz, snapped to the f_s/2^24 record grid
    (Eq. freqapprox), amplitudes U[0.5, 1], quadratic Schroeder phases; record 2^24 samples;
    full scale = max |x| over the record (passed in by the caller once known)."""
    rng = np.random.default_rng(seed)
    f = 80e6 + 1e4 * np.arange(K, dtype=np.float64)
    A = rng.uniform(0.5, 1.0, K)
    th = schroeder_quadratic(K)
    return Workload(f"table-{K}tone-2^{log2_len}", 280e6, f, A, th, [], 1 << log2_len, 1 << log2_len,
                    grid_log2=log2_len)


def stream_rotating(seed: int = 0, fs: float = 280e6, K: int = 10000, group: int = 100,
                    ramp_s: float = 1e-3, seconds: float = 1.0, chunk: int = 1 << 20) -> Workload:
    """10,000 grid tones (10 kHz grid in 80-180 MHz at 280 MS/s; 2 kHz grid in 2-22 MHz at 50 MS/s,
    whose band the Nyquist limit forces), amplitude 1/10,000.  In millisecond m, group m mod 100
    ramps linearly over 1 ms from its current frequency to a new seeded grid frequency."""
    rng = np.random.default_rng(seed)
    if fs >= 200e6:
        f_lo, step = 80e6, 1e4
    else:
        f_lo, step = 2e6, 2e3
    slots = np.arange(K)
    f = f_lo + step * slots.astype(np.float64)
    A = np.full(K, 1.0 / K)
    th = rng.uniform(0.0, 2.0 * math.pi, K)
    cur = f.copy()
    chirps = []
    n_ms = int(round(seconds / ramp_s))
    L = int(round(ramp_s * fs))
    ngroups = K // group
    for m in range(n_ms):
        g = m % ngroups
        tones = np.arange(g * group, (g + 1) * group)
        targets = f_lo + step * rng.integers(0, K, size=group).astype(np.float64)
        for t, ft in zip(tones, targets):
            chirps.append(dict(tone=int(t), f_start=float(cur[t]), f_end=float(ft), duration=ramp_s,
                               profile=LINEAR, start_sample=m * L))
            cur[t] = ft
    n = int(round(seconds * fs))
    return Workload(f"stream-{K}tone-{fs/1e6:g}MSps", fs, f, A, th, chirps, n, chunk)


def chirping_stream(seed: int = 0, K: int = 10000, fs: float = 280e6, segments: int = 7,
                    segment_samples: int = 9 << 20) -> Workload:
    """K tones that all chirp all the time: in segment s (samples s S .. (s+1) S - 1, S = 9 x 2^20,
    33.7 ms at 280 MS/s) every tone ramps from its current frequency to a new seeded target in
    80-180 MHz over L = S - 1 samples, so the next chirp starts at the next segment's first sample
    (a chirp spans m = 0..L).  Even tones linear, odd tones minimum-jerk; amplitudes U[0.5, 1]/K,
    uniform phases: the 1000-tone 35 ms chirp shape at K tones, continued indefinitely."""
    rng = np.random.default_rng(seed)
    cur = rng.uniform(80e6, 180e6, K)
    f0 = cur.copy()
    A = rng.uniform(0.5, 1.0, K) / K
    th = rng.uniform(0.0, 2.0 * math.pi, K)
    L = segment_samples - 1
    chirps = []
    for seg in range(segments):
        tgt = rng.uniform(80e6, 180e6, K)
        for k in range(K):
            chirps.append(dict(tone=k, f_start=float(cur[k]), f_end=float(tgt[k]), duration=L / fs,
                               profile=(LINEAR if k % 2 == 0 else MINJERK), start_sample=seg * segment_samples))
        cur = tgt
    n = segments * segment_samples
    return Workload(f"chirping-{K}tone-{fs/1e6:g}MSps", fs, f0, A, th, chirps, n, 1 << 20)


@dataclass
class Request:
    """One tweezer-rearrangement request (Sec. V-B): a static comb with some tones chirped."""
    rid: int
    arrival_s: float
    fs: float
    freq_hz: np.ndarray
    amp: np.ndarray
    phase_rad: np.ndarray
    chirps: list
    chunk: int
    n_chunks: int


def served_requests(seed: int = 0, rate_hz: float = 100.0, seconds: float = 10.0, fs: float = 280e6,
                    n_chunks: int = 8, max_tones: int = 10000, min_tones: int = 50) -> list[Request]:
    """Poisson arrivals at rate_hz for `seconds`; tones log-uniform in [50, 10,000] on a 10 kHz
    grid in 80-180 MHz with half of the comb positions empty (50 % loading); up to 100 tones chirp
    over 0.1-2 ms (linear / minimum-jerk 50/50) to seeded band frequencies; chunk 2^U{16..20};
    each request streams n_chunks consecutive chunks."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= seconds:
            break
        K = int(round(math.exp(rng.uniform(math.log(min_tones), math.log(max_tones)))))
        slots = np.sort(rng.choice(20000, size=K, replace=False))
        f = 80e6 + 5e3 * slots.astype(np.float64)
        A = np.full(K, 1.0 / K)
        th = rng.uniform(0.0, 2.0 * math.pi, K)
        nch = int(rng.integers(0, min(100, K) + 1))
        ch_t = rng.choice(K, size=nch, replace=False) if nch else np.zeros(0, dtype=np.int64)
        chirps = []
        for tone in ch_t:
            dur = float(rng.uniform(0.1e-3, 2e-3))
            chirps.append(dict(tone=int(tone), f_start=float(f[tone]), f_end=float(80e6 + 5e3 * rng.integers(0, 20000)),
                               duration=dur, profile=int(rng.integers(0, 2)), start_sample=0))
        chunk = 1 << int(rng.integers(16, 21))
        out.append(Request(rid, t, fs, f, A, th, chirps, chunk, n_chunks))
        rid += 1
    return out


def tiny(seed: int = 0, K: int = 3, fs: float = 280e6, n_samples: int = 4096, chirp: bool = True) -> Workload:
    """A few tones, optionally with short chirps that start and end inside the record."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(1e6, 139e6, K)
    A = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(-math.pi, math.pi, K)
    chirps = []
    if chirp:
        for k in range(K):
            if k % 3 == 2:
                continue
            L0 = int(rng.integers(50, n_samples // 2))
            chirps.append(dict(tone=k, f_start=float(rng.uniform(1e6, 139e6)), f_end=float(rng.uniform(1e6, 139e6)),
                               duration=L0 / fs, profile=k % 2, start_sample=int(rng.integers(0, n_samples // 2))))
    return Workload(f"tiny-{K}", fs, f, A, th, chirps, n_samples, n_samples)
