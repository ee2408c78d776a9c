"""CPU oracle for multi-tone additive synthesis -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import this package.  The product library (``paper_2403_15582_gb300``)
never imports, links or calls it, and the two share no code.

Paper: Tu & Subhankar, "Fast real-time arbitrary waveform generation using graphic processing
units" (IEEE TSP 2025).  Every function cites the passage it follows.

Exactness model.  Phase is an integer word in units of 2^-64 turn.  Static tones step by a
frequency word F; chirps are produced by a cascade of seven 192-bit accumulators whose initial
values d_k are the exact forward differences of the chirp-phase polynomial, times 2^128,
rounded half-to-even (``chirp_coefficients``).  The arithmetic is in ``awg_oracle.c``; this
module derives the inputs with Python integers and ``fractions.Fraction`` (exact).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` against closed
forms, the paper's own equations evaluated in exact rationals, brute force and invariants.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from fractions import Fraction
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "awg_oracle.c")

MASK64 = (1 << 64) - 1
MASK192 = (1 << 192) - 1
PROFILE_LINEAR = 0
PROFILE_MINJERK = 1
PROFILE_EXPONENTIAL = 2
MAX_CHIRP_SAMPLES = (1 << 28) - 1


# --------------------------------------------------------------------------------------------
# build / load
# --------------------------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile awg_oracle.c into liboracle.so with the host gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", _LIB_PATH, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        L.oracle_render.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, i64, i64, P, ctypes.c_int, P, P, P, P, P]
        L.oracle_render.restype = ctypes.c_int
        L.oracle_render_work_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_render_work_bytes.restype = ctypes.c_size_t
        L.oracle_render_at.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, P, i64, P, ctypes.c_int, P, P, P, P, P]
        L.oracle_amp_at.argtypes = [dbl, i32, i64, i64, dbl, P, i64, P]
        L.oracle_amp_at.restype = None
        L.oracle_render_at.restype = None
        L.oracle_phase_words_seq.argtypes = [u64, u64, i32, i64, i64, P, u64, i64, i64, P]
        L.oracle_phase_words_at.argtypes = [u64, u64, i32, i64, i64, P, u64, P, i64, P]
        L.oracle_cascade_at.argtypes = [P, i64, P]
        L.oracle_chirp_end_word.argtypes = [u64, u64, i32, i64, i64, P]
        L.oracle_chirp_end_word.restype = u64
        L.oracle_quantize.argtypes = [P, i64, dbl, P]
        _lib = L
    return _lib


# --------------------------------------------------------------------------------------------
# a1: tone set-up, Hz -> words
# --------------------------------------------------------------------------------------------
def freq_word(f_hz: float, fs: float) -> int:
    """F = rint(f/fs * 2^64) mod 2^64: the per-sample phase step of a tone of frequency f.

    Eq. main (Sec. II) writes the tone as sin(2*pi*f*t + theta) with t = i/f_s; in turns the
    per-sample increment is f/f_s, held here as a 64-bit fixed-point word (round half to even,
    IEEE double division)."""
    r = float(f_hz) / float(fs)
    return int(round(math.ldexp(r, 64))) & MASK64


def phase_word(theta_rad: float) -> int:
    """Phi0 = rint(frac(theta/2pi) * 2^64) mod 2^64: the initial phase theta_j of Eq. main."""
    t = float(theta_rad) / (2.0 * math.pi)
    frac = t - math.floor(t)
    return int(round(math.ldexp(frac, 64))) & MASK64


def grid_index(f_hz: float, fs: float, log2_len: int) -> int:
    """j = nint(f/f_s * L_s) of Eq. freqapprox (Sec. II), ties to even."""
    return int(round(math.ldexp(float(f_hz) / float(fs), log2_len)))


def grid_word(j: int, log2_len: int) -> int:
    """F of the grid tone j/L_s * f_s (Eq. freqapprox): exactly j * 2^(64 - log2 L)."""
    return (int(j) << (64 - log2_len)) & MASK64


def chirp_length(duration_s: float, fs: float) -> int:
    """L = round-half-even(T * f_s): the chirp spans samples m = 0..L (Eq. freqchirp case 1,
    0 <= i <= T f_s)."""
    return int(round(float(duration_s) * float(fs)))


# --------------------------------------------------------------------------------------------
# a2: chirp set-up -- exact polynomial, forward differences, 2^128-scaled words
# --------------------------------------------------------------------------------------------
def _signed_diff(F_end: int, F_start: int) -> int:
    """D = F_end - F_start as a true integer (both words lie in [0, 2^64))."""
    return int(F_end) - int(F_start)


def chirp_phase_poly(F_start: int, F_end: int, L: int, profile: int):
    """Return P(m), the chirp phase in words relative to the chirp start, as an exact rational
    function of the integer sample offset m (0 <= m <= L).

    min-jerk (Eq. freqchirp case 1): phi[i] = 2 pi i/f_s (f_start + p[i]),
    p[i] = (f_fin - f_start)(5/2 tau^3 - 3 tau^4 + tau^5), tau = i/(T f_s).  In words, with
    L = T f_s and D = F_end - F_start:  P(m) = F_start m + D (5 m^4 L^2 - 6 m^5 L + 2 m^6)/(2 L^5).
    linear (named in Sec. II, formula not printed): the integral of a linear frequency ramp,
    P(m) = F_start m + D m^2 / (2 L)."""
    D = _signed_diff(F_end, F_start)
    Fs_ = int(F_start)
    if profile == PROFILE_MINJERK:
        def P(m: int) -> Fraction:
            return Fs_ * m + Fraction(D * (5 * m**4 * L**2 - 6 * m**5 * L + 2 * m**6), 2 * L**5)
    elif profile == PROFILE_LINEAR:
        def P(m: int) -> Fraction:
            return Fs_ * m + Fraction(D * m * m, 2 * L)
    else:
        raise ValueError("unknown profile")
    return P


def chirp_coefficients(F_start: int, F_end: int, L: int, profile: int) -> list[int]:
    """d_0..d_6 as integers mod 2^192 (Q64.128 two's complement).

    c_k = Delta^k P(0) (exact forward differences of the degree-<=6 phase polynomial, so that
    P(m) = sum_k c_k C(m,k) exactly); d_k = round_half_even(c_k * 2^128) mod 2^192 for k >= 1,
    and d_0 = 2^127 (P(0) = 0 plus the offset that makes the top 64 bits round to nearest)."""
    if not (1 <= L <= MAX_CHIRP_SAMPLES):
        raise ValueError("chirp length out of range")
    P = chirp_phase_poly(F_start, F_end, L, profile)
    vals = [P(m) for m in range(7)]
    d = [1 << 127]
    for k in range(1, 7):
        ck = sum(((-1) ** (k - j)) * math.comb(k, j) * vals[j] for j in range(k + 1))
        d.append(round(ck * (1 << 128)) & MASK192)
    return d


def chirp_state(F_start: int, F_end: int, L: int, profile: int):
    """(has_chirp, d) of a chirp for the C oracle.  Polynomial profiles: (1, d_0..d_6).
    Exponential (named in Sec. II, formula not printed; see exp_offset in awg_oracle.c): (2, d)
    with d_0 = F_start and d_1 = F_end, which must both be > 0 (the frequency ratio)."""
    if profile == PROFILE_EXPONENTIAL:
        if not (1 <= L <= MAX_CHIRP_SAMPLES):
            raise ValueError("chirp length out of range")
        if F_start <= 0 or F_end <= 0:
            raise ValueError("an exponential chirp needs f_start, f_end > 0")
        return 2, [int(F_start), int(F_end), 0, 0, 0, 0, 0]
    return 1, chirp_coefficients(F_start, F_end, L, profile)


def cascade_state(d: Sequence[int], m: int) -> list[int]:
    """acc_k(m) = sum_{i>=k} d_i C(m, i-k) mod 2^192: the cascade after m steps (exact skip)."""
    return [sum(d[i] * math.comb(m, i - k) for i in range(k, 7)) & MASK192 for k in range(7)]


def limbs192(v: int) -> list[int]:
    v &= MASK192
    return [v & MASK64, (v >> 64) & MASK64, (v >> 128) & MASK64]


# --------------------------------------------------------------------------------------------
# waveform description
# --------------------------------------------------------------------------------------------
@dataclass
class Waveform:
    """Per-tone integer state, as the oracle sees it (all words are Python ints)."""

    fs: float
    F: list = field(default_factory=list)          # static frequency word
    phi_ref: list = field(default_factory=list)    # static phase word at sample 0
    A: list = field(default_factory=list)          # amplitude (FP64)
    has_chirp: list = field(default_factory=list)
    n_s: list = field(default_factory=list)
    L: list = field(default_factory=list)
    d: list = field(default_factory=list)          # 7 ints mod 2^192 (zeros if no chirp)
    F_end: list = field(default_factory=list)
    # amplitude ramps a_k(n) (Eq. dynamicandstatic): tone -> (profile, a_ns, a_L, A_end)
    ramps: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return len(self.F)

    def ramp_arrays(self):
        """(ramp pairs, a_ns, a_L, A_end) for the C oracle, or Nones without ramps."""
        if not self.ramps:
            return None, None, None, None
        K = self.K
        rp = np.zeros(2 * K, dtype=np.int32)
        ns = np.zeros(K, dtype=np.int64)
        L = np.zeros(K, dtype=np.int64)
        Ae = np.array(self.A, dtype=np.float64)
        for k, (prof, a_ns, a_L, A_end) in self.ramps.items():
            rp[2 * k], rp[2 * k + 1] = 1, int(prof)
            ns[k], L[k], Ae[k] = int(a_ns), int(a_L), float(A_end)
        return rp, ns, L, Ae

    def full_scale(self) -> float:
        """Default full scale: sum |A_k|, which can never clip."""
        return float(sum(abs(a) for a in self.A))

    def arrays(self):
        K = self.K
        F = np.array(self.F, dtype=np.uint64)
        phi = np.array(self.phi_ref, dtype=np.uint64)
        A = np.array(self.A, dtype=np.float64)
        hc = np.array(self.has_chirp, dtype=np.int32)
        ns = np.array(self.n_s, dtype=np.int64)
        L = np.array(self.L, dtype=np.int64)
        d = np.zeros((K, 21), dtype=np.uint64)
        for k in range(K):
            if self.has_chirp[k]:
                d[k] = np.array(sum((limbs192(v) for v in self.d[k]), []), dtype=np.uint64)
        Fe = np.array(self.F_end, dtype=np.uint64)
        return F, phi, A, hc, ns, L, d, Fe


def make_waveform(fs: float, freq_hz, amp, phase_rad, chirps=None, grid_log2: Optional[int] = None) -> Waveform:
    """Build the oracle's tone state from Hz / radians.

    chirps: optional list of dicts {tone, f_start, f_end, duration, profile, start_sample}.
    The chirp starts from the tone's phase word at start_sample (the phase offset theta_j is
    propagated from the initial waveform, Eq. dynamicandstatic); after it, the tone is static at
    f_end with the phase reached at m = L (Eq. freqchirp case 2).  With grid_log2 the static
    frequencies are snapped to the f_s / 2^grid_log2 grid (Eq. freqapprox)."""
    w = Waveform(fs=float(fs))
    K = len(freq_hz)
    for k in range(K):
        if grid_log2 is None:
            w.F.append(freq_word(freq_hz[k], fs))
        else:
            w.F.append(grid_word(grid_index(freq_hz[k], fs, grid_log2), grid_log2))
        w.phi_ref.append(phase_word(phase_rad[k]))
        w.A.append(float(amp[k]))
        w.has_chirp.append(0)
        w.n_s.append(0)
        w.L.append(0)
        w.d.append([0] * 7)
        w.F_end.append(0)
    for c in chirps or []:
        k = int(c["tone"])
        Fs_ = freq_word(c["f_start"], fs)
        Fe_ = freq_word(c["f_end"], fs)
        L = chirp_length(c["duration"], fs)
        w.has_chirp[k], w.d[k] = chirp_state(Fs_, Fe_, L, int(c["profile"]))
        w.n_s[k] = int(c.get("start_sample", 0))
        w.L[k] = L
        w.F_end[k] = Fe_
    return w


# --------------------------------------------------------------------------------------------
# rendering
# --------------------------------------------------------------------------------------------
def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pn(a):
    return None if a is None else _p(a)


def render(w: Waveform, n0: int, N: int, nthreads: int = 1) -> np.ndarray:
    """x[n] for n = n0 .. n0+N-1 in FP64 (Eq. dynamicandstatic: sum of A_k sin(phi_k[n]))."""
    L_ = lib()
    F, phi, A, hc, ns, Lc, d, Fe = w.arrays()
    out = np.zeros(N, dtype=np.float64)
    if N == 0:
        return out
    work = np.zeros(L_.oracle_render_work_bytes(w.K, nthreads), dtype=np.uint8)
    rp, ans, aL, Ae = w.ramp_arrays()
    used = L_.oracle_render(w.K, _p(F), _p(phi), _p(A), _p(hc), _p(ns), _p(Lc), _p(d), _p(Fe),
                            int(n0), int(N), _p(out), int(nthreads), _p(work), _pn(rp), _pn(ans), _pn(aL), _pn(Ae))
    render.last_threads = used
    return out


render.last_threads = 1


def render_at(w: Waveform, samples, nthreads: int = 1) -> np.ndarray:
    """x[n] at arbitrary absolute sample indices, each from the closed-form phase."""
    L_ = lib()
    F, phi, A, hc, ns, Lc, d, Fe = w.arrays()
    idx = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
    out = np.zeros(idx.size, dtype=np.float64)
    if idx.size == 0:
        return out
    work = np.zeros(L_.oracle_render_work_bytes(w.K, 1), dtype=np.uint8)
    rp, ans, aL, Ae = w.ramp_arrays()
    L_.oracle_render_at(w.K, _p(F), _p(phi), _p(A), _p(hc), _p(ns), _p(Lc), _p(d), _p(Fe),
                        _p(idx), int(idx.size), _p(out), int(nthreads), _p(work), _pn(rp), _pn(ans), _pn(aL), _pn(Ae))
    return out


def amp_at(A: float, profile: int, a_ns: int, a_L: int, A_end: float, samples) -> np.ndarray:
    """Amplitude of one ramping tone at the given samples (the oracle's a(n))."""
    idx = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
    out = np.zeros(idx.size, dtype=np.float64)
    lib().oracle_amp_at(float(A), int(profile), int(a_ns), int(a_L), float(A_end), _p(idx), int(idx.size), _p(out))
    return out


def add_ramps(w: Waveform, ramps, fs: Optional[float] = None) -> Waveform:
    """Attach amplitude ramps [{tone, amp_end, duration, profile, start_sample}] to a waveform; a
    ramp moves the tone's amplitude from its value A_k to amp_end over L = rint(duration fs)
    samples (the same length rule as a chirp).  One ramp per tone."""
    fs = w.fs if fs is None else fs
    for r in ramps:
        w.ramps[int(r["tone"])] = (int(r["profile"]), int(r.get("start_sample", 0)), chirp_length(r["duration"], fs),
                                   float(r["amp_end"]))
    return w


def quantize(x: np.ndarray, FS: float) -> np.ndarray:
    """int16 DAC code: clamp(rint(x * 32767/FS), -32767, 32767), ties to even."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size, dtype=np.int16)
    lib().oracle_quantize(_p(x), int(x.size), float(FS), _p(out))
    return out


def _tone_args(w: Waveform, k: int):
    d = np.array(sum((limbs192(v) for v in w.d[k]), []), dtype=np.uint64)
    return (w.F[k], w.phi_ref[k], int(w.has_chirp[k]), int(w.n_s[k]), int(w.L[k]), d, w.F_end[k])


def phase_words_seq(w: Waveform, k: int, n0: int, N: int) -> np.ndarray:
    """Phase words of tone k for n0..n0+N-1, produced by sequential stepping (the definition)."""
    F, phi, hc, ns, L, d, Fe = _tone_args(w, k)
    out = np.zeros(N, dtype=np.uint64)
    lib().oracle_phase_words_seq(F, phi, hc, ns, L, _p(d), Fe, int(n0), int(N), _p(out))
    return out


def phase_words_at(w: Waveform, k: int, samples) -> np.ndarray:
    """Phase words of tone k at arbitrary samples, by the closed form."""
    F, phi, hc, ns, L, d, Fe = _tone_args(w, k)
    idx = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
    out = np.zeros(idx.size, dtype=np.uint64)
    lib().oracle_phase_words_at(F, phi, hc, ns, L, _p(d), Fe, _p(idx), int(idx.size), _p(out))
    return out


def cascade_state_c(d: Sequence[int], m: int) -> list[int]:
    """The C oracle's closed-form cascade state (7 ints mod 2^192), for cross-checks."""
    arr = np.array(sum((limbs192(v) for v in d), []), dtype=np.uint64)
    out = np.zeros(21, dtype=np.uint64)
    lib().oracle_cascade_at(_p(arr), int(m), _p(out))
    return [int(out[3 * k]) | (int(out[3 * k + 1]) << 64) | (int(out[3 * k + 2]) << 128) for k in range(7)]


def chirp_end_word(w: Waveform, k: int) -> int:
    """Phi at the last chirp sample m = L (the post-chirp anchor of Eq. freqchirp case 2)."""
    F, phi, hc, ns, L, d, Fe = _tone_args(w, k)
    return int(lib().oracle_chirp_end_word(F, phi, hc, ns, L, _p(d)))


def make_waveform_window(fs: float, freq_hz, amp, phase_rad, chirps, n0: int, N: int) -> Waveform:
    """Waveform state for the window [n0, n0+N) when tones chirp several times.

    Each tone's chirps are applied in time order; a chirp that ends before n0 is folded into the
    tone's static state (the tone continues at f_end from the phase reached at the chirp's end,
    Eq. freqchirp case 2), and the chirp overlapping the window (at most one per tone) is kept."""
    w = make_waveform(fs, freq_hz, amp, phase_rad)
    by_tone = {}
    for c in chirps:
        by_tone.setdefault(int(c["tone"]), []).append(c)
    for k, lst in by_tone.items():
        lst.sort(key=lambda c: c.get("start_sample", 0))
        for c in lst:
            Fs_ = freq_word(c["f_start"], fs)
            Fe_ = freq_word(c["f_end"], fs)
            L = chirp_length(c["duration"], fs)
            ns = int(c.get("start_sample", 0))
            if ns >= n0 + N:
                break
            if w.has_chirp[k]:   # fold the previous chirp
                end = chirp_end_word(w, k)
                n_e = w.n_s[k] + w.L[k]
                w.F[k] = w.F_end[k]
                w.phi_ref[k] = (end - n_e * w.F_end[k]) % (1 << 64)
                w.has_chirp[k] = 0
            w.has_chirp[k], w.d[k] = chirp_state(Fs_, Fe_, L, int(c["profile"]))
            w.n_s[k], w.L[k] = ns, L
            w.F_end[k] = Fe_
            if ns + L >= n0:
                break
    return w
