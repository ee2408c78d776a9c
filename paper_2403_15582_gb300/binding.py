"""ctypes binding of libawg.so (include/awg.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libawg.so")

AWG_OK, AWG_EINVAL, AWG_ENOMEM, AWG_ECUDA, AWG_ETIMEOUT, AWG_EDEADLINE, AWG_ESTATE = 0, -1, -2, -3, -4, -5, -6
PREC_BF16, PREC_FP16 = 0, 1
SINE_SFU, SINE_ROTATOR = 0, 1
PERIODIC_DIRECT, PERIODIC_GEMM_BF16, PERIODIC_GEMM_FP16 = 0, 1, 2
STATIC_DIRECT, STATIC_GEMM_FP16, STATIC_GEMM_BF16 = 0, 1, 2
PROFILE_LINEAR, PROFILE_MINJERK, PROFILE_EXPONENTIAL = 0, 1, 2
NOALLOC_MAX_RECORDS, NOALLOC_MAX_SLOTS = 71493, 16384   # AWG_NOALLOC_MAX_RECORDS / _SLOTS of awg.h

# (name, restype, argtypes) of every symbol declared in include/awg.h
P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
SIGNATURES = [
    ("awg_version", ctypes.c_int, []),
    ("awg_last_error", ctypes.c_char_p, []),
    ("awg_freq_word", ctypes.c_int, [dbl, dbl, P]),
    ("awg_phase_word", ctypes.c_int, [dbl, P]),
    ("awg_grid_word", ctypes.c_int, [dbl, dbl, i32, P, P]),
    ("awg_chirp_length", ctypes.c_int, [dbl, dbl, P]),
    ("awg_chirp_coeffs", ctypes.c_int, [u64, u64, i64, i32, P]),
    ("awg_chirp_render_flags", ctypes.c_int, [u64, u64, i64, i32, P]),
    ("awg_create", P, [dbl]),
    ("awg_destroy", None, [P]),
    ("awg_set_tones", ctypes.c_int, [P, P, P, P, i32]),
    ("awg_set_tones_grid", ctypes.c_int, [P, P, i32, P, P, i32]),
    ("awg_set_chirps", ctypes.c_int, [P, P, P, P, P, P, P, i32]),
    ("awg_set_amp_ramps", ctypes.c_int, [P, P, P, P, P, P, i32]),
    ("awg_set_full_scale", ctypes.c_int, [P, dbl]),
    ("awg_full_scale", dbl, [P]),
    ("awg_sample_rate", dbl, [P]),
    ("awg_table_gemm", ctypes.c_int, [P, i32, i32, P, P, P]),
    ("awg_server_create", P, [dbl, i64, i32, dbl]),
    ("awg_server_destroy", None, [P]),
    ("awg_server_set_prefetch", ctypes.c_int, [P, i32]),
    ("awg_server_set_static_engine", ctypes.c_int, [P, i32, i32]),
    ("awg_server_submit", i64, [P, P]),
    ("awg_server_poll", ctypes.c_int, [P, i64, P, P]),
    ("awg_server_read", ctypes.c_int, [P, i64, P, i64]),
    ("awg_server_release", ctypes.c_int, [P, i64]),
    ("awg_server_drain", ctypes.c_int, [P, i32]),
    ("awg_server_stats", ctypes.c_int, [P, P]),
    ("awg_server_trace_rounds", i32, [P, P, i32]),
    ("awg_server_trace_chunks", i32, [P, P, i32]),
    ("awg_ring_create", P, [P, i64, i32]),
    ("awg_ring_destroy", None, [P]),
    ("awg_ring_push", ctypes.c_int, [P, P, i32]),
    ("awg_ring_start", ctypes.c_int, [P, i32, i64, P, i64]),
    ("awg_ring_finish", ctypes.c_int, [P, i32, P]),
    ("awg_ring_slot", P, [P, i32]),
    ("awg_seek", ctypes.c_int, [P, i64]),
    ("awg_cursor", i64, [P]),
    ("awg_set_sine_mode", ctypes.c_int, [P, i32]),
    ("awg_sine_mode", i32, [P]),
    ("awg_set_static_engine", ctypes.c_int, [P, i32]),
    ("awg_static_engine", i32, [P]),
    ("awg_set_periodic", ctypes.c_int, [P, i32, i32, P]),
    ("awg_periodic_start", i64, [P]),
    ("awg_clear_periodic", ctypes.c_int, [P]),
    ("awg_render", ctypes.c_int, [P, i64, P, P]),
    ("awg_render_f32", ctypes.c_int, [P, i64, P, P, P]),
    ("awg_render_chunks", ctypes.c_int, [P, i64, i32, P, P]),
    ("awg_render_stream", ctypes.c_int, [P, i64, i64, P, P]),
    ("awg_launch_count", i64, [P]),
    ("awg_render_multiplexed", ctypes.c_int, [P, i32, i64, P, P]),
    ("awg_phase_words", ctypes.c_int, [P, i64, P, i32]),
    ("awg_render_phases", ctypes.c_int, [P, i32, i64, i32, P]),
    ("awg_tone_split", i32, [P]),
    ("awg_last_render_ms", ctypes.c_float, [P]),
    ("awg_render_noalloc", ctypes.c_int, [P, i64, P, P]),
    ("awg_profile_begin", ctypes.c_int, [P]),
    ("awg_profile_end", ctypes.c_int, [P, P, P, i32, P]),
    ("awg_device_status", ctypes.c_int, [P]),
    ("awg_test_wait_timeout", ctypes.c_int, [P, i64, P]),
    ("awg_sfu_rate_probe", ctypes.c_int, [P, i32, i32, P]),
    ("awg_chirp_rate_probe", ctypes.c_int, [P, i32, i32, P]),
]

_lib = None


class AwgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"awg error {code}: {msg}")
        self.code = code


def lib():
    """Load libawg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2403_15582_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != AWG_OK:
        raise AwgError(code, lib().awg_last_error().decode())
    return code


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def freq_word(f_hz: float, fs: float) -> int:
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().awg_freq_word(float(f_hz), float(fs), _p(out)))
    return int(out[0])


def phase_word(theta: float) -> int:
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().awg_phase_word(float(theta), _p(out)))
    return int(out[0])


def grid_word(f_hz: float, fs: float, log2_len: int):
    out = np.zeros(1, dtype=np.uint64)
    j = np.zeros(1, dtype=np.int64)
    _check(lib().awg_grid_word(float(f_hz), float(fs), int(log2_len), _p(out), _p(j)))
    return int(out[0]), int(j[0])


def chirp_length(duration: float, fs: float) -> int:
    out = np.zeros(1, dtype=np.int64)
    _check(lib().awg_chirp_length(float(duration), float(fs), _p(out)))
    return int(out[0])


CHIRP_TABLE, CHIRP_LINEAR, CHIRP_EXP, CHIRP_FLAT3, CHIRP_LOW6, CHIRP_PAIR, CHIRP_LOW3 = 1, 2, 16, 32, 64, 128, 256


def chirp_render_flags(F_start: int, F_end: int, L: int, profile: int) -> int:
    """The render's flags of a chirp (host only): CHIRP_* bits, see awg_chirp_render_flags."""
    out = np.zeros(1, dtype=np.int32)
    _check(lib().awg_chirp_render_flags(int(F_start), int(F_end), int(L), int(profile), _p(out)))
    return int(out[0])


def chirp_coeffs(F_start: int, F_end: int, L: int, profile: int) -> list[int]:
    out = np.zeros(21, dtype=np.uint64)
    _check(lib().awg_chirp_coeffs(int(F_start), int(F_end), int(L), int(profile), _p(out)))
    return [int(out[3 * k]) | (int(out[3 * k + 1]) << 64) | (int(out[3 * k + 2]) << 128) for k in range(7)]


def sfu_rate_probe(out, blocks: int, runs: int, stream=None):
    """Launch the SFU-rate probe (the render's static loop alone): blocks x 128 x runs x 32 sines;
    `out` is a device float tensor of at least blocks x 128 elements."""
    _check(lib().awg_sfu_rate_probe(_ptr(out), int(blocks), int(runs), _stream_ptr(stream)))


def chirp_rate_probe(out, blocks: int, runs: int, stream=None):
    """Launch the chirp-loop rate probe (the render's chirp cascade alone): blocks x 128 x runs x 32
    sines; `out` is a device float tensor of at least blocks x 128 elements."""
    _check(lib().awg_chirp_rate_probe(_ptr(out), int(blocks), int(runs), _stream_ptr(stream)))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    if t is None:
        return ctypes.c_void_p(0)
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


class Synth:
    """One synthesiser handle (awg_t*).  Outputs are torch tensors (device or pinned host)."""

    def __init__(self, sample_rate: float):
        h = lib().awg_create(float(sample_rate))
        if not h:
            raise AwgError(AWG_ECUDA, lib().awg_last_error().decode())
        self._h = ctypes.c_void_p(h)
        self.fs = float(sample_rate)

    def close(self):
        if getattr(self, "_h", None):
            lib().awg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_tones(self, freq_hz, amp, phase_rad, grid_log2: int | None = None):
        f, a, ph = _f64(freq_hz), _f64(amp), _f64(phase_rad)
        if grid_log2:
            _check(lib().awg_set_tones_grid(self._h, _p(f), int(grid_log2), _p(a), _p(ph), int(f.size)))
        else:
            _check(lib().awg_set_tones(self._h, _p(f), _p(a), _p(ph), int(f.size)))

    def set_chirps(self, tone, f_start, f_end, duration, profile, start_sample):
        t = np.ascontiguousarray(np.asarray(tone, dtype=np.int32))
        f0, f1, du = _f64(f_start), _f64(f_end), _f64(duration)
        pr = np.ascontiguousarray(np.asarray(profile, dtype=np.int32))
        st = np.ascontiguousarray(np.asarray(start_sample, dtype=np.int64))
        _check(lib().awg_set_chirps(self._h, _p(t), _p(f0), _p(f1), _p(du), _p(pr), _p(st), int(t.size)))

    def set_chirp_list(self, chirps):
        if not chirps:
            return
        self.set_chirps([c["tone"] for c in chirps], [c["f_start"] for c in chirps], [c["f_end"] for c in chirps],
                        [c["duration"] for c in chirps], [c["profile"] for c in chirps],
                        [c.get("start_sample", 0) for c in chirps])

    def set_full_scale(self, v: float):
        _check(lib().awg_set_full_scale(self._h, float(v)))

    @property
    def full_scale(self) -> float:
        return float(lib().awg_full_scale(self._h))

    def seek(self, sample: int):
        _check(lib().awg_seek(self._h, int(sample)))

    @property
    def cursor(self) -> int:
        return int(lib().awg_cursor(self._h))

    @property
    def tone_split(self) -> int:
        return int(lib().awg_tone_split(self._h))

    def render(self, n: int, out, stream=None):
        _check(lib().awg_render(self._h, int(n), _ptr(out), _stream_ptr(stream)))

    def set_amp_ramps(self, tone, amp_end, duration_s, profile, start_sample):
        t = np.ascontiguousarray(tone, dtype=np.int32)
        a, d = _f64(amp_end), _f64(duration_s)
        p = np.ascontiguousarray(profile, dtype=np.int32)
        s0 = np.ascontiguousarray(start_sample, dtype=np.int64)
        _check(lib().awg_set_amp_ramps(self._h, _p(t), _p(a), _p(d), _p(p), _p(s0), int(t.size)))

    def set_ramp_list(self, ramps):
        """Ramps as dicts {tone, amp_end, duration, profile, start_sample}."""
        r = list(ramps)
        if r:
            self.set_amp_ramps([x["tone"] for x in r], [x["amp_end"] for x in r], [x["duration"] for x in r],
                               [x["profile"] for x in r], [x.get("start_sample", 0) for x in r])

    def set_sine_mode(self, mode: int):
        """SINE_SFU (default) or SINE_ROTATOR for static tone segments."""
        _check(lib().awg_set_sine_mode(self._h, int(mode)))

    @property
    def sine_mode(self) -> int:
        return int(lib().awg_sine_mode(self._h))

    def set_static_engine(self, engine: int):
        """STATIC_DIRECT (default), STATIC_GEMM_FP16 or STATIC_GEMM_BF16 for window-static tones."""
        _check(lib().awg_set_static_engine(self._h, int(engine)))

    @property
    def static_engine(self) -> int:
        return int(lib().awg_static_engine(self._h))

    def set_periodic(self, log2_len: int, method: int = 0, stream=None):
        """Periodic hand-off after the chirps (PERIODIC_DIRECT, PERIODIC_GEMM_BF16 / _FP16)."""
        _check(lib().awg_set_periodic(self._h, int(log2_len), int(method), _stream_ptr(stream)))

    @property
    def periodic_start(self) -> int:
        return int(lib().awg_periodic_start(self._h))

    def clear_periodic(self):
        _check(lib().awg_clear_periodic(self._h))

    def render_chunks(self, chunk: int, n_chunks: int, out, stream=None):
        """n_chunks consecutive chunks of `chunk` samples into out, as one pipelined sequence."""
        _check(lib().awg_render_chunks(self._h, int(chunk), int(n_chunks), _ptr(out), _stream_ptr(stream)))

    @property
    def launch_count(self) -> int:
        """Kernels this handle has launched so far."""
        return int(lib().awg_launch_count(self._h))

    def render_stream(self, n: int, chunk: int, out, stream=None):
        """n samples as pipelined chunks of `chunk` samples (the last one shorter)."""
        _check(lib().awg_render_stream(self._h, int(n), int(chunk), _ptr(out), _stream_ptr(stream)))

    def table_gemm(self, log2_len: int, precision: int, out_q=None, out_f=None, stream=None):
        _check(lib().awg_table_gemm(self._h, int(log2_len), int(precision), _ptr(out_q), _ptr(out_f), _stream_ptr(stream)))

    def render_noalloc(self, n: int, out, stream=None):
        _check(lib().awg_render_noalloc(self._h, int(n), _ptr(out), _stream_ptr(stream)))

    def render_f32(self, n: int, out_f32, out_q=None, stream=None):
        _check(lib().awg_render_f32(self._h, int(n), _ptr(out_f32), _ptr(out_q), _stream_ptr(stream)))

    def phase_words(self, sample: int, n: int) -> np.ndarray:
        out = np.zeros(n, dtype=np.uint64)
        _check(lib().awg_phase_words(self._h, int(sample), _p(out), int(n)))
        return out

    def render_phases(self, tone: int, n0: int, count: int) -> np.ndarray:
        out = np.zeros(count, dtype=np.uint32)
        _check(lib().awg_render_phases(self._h, int(tone), int(n0), int(count), _p(out)))
        return out

    def last_render_ms(self) -> float:
        return float(lib().awg_last_render_ms(self._h))

    def profile_begin(self):
        _check(lib().awg_profile_begin(self._h))

    def profile_end(self, cap: int = 1 << 16):
        """-> (prep_ms array, render_ms array, kernel launches) of the render calls since begin."""
        prep = np.zeros(cap, dtype=np.float32)
        rend = np.zeros(cap, dtype=np.float32)
        launches = np.zeros(1, dtype=np.int64)
        n = lib().awg_profile_end(self._h, _p(prep), _p(rend), int(cap), _p(launches))
        if n < 0:
            _check(n)
        n = min(n, cap)
        return prep[:n].copy(), rend[:n].copy(), int(launches[0])

    def device_status(self) -> int:
        v = lib().awg_device_status(self._h)
        return int(v)

    def test_wait_timeout(self, limit_us: int, stream=None):
        _check(lib().awg_test_wait_timeout(self._h, int(limit_us), _stream_ptr(stream)))


class RingStats(ctypes.Structure):
    _fields_ = [("played", ctypes.c_int64), ("underruns", ctypes.c_int64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double), ("lead_min_ms", ctypes.c_double),
                ("lead_p50_ms", ctypes.c_double), ("chunk_playback_ms", ctypes.c_double), ("checksum", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def render_multiplexed(synths, n: int, out, stream=None):
    """Interleave n samples of each Synth's channel into out[i * len(synths) + c]."""
    arr = (ctypes.c_void_p * len(synths))(*[s._h.value for s in synths])
    _check(lib().awg_render_multiplexed(arr, len(synths), int(n), _ptr(out), _stream_ptr(stream)))


class Ring:
    """Streaming ring of pinned host chunk slots fed by a Synth and drained by a sink thread."""

    def __init__(self, synth: Synth, chunk: int, n_slots: int):
        r = lib().awg_ring_create(synth.handle, int(chunk), int(n_slots))
        if not r:
            raise AwgError(AWG_EINVAL, lib().awg_last_error().decode())
        self._r = ctypes.c_void_p(r)
        self.synth = synth
        self.chunk = int(chunk)
        self.n_slots = int(n_slots)

    def close(self):
        if getattr(self, "_r", None):
            lib().awg_ring_destroy(self._r)
            self._r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, stream=None, timeout_ms: int = 10000):
        _check(lib().awg_ring_push(self._r, _stream_ptr(stream), int(timeout_ms)))

    def start(self, prefill: int, n_chunks: int, capture: np.ndarray | None = None):
        cap_p = _p(capture) if capture is not None else ctypes.c_void_p(0)
        cap_n = int(capture.size) if capture is not None else 0
        self._capture = capture
        _check(lib().awg_ring_start(self._r, int(prefill), int(n_chunks), cap_p, cap_n))

    def finish(self, timeout_ms: int = 60000) -> dict:
        st = RingStats()
        _check(lib().awg_ring_finish(self._r, int(timeout_ms), ctypes.byref(st)))
        return st.as_dict()

    def slot(self, i: int) -> np.ndarray:
        ptr = lib().awg_ring_slot(self._r, int(i))
        if not ptr:
            raise AwgError(AWG_EINVAL, "slot index out of range")
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_int16)), shape=(self.chunk,)).copy()


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_REJECTED = 0, 1, 2, 3


class _Request(ctypes.Structure):
    _fields_ = [("freq_hz", P), ("amp", P), ("phase_rad", P), ("n_tones", i32), ("chirp_tone", P),
                ("chirp_f_start_hz", P), ("chirp_f_end_hz", P), ("chirp_duration_s", P), ("chirp_profile", P),
                ("chirp_start_sample", P), ("n_chirps", i32), ("chunk", i64), ("n_chunks", i32), ("full_scale", dbl)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", i64), ("admitted", i64), ("rejected_deadline", i64), ("rejected_memory", i64),
                ("completed", i64), ("chunks", i64), ("deadline_misses", i64), ("latency_p50_ms", dbl),
                ("latency_p99_ms", dbl), ("latency_max_ms", dbl), ("latency_p99_of_period", dbl),
                ("first_chunk_p50_ms", dbl),
                ("first_chunk_p99_ms", dbl), ("rounds", i64), ("mean_batch", dbl), ("max_batch", i64),
                ("tone_samples_per_s", dbl), ("samples_per_s", dbl), ("busy_fraction", dbl), ("est_throughput", dbl),
                ("est_round_cost_ms", dbl), ("est_cta_rate", dbl), ("est_engine_throughput", dbl)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Server:
    """Served request stream (continuous batching) on the current device."""

    def __init__(self, sample_rate: float, mem_budget_bytes: int = 8 << 30, max_active: int = 64,
                 max_queue_ms: float = 5.0):
        h = lib().awg_server_create(float(sample_rate), int(mem_budget_bytes), int(max_active), float(max_queue_ms))
        if not h:
            raise AwgError(AWG_EINVAL, lib().awg_last_error().decode())
        self._s = ctypes.c_void_p(h)
        self.fs = float(sample_rate)

    def close(self):
        if getattr(self, "_s", None):
            lib().awg_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_prefetch(self, chunks: int):
        _check(lib().awg_server_set_prefetch(self._s, int(chunks)))

    def set_static_engine(self, engine: int, min_tones: int):
        _check(lib().awg_server_set_static_engine(self._s, int(engine), int(min_tones)))

    def submit(self, freq_hz, amp, phase_rad, chunk: int, n_chunks: int, chirps=(), full_scale: float = 0.0) -> int:
        f, a, th = _f64(freq_hz), _f64(amp), _f64(phase_rad)
        ch = list(chirps)
        ct = np.ascontiguousarray([c["tone"] for c in ch], dtype=np.int32)
        c0 = _f64([c["f_start"] for c in ch])
        c1 = _f64([c["f_end"] for c in ch])
        cd = _f64([c["duration"] for c in ch])
        cp = np.ascontiguousarray([c["profile"] for c in ch], dtype=np.int32)
        cs = np.ascontiguousarray([c.get("start_sample", 0) for c in ch], dtype=np.int64)
        q = _Request(_p(f).value, _p(a).value, _p(th).value, int(f.size), _p(ct).value, _p(c0).value, _p(c1).value,
                     _p(cd).value, _p(cp).value, _p(cs).value, len(ch), int(chunk), int(n_chunks), float(full_scale))
        rid = lib().awg_server_submit(self._s, ctypes.byref(q))
        if rid < 0:
            _check(int(rid))
        return int(rid)

    def poll(self, rid: int):
        st = np.zeros(1, dtype=np.int32)
        done = np.zeros(1, dtype=np.int32)
        _check(lib().awg_server_poll(self._s, int(rid), _p(st), _p(done)))
        return int(st[0]), int(done[0])

    def read(self, rid: int, n_samples: int) -> np.ndarray:
        out = np.zeros(n_samples, dtype=np.int16)
        _check(lib().awg_server_read(self._s, int(rid), _p(out), int(n_samples)))
        return out

    def release(self, rid: int):
        _check(lib().awg_server_release(self._s, int(rid)))

    def drain(self, timeout_ms: int = 60000):
        _check(lib().awg_server_drain(self._s, int(timeout_ms)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().awg_server_stats(self._s, ctypes.byref(st)))
        return st.as_dict()

    ROUND_DTYPE = np.dtype([("t_plan", "f8"), ("t_issued", "f8"), ("t_start", "f8"), ("t_done", "f8"),
                            ("work", "f8"), ("first_due", "f8"), ("pieces", "i4"), ("tiles", "i4")])
    CHUNK_DTYPE = np.dtype([("id", "i8"), ("chunk", "i4"), ("late", "i4"), ("release", "f8"), ("due", "f8"),
                            ("done", "f8")])

    def trace_rounds(self, cap: int = 1 << 16) -> np.ndarray:
        """The most recent rounds (structured array, ROUND_DTYPE)."""
        out = np.zeros(cap, dtype=self.ROUND_DTYPE)
        n = lib().awg_server_trace_rounds(self._s, out.ctypes.data, int(cap))
        if n < 0:
            _check(int(n))
        return out[:n]

    def trace_chunks(self, cap: int = 1 << 16) -> np.ndarray:
        """The most recent chunk completions (structured array, CHUNK_DTYPE)."""
        out = np.zeros(cap, dtype=self.CHUNK_DTYPE)
        n = lib().awg_server_trace_chunks(self._s, out.ctypes.data, int(cap))
        if n < 0:
            _check(int(n))
        return out[:n]
