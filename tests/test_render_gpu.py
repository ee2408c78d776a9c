"""GPU parity: the CUDA render path against the CPU oracle, called through the C ABI.

Bars: phase words bit-exact; int16 codes within 1 LSB of the oracle's FP64 sum quantised in FP64;
the FP32 sum within a bound derived from the arithmetic (per-tone sine/argument error plus FP32
summation), written out in `fp32_bound`."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
TWO64 = 1 << 64


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def synth_from(awg, wk):
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=wk.grid_log2)
    s.set_chirp_list(wk.chirps)
    return s


def oracle_from(oracle, wk):
    return oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, grid_log2=wk.grid_log2)


def render(s, n, f32=True):
    q = torch.empty(max(n, 1), dtype=torch.int16, device="cuda")
    if f32:
        x = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        s.render_f32(n, x, q)
        torch.cuda.synchronize()
        return q[:n].cpu().numpy(), x[:n].cpu().numpy()
    s.render(n, q)
    torch.cuda.synchronize()
    return q[:n].cpu().numpy(), None


def fp32_bound(amps, split):
    """|x_gpu - x_exact| bound: per tone <= 5e-6 |A| (SFU sine 2^-21.4, 23-bit argument, FP32
    argument scaling, in-run phase cascade <= 2500 * 2^-32 turn), plus FP32 summation of
    K/split + split terms (each rounding <= 2^-24 of the running sum, bounded by sum |A|)."""
    K = len(amps)
    S = sum(abs(a) for a in amps)
    return S * (5e-6 + (K / max(split, 1) + split + 2) * 2.0**-24)


def check(q, x, w, oracle, x_ref, split):
    FS = w.full_scale()
    q_ref = oracle.quantize(x_ref, FS)
    dq = np.abs(q.astype(np.int32) - q_ref.astype(np.int32))
    assert dq.max(initial=0) <= 1, f"max LSB error {dq.max()}"
    if x is not None:
        err = np.max(np.abs(x.astype(np.float64) - x_ref), initial=0.0)
        assert err <= fp32_bound(w.A, split), (err, fp32_bound(w.A, split))
    return float(np.mean(dq == 0)) if dq.size else 1.0


def _sdiff32(a, b):
    d = (np.asarray(a, dtype=np.int64) - np.asarray(b, dtype=np.int64)) % (1 << 32)
    return np.where(d >= 1 << 31, d - (1 << 32), d)


# ---------------------------------------------------------------------------------------------
def test_static_100_full_record(awg, oracle):
    """100 static tones, 2^20 samples: the whole record, FP32 and int16."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.static_100(seed=0)
    s = synth_from(awg, wk)
    w = oracle_from(oracle, wk)
    q, x = render(s, wk.n_samples)
    x_ref = oracle.render(w, 0, wk.n_samples, nthreads=NTHREADS)
    frac = check(q, x, w, oracle, x_ref, s.tone_split)
    assert frac > 0.9
    assert s.device_status() == 0


def test_phase_words_bit_exact(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    for seed in range(4):
        wk = wl.tiny(seed=seed, K=9, n_samples=20000)
        s = synth_from(awg, wk)
        w = oracle_from(oracle, wk)
        samples = {0, 1, 4095, 4096, 19999, 1 << 30, (1 << 40) + 3}
        for c in wk.chirps:
            L = oracle.chirp_length(c["duration"], wk.fs)
            ns = c["start_sample"]
            samples |= {max(ns - 1, 0), ns, ns + 1, ns + L // 2, ns + L - 1, ns + L, ns + L + 1}
        for n in sorted(samples):
            got = s.phase_words(n, w.K)
            for k in range(w.K):
                assert int(got[k]) == int(oracle.phase_words_at(w, k, [n])[0]), (seed, n, k)


def test_phase_words_long_chirps(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.chirp_1000(seed=1, K=64)
    s = synth_from(awg, wk)
    w = oracle_from(oracle, wk)
    rng = np.random.default_rng(0)
    L = wk.n_samples
    for n in [0, 1, L - 1, L, L + 1, L + 12345] + list(rng.integers(0, L, 12)):
        got = s.phase_words(int(n), w.K)
        ref = [int(oracle.phase_words_at(w, k, [int(n)])[0]) for k in range(w.K)]
        assert [int(g) for g in got] == ref, n


@pytest.mark.parametrize("dur_ms", [0.1, 0.5, 2.0, 35.0])
def test_render_phase_cascade_within_bound(awg, oracle, dur_ms):
    """The 32-bit phases the kernel feeds to the sine stay within the stated bound of the exact
    words: 2500 units of 2^-32 turn for minimum-jerk runs (g, h rounding over 31 steps of a
    32-sample run; or, where two lanes share a run set-up and a cascade spans 63 steps, f and g
    rounding over 63 steps plus the neglected third order and the left-out LOW6 or LOW3 terms,
    31.5 + 976.5 + 512 + 269), 1100 for linear chirps (f and g rounding over 63 steps: 31.5 + 976.5), 40 for static
    segments.  Tones 0 and 2 (minimum-jerk) and 1 and 4 (linear) form the render's lane pairs
    where their chirps allow it, so both roles of a shared set-up are traced."""
    fs = 280e6
    L = int(round(dur_ms * 1e-3 * fs))
    f = [90e6, 100e6, 120e6, 60e6, 70e6]
    A = [1, 1, 1, 1, 1]
    th = [0.1, 0.2, 0.3, 0.4, 0.5]
    s = awg.Synth(fs)
    s.set_tones(f, A, th)
    ns = 5000
    chirps = [dict(tone=0, f_start=90e6, f_end=179e6, duration=L / fs, profile=1, start_sample=ns),
              dict(tone=1, f_start=100e6, f_end=1e6, duration=L / fs, profile=0, start_sample=ns + 17),
              dict(tone=2, f_start=125e6, f_end=80e6, duration=L / fs, profile=1, start_sample=ns + 4096),
              dict(tone=4, f_start=70e6, f_end=150e6, duration=L / fs, profile=0, start_sample=ns + 33)]
    s.set_chirp_list(chirps)
    w = oracle.make_waveform(fs, f, A, th, chirps)
    for n0 in (0, ns + L // 2 - 30000, ns + L - 20000):
        n0 = max(n0, 0)
        cnt = 60000
        idx = np.arange(n0, n0 + cnt, dtype=np.int64)
        for k, bound in ((0, 2500), (1, 1100), (2, 2500), (3, 40), (4, 1100)):
            got = s.render_phases(k, n0, cnt)
            words = oracle.phase_words_at(w, k, idx)
            ref = ((words.astype(object) + (1 << 40)) >> 32) % (1 << 32)
            d = np.abs(_sdiff32(got.astype(np.int64), np.array(ref, dtype=np.int64)))
            assert d.max() <= bound, (dur_ms, n0, k, int(d.max()))


def test_tiny_waveforms_all_samples(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    for seed in range(6):
        wk = wl.tiny(seed=seed, K=5, n_samples=9000 + 777 * seed)
        s = synth_from(awg, wk)
        w = oracle_from(oracle, wk)
        q, x = render(s, wk.n_samples)
        x_ref = oracle.render(w, 0, wk.n_samples)
        check(q, x, w, oracle, x_ref, s.tone_split)


def test_chirp_1000_windows(awg, oracle):
    """1000 chirping tones (35 ms at 280 MS/s): windows at the start, the middle and across the
    chirp end, with ragged lengths; each compared sample by sample with the oracle."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.chirp_1000(seed=0)
    s = synth_from(awg, wk)
    w = oracle_from(oracle, wk)
    L = wk.n_samples
    for n0, cnt in ((0, 3 * 4096 + 123), (L // 2 - 4000, 9001), (L - 6000, 12345)):
        s.seek(n0)
        q, x = render(s, cnt)
        x_ref = oracle.render(w, n0, cnt, nthreads=NTHREADS)
        check(q, x, w, oracle, x_ref, s.tone_split)


def test_chirp_1000_full_record_sampled(awg, oracle):
    """The full 9.8M-sample record rendered in 2^18-sample chunks, as the benchmark does, checked
    at sampled indices with the oracle's closed form."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.chirp_1000(seed=0)
    s = synth_from(awg, wk)
    w = oracle_from(oracle, wk)
    N = wk.n_samples
    q = torch.empty(N, dtype=torch.int16, device="cuda")
    for c0 in range(0, N, wk.chunk):
        s.render(min(wk.chunk, N - c0), q[c0:])
    torch.cuda.synchronize()
    qh = q.cpu().numpy()
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, N, 700), [0, 1, N - 1, wk.chunk - 1, wk.chunk]]))
    x_ref = oracle.render_at(w, idx, nthreads=NTHREADS)
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(qh[idx].astype(np.int32) - q_ref)) <= 1
    assert s.device_status() == 0


def test_chunk_invariance_bit_exact(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=7, K=40, n_samples=30000)
    s = synth_from(awg, wk)
    q1, x1 = render(s, 30000)
    s.seek(0)
    parts = [1, 4095, 4097, 7, 11800, 30000 - 1 - 4095 - 4097 - 7 - 11800]
    qs, xs = [], []
    for p in parts:
        q, x = render(s, p)
        qs.append(q)
        xs.append(x)
    assert np.array_equal(np.concatenate(qs), q1)
    assert np.array_equal(np.concatenate(xs), x1)
    assert s.cursor == 30000


def test_render_chunks_pipelined_equals_chunk_by_chunk(awg, oracle):
    """A pipelined sequence of chunk renders (overlapping on the device) writes the same int16
    samples as the chunks rendered one call at a time, across two sequences in a row (the record
    buffers alternate), interleaved with plain renders, and with chunks where no chirp is active
    (no set-up kernel); spot-checked against the oracle."""
    rng = np.random.default_rng(21)
    K, fs, chunk = 300, 280e6, 1 << 16
    f = rng.uniform(80e6, 180e6, K)
    a = rng.uniform(0.5, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(80e6, 180e6)),
                   duration=float(rng.uniform(0.2e-3, 1.2e-3)), profile=int(t % 2), start_sample=int(rng.integers(0, 200000)))
              for t in rng.choice(K, 120, replace=False)]
    n_chunks = 9                  # chirps end by sample ~540k; the last chunks hold none
    total = 2 * n_chunks * chunk + 4096 + 2 * chunk

    def make():
        s = awg.Synth(fs)
        s.set_tones(f, a, th)
        s.set_chirp_list(chirps)
        return s

    ref = torch.empty(total, dtype=torch.int16, device="cuda")
    s = make()
    for c0 in range(0, total, chunk):
        s.render(min(chunk, total - c0), ref[c0:])
    got = torch.full((total,), 12345, dtype=torch.int16, device="cuda")
    s2 = make()
    s2.render_chunks(chunk, n_chunks, got)
    s2.render_chunks(chunk, n_chunks, got[n_chunks * chunk:])
    s2.render(4096, got[2 * n_chunks * chunk:])
    s2.render_chunks(chunk, 2, got[2 * n_chunks * chunk + 4096:])
    torch.cuda.synchronize()
    assert s2.device_status() == 0 and s2.cursor == total
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.array_equal(r, g)   # chunk invariance: the chunking differs, the samples do not
    # awg_render_stream: chunks that do not divide the window, the short last one in the sequence
    s3 = make()
    got3 = torch.full((total,), 12345, dtype=torch.int16, device="cuda")
    before = s3.launch_count
    s3.render_stream(123_457, 50_000, got3)
    s3.render_stream(total - 123_457, 70_001, got3[123_457:])
    torch.cuda.synchronize()
    assert s3.device_status() == 0 and s3.cursor == total
    assert np.array_equal(r, got3.cpu().numpy())
    assert s3.launch_count - before >= 3 + (total - 123_457 + 70_000) // 70_001
    w = oracle.make_waveform_window(fs, f, a, th, chirps, 0, total)
    idx = np.unique(rng.integers(0, total, 400))
    q_ref = oracle.quantize(oracle.render_at(w, idx, nthreads=NTHREADS), w.full_scale())
    assert np.max(np.abs(g[idx].astype(np.int32) - q_ref)) <= 1
    # profiling mode: a sequence stays pipelined and records one call (set-up, then the span of its
    # renders), with the same samples
    s4 = make()
    got4 = torch.full((total,), 12345, dtype=torch.int16, device="cuda")
    s4.profile_begin()
    before = s4.launch_count
    s4.render_stream(total, 70_001, got4)
    torch.cuda.synchronize()
    prep_ms, rend_ms, launches = s4.profile_end()
    assert len(prep_ms) == 1 and len(rend_ms) == 1 and prep_ms[0] > 0 and rend_ms[0] > 0
    assert launches == s4.launch_count - before >= 3
    assert np.array_equal(r, got4.cpu().numpy())


@pytest.mark.parametrize("K", [1, 63, 64, 65, 129, 1000, 2000])
def test_tone_split_sizes(awg, oracle, K):
    rng = np.random.default_rng(K)
    f = rng.uniform(0, 280e6, K)
    a = rng.uniform(-1, 1, K)
    th = rng.uniform(0, 6.3, K)
    s = awg.Synth(280e6)
    s.set_tones(f, a, th)
    w = oracle.make_waveform(280e6, f, a, th)
    s.seek(12345)
    q, x = render(s, 5000)
    check(q, x, w, oracle, oracle.render(w, 12345, 5000, nthreads=NTHREADS), s.tone_split)


def test_edge_cases(awg, oracle):
    fs = 280e6
    s = awg.Synth(fs)
    # no tones: silence
    s.set_tones([], [], [])
    q, x = render(s, 5000)
    assert not q.any() and not x.any()
    # n = 0 is a no-op
    s.render(0, None)
    assert s.cursor == 5000
    # DC, Nyquist, an aliased tone above fs/2, negative amplitude, far-out sample index
    f = [0.0, fs / 2, 200e6, 13e6]
    a = [0.25, 0.5, -0.75, 1.0]
    th = [0.3, 1.1, 2.0, -0.5]
    s.set_tones(f, a, th)
    w = oracle.make_waveform(fs, f, a, th)
    for n0 in (0, 7, (1 << 40) + 5):
        s.seek(n0)
        q, x = render(s, 4100)
        check(q, x, w, oracle, oracle.render(w, n0, 4100), s.tone_split)
    # explicit full scale that clips
    s.set_full_scale(0.5)
    s.seek(0)
    q, _ = render(s, 2000, f32=False)
    assert q.max() <= 32767 and q.min() >= -32767
    ref = oracle.quantize(oracle.render(w, 0, 2000), 0.5)
    assert np.max(np.abs(q.astype(np.int32) - ref)) <= 1


def test_exact_path_for_very_fast_chirps(awg, oracle):
    """Chirps so short that the in-run cubic cascade would not be accurate use the exact
    per-sample closed form; output still within 1 LSB."""
    fs = 280e6
    f = [50e6, 70e6, 90e6]
    s = awg.Synth(fs)
    s.set_tones(f, [1, 1, 1], [0, 1, 2])
    chirps = [dict(tone=0, f_start=50e6, f_end=130e6, duration=300 / fs, profile=1, start_sample=100),
              dict(tone=1, f_start=70e6, f_end=10e6, duration=2 / fs, profile=1, start_sample=4090),
              dict(tone=2, f_start=90e6, f_end=95e6, duration=1 / fs, profile=0, start_sample=33)]
    s.set_chirp_list(chirps)
    w = oracle.make_waveform(fs, f, [1, 1, 1], [0, 1, 2], chirps)
    q, x = render(s, 9000)
    check(q, x, w, oracle, oracle.render(w, 0, 9000), s.tone_split)


def test_chirp_sequence_on_one_tone(awg, oracle):
    """A second chirp on a tone, set after the first has been rendered, continues from the first
    chirp's end state."""
    fs = 280e6
    s = awg.Synth(fs)
    s.set_tones([80e6, 100e6], [0.5, 0.5], [0.0, 1.0])
    c1 = dict(tone=0, f_start=80e6, f_end=120e6, duration=5000 / fs, profile=1, start_sample=1000)
    s.set_chirp_list([c1])
    q1, x1 = render(s, 10000)
    c2 = dict(tone=0, f_start=120e6, f_end=60e6, duration=3000 / fs, profile=0, start_sample=12000)
    s.set_chirp_list([c2])
    q2, x2 = render(s, 10000)
    # oracle: second chirp applied to the folded state of the first
    w = oracle.make_waveform(fs, [80e6, 100e6], [0.5, 0.5], [0.0, 1.0], [c1])
    x_ref1 = oracle.render(w, 0, 10000)
    Fe = w.F_end[0]
    end = oracle.chirp_end_word(w, 0)
    n_e = c1["start_sample"] + w.L[0]
    w.F[0] = Fe
    w.phi_ref[0] = (end - n_e * Fe) % TWO64
    L2 = oracle.chirp_length(c2["duration"], fs)
    w.has_chirp[0], w.n_s[0], w.L[0] = 1, c2["start_sample"], L2
    w.d[0] = oracle.chirp_coefficients(oracle.freq_word(120e6, fs), oracle.freq_word(60e6, fs), L2, 0)
    w.F_end[0] = oracle.freq_word(60e6, fs)
    x_ref2 = oracle.render(w, 10000, 10000)
    check(q1, x1, w, oracle, x_ref1, s.tone_split)
    check(q2, x2, w, oracle, x_ref2, s.tone_split)


def test_set_chirps_validation(awg):
    fs = 280e6
    s = awg.Synth(fs)
    s.set_tones([80e6, 90e6], [1, 1], [0, 0])
    s.set_chirps([0], [80e6], [90e6], [1e-3], [1], [100])
    bad = [
        dict(tone=[5], f0=[80e6], f1=[90e6], d=[1e-3], p=[0], st=[0]),          # tone out of range
        dict(tone=[1, 1], f0=[80e6] * 2, f1=[90e6] * 2, d=[1e-3] * 2, p=[0, 0], st=[0, 10**6]),   # twice in one call
        dict(tone=[0], f0=[80e6], f1=[90e6], d=[1e-3], p=[0], st=[10**7]),      # pending chirp on tone 0
        dict(tone=[1], f0=[80e6], f1=[290e6], d=[1e-3], p=[0], st=[0]),         # f_end >= fs
        dict(tone=[1], f0=[80e6], f1=[90e6], d=[0.0], p=[0], st=[0]),           # zero length
        dict(tone=[1], f0=[80e6], f1=[90e6], d=[1e-3], p=[3], st=[0]),          # bad profile
    ]
    for b in bad:
        with pytest.raises(awg.AwgError) as e:
            s.set_chirps(b["tone"], b["f0"], b["f1"], b["d"], b["p"], b["st"])
        assert e.value.code == awg.AWG_EINVAL
    q = torch.empty(1000, dtype=torch.int16, device="cuda")
    s.render(1000, q)
    with pytest.raises(awg.AwgError):
        s.set_chirps([1], [80e6], [90e6], [1e-3], [0], [10])     # starts before the cursor


def test_maximum_sizes(awg, oracle):
    """Large tone counts (65,536 tones: 4096 per CTA of a 16-CTA cluster) far into the stream, and
    one render call of more than 2^30 samples (output offsets beyond 2^31 bytes), each checked at
    sampled indices against the oracle's closed form."""
    rng = np.random.default_rng(77)
    fs = 280e6
    K = 65536
    f = rng.uniform(0, fs, K)
    a = rng.uniform(-1, 1, K) / 256
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.uniform(1e-3, 5e-3)), profile=int(t % 2), start_sample=(1 << 33) + int(rng.integers(0, 200000)))
              for t in rng.choice(K, 1000, replace=False)]
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    s.seek(1 << 33)
    s.set_chirp_list(chirps)
    n = 1 << 20
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, q)
    torch.cuda.synchronize()
    assert s.device_status() == 0 and s.tone_split == 16
    w = oracle.make_waveform(fs, f, a, th, chirps)
    idx = np.unique(rng.integers(0, n, 200))
    x_ref = oracle.render_at(w, (1 << 33) + idx, nthreads=NTHREADS)
    xs = x.cpu().numpy()[idx].astype(np.float64)
    assert np.max(np.abs(xs - x_ref)) <= fp32_bound(a, 16)
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(q.cpu().numpy()[idx].astype(np.int32) - q_ref)) <= 1

    # one call of 2^30 + 4097 samples (2 GiB of int16)
    f2, a2, th2 = [12.5e6, 77.77e6, 133e6], [0.5, -0.3, 0.2], [0.1, 0.2, 0.3]
    s2 = awg.Synth(fs)
    s2.set_tones(f2, a2, th2)
    N = (1 << 30) + 4097
    big = torch.empty(N, dtype=torch.int16, device="cuda")
    s2.render(N, big)
    torch.cuda.synchronize()
    assert s2.device_status() == 0 and s2.cursor == N
    w2 = oracle.make_waveform(fs, f2, a2, th2)
    idx2 = np.unique(np.concatenate([rng.integers(0, N, 100), rng.integers(N - (1 << 20), N, 100), [N - 1, 1 << 30]]))
    q2 = oracle.quantize(oracle.render_at(w2, idx2, nthreads=NTHREADS), w2.full_scale())
    got = big[torch.as_tensor(idx2, device="cuda")].cpu().numpy().astype(np.int32)
    assert np.max(np.abs(got - q2)) <= 1
    del big


def test_split_sums_across_launches(awg, oracle):
    """A window of more than 512 tiles with a tone split of 16 goes out in several render launches
    chained by programmatic dependent launch on alternating scratch buffers: the same samples as
    chunk-by-chunk and pipelined rendering, bit for bit, and within 1 LSB of the oracle."""
    rng = np.random.default_rng(91)
    fs, K = 280e6, 1600
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.uniform(1e-3, 8e-3)), profile=int(t % 3), start_sample=int(rng.integers(0, 2_000_000)))
              for t in rng.choice(K, 300, replace=False)]

    def make():
        s = awg.Synth(fs)
        s.set_tones(f, a, th)
        s.set_chirp_list(chirps)
        return s

    n = 1200 * 4096 + 777              # 1201 tiles: three launches of at most 512
    s = make()
    assert s.tone_split == 16
    one = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, one)
    s2 = make()
    cut = torch.empty(n, dtype=torch.int16, device="cuda")
    c = 0
    for piece in (100_001, 3 * 1 << 20, 4096):
        s2.render(piece, cut[c:])
        c += piece
    s2.render_stream(n - c, 1 << 18, cut[c:])
    torch.cuda.synchronize()
    assert s.device_status() == 0 and s2.device_status() == 0
    q1 = one.cpu().numpy()
    assert np.array_equal(q1, cut.cpu().numpy())
    w = oracle.make_waveform(fs, f, a, th, chirps)
    idx = np.unique(np.concatenate([rng.integers(0, n, 300), [0, 512 * 4096 - 1, 512 * 4096, 1024 * 4096, n - 1]]))
    x_ref = oracle.render_at(w, idx, nthreads=NTHREADS)
    assert np.max(np.abs(x.cpu().numpy()[idx].astype(np.float64) - x_ref)) <= fp32_bound(a, 16)
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(q1[idx].astype(np.int32) - q_ref)) <= 1


@pytest.mark.parametrize("mode", [0, 1])
def test_chirp_boundaries_in_every_lane(awg, oracle, mode):
    """Chirp starts and ends at every run position of a tile (every lane of the four warps), at
    the first, second and last sample of a run, with both ends in one run (lengths 1..31), in
    adjacent runs, warps and tiles; linear, minimum-jerk and exponential profiles; a few tones
    ramping through the same tiles.  Every sample against the oracle, both sine variants, with a
    tone split of 3."""
    fs = 280e6
    K = 200
    rng = np.random.default_rng(11)
    f = rng.uniform(5e6, 135e6, K)
    a = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(0, 2 * np.pi, K)
    lengths = (1, 2, 5, 31, 32, 33, 64, 95, 4095, 4096, 4097, 20000)
    offsets = (0, 1, 31)
    chirps = []
    for k in range(160):
        lane = (k * 37) % 128
        n_s = 4096 * (1 + k % 40) + 32 * lane + offsets[k % 3]
        L = lengths[k % len(lengths)]
        prof = k % 3
        chirps.append(dict(tone=k, f_start=float(f[k]), f_end=float(rng.uniform(1e6, 139e6)),
                           duration=L / fs, profile=prof, start_sample=int(n_s)))
    ramps = [dict(tone=int(t), amp_end=0.3 * float(a[t]), duration=5000 / fs, profile=int(t % 2),
                  start_sample=int(4096 * (3 + t % 30) + 17 * t)) for t in range(150, 200, 2)]
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    s.set_chirp_list(chirps)
    s.set_amp_ramps([r["tone"] for r in ramps], [r["amp_end"] for r in ramps], [r["duration"] for r in ramps],
                    [r["profile"] for r in ramps], [r["start_sample"] for r in ramps])
    s.set_sine_mode(mode)
    assert s.tone_split == 3
    w = oracle.add_ramps(oracle.make_waveform(fs, f, a, th, chirps), ramps)
    n = 4096 * 43
    q, x = render(s, n)
    assert s.device_status() == 0
    check(q, x, w, oracle, oracle.render(w, 0, n, nthreads=NTHREADS), s.tone_split)


def test_sfu_rate_probe_runs(awg):
    """The SFU-rate probe (the render's static loop alone) writes one finite float per thread and
    refuses bad arguments."""
    blocks, runs = 8, 4
    out = torch.full((blocks * 128,), float("nan"), dtype=torch.float32, device="cuda")
    awg.sfu_rate_probe(out, blocks, runs)
    torch.cuda.synchronize()
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.max(np.abs(v)) <= runs * 32 * 1e-3 * 1.0001
    with pytest.raises(awg.AwgError):
        awg.sfu_rate_probe(out, 0, runs)
    with pytest.raises(awg.AwgError):
        awg.sfu_rate_probe(None, blocks, runs)


def test_chirp_rate_probe_runs(awg):
    """The chirp-loop rate probe (the render's chirp cascade alone) writes one finite float per
    thread and refuses bad arguments."""
    blocks, runs = 8, 4
    out = torch.full((blocks * 128,), float("nan"), dtype=torch.float32, device="cuda")
    awg.chirp_rate_probe(out, blocks, runs)
    torch.cuda.synchronize()
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.max(np.abs(v)) <= runs * 32 * 1e-3 * 1.0001
    with pytest.raises(awg.AwgError):
        awg.chirp_rate_probe(out, blocks, 0)
    with pytest.raises(awg.AwgError):
        awg.chirp_rate_probe(None, blocks, runs)
