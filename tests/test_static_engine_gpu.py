"""The tensor-core static engine: in each 4096-sample tile the tones that are static there (either
segment of a chirped tone, constant amplitude) are summed by the split-precision table GEMM (rows of
256 samples aligned to absolute indices), the rest by the render kernel, which adds the GEMM's FP32
sum before quantising.  Parity against the oracle (int16 within 1 LSB, FP32
within the GEMM's and the render's bounds), for static combs at any frequency far into the stream
and for windows where chirps and amplitude ramps run beside static tones; the same samples
however the stream is cut into calls."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
FS = 280e6


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


# The engine's FP32 sum against the FP64 oracle, in LSB of the handle's full scale.  Its error is
# the table GEMM's (tensor-core FP32 accumulation and the hi + lo residual, random walks over the
# tones; see the table GEMM tests) plus, for the tones the render kernel sums, the SFU sine and the
# FP32 sum of the render (below 1e-5 of sum |A|): far below a quarter of an LSB at these sizes,
# while a systematic error of one LSB breaks the bound.
FP32_BOUND_LSB = 0.25


def fp32_lsb(x, x_ref, FS):
    return float(np.max(np.abs(x.astype(np.float64) - x_ref))) / (FS / 32767.0)


def render(s, n, n0=None):
    if n0 is not None:
        s.seek(n0)
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, q)
    torch.cuda.synchronize()
    assert s.device_status() == 0
    return q.cpu().numpy(), x.cpu().numpy()


@pytest.mark.parametrize("engine", [1, 2])
def test_static_comb_any_frequency_far_into_the_stream(awg, oracle, engine):
    rng = np.random.default_rng(engine)
    K = 500
    f = rng.uniform(0, FS, K)
    a = rng.uniform(-1, 1, K)
    th = rng.uniform(0, 2 * np.pi, K)
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_static_engine(engine)
    assert s.static_engine == engine
    n0, n = (1 << 35) + 123, 100_001
    q, x = render(s, n, n0)
    w = oracle.make_waveform(FS, f, a, th)
    x_ref = oracle.render(w, n0, n, nthreads=NTHREADS)
    err = fp32_lsb(x, x_ref, w.full_scale())
    assert err <= FP32_BOUND_LSB, err
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(q.astype(np.int32) - q_ref)) <= 1


def test_hybrid_window_with_chirps_and_ramps(awg, oracle):
    rng = np.random.default_rng(5)
    K = 300
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.integers(2000, 30000)) / FS, profile=int(t % 2),
                   start_sample=int(rng.integers(0, 40000))) for t in rng.choice(K, 40, replace=False)]
    ramps = [dict(tone=int(t), amp_end=float(rng.uniform(0, 1)), duration=float(rng.integers(500, 20000)) / FS,
                  profile=int(t % 2), start_sample=int(rng.integers(0, 40000))) for t in rng.choice(K, 30, replace=False)]
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_chirp_list(chirps)
    s.set_ramp_list(ramps)
    s.set_full_scale(2.0 * float(np.sum(a)))
    s.set_static_engine(awg.STATIC_GEMM_FP16)
    n = 80_000
    q, x = render(s, n, 0)
    w = oracle.add_ramps(oracle.make_waveform(FS, f, a, th, chirps), ramps)
    x_ref = oracle.render(w, 0, n, nthreads=NTHREADS)
    err = fp32_lsb(x, x_ref, s.full_scale)
    assert err <= FP32_BOUND_LSB, err
    q_ref = oracle.quantize(x_ref, s.full_scale)
    assert np.max(np.abs(q.astype(np.int32) - q_ref)) <= 1


def test_same_samples_however_the_stream_is_cut(awg):
    rng = np.random.default_rng(9)
    K = 1000
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.integers(2000, 30000)) / FS, profile=int(t % 2),
                   start_sample=int(rng.integers(0, 150000))) for t in rng.choice(K, 50, replace=False)]

    def make():
        s = awg.Synth(FS)
        s.set_tones(f, a, th)
        s.set_chirp_list(chirps)
        s.set_static_engine(awg.STATIC_GEMM_FP16)
        return s

    n = 300_000
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    make().render(n, ref)
    s = make()
    got = torch.empty(n, dtype=torch.int16, device="cuda")
    c = 0
    for piece in (1, 255, 257, 4096, 70_001, 1 << 16):
        s.render(piece, got[c:])
        c += piece
    s.render_chunks(1 << 14, 5, got[c:])
    c += 5 << 14
    s.render(n - c, got[c:])
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy(), got.cpu().numpy())
    # channel multiplexing with the engine
    s2, s3 = make(), make()
    mux = torch.empty(2 * n, dtype=torch.int16, device="cuda")
    awg.render_multiplexed([s2, s3], n, mux)
    torch.cuda.synchronize()
    m = mux.cpu().numpy()
    assert np.array_equal(m[0::2], ref.cpu().numpy()) and np.array_equal(m[1::2], ref.cpu().numpy())


def test_flagged_tones_over_several_ctas(awg, oracle):
    """400 tones hold a chirp or a ramp (the render's list split over 5 CTAs per tile, ranges from
    the flagged tones), starting at different times so that windows list different tones: the
    oracle at sampled indices, and the same samples however the stream is cut."""
    rng = np.random.default_rng(13)
    K, n = 4000, 400_000
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K) / 100
    th = rng.uniform(0, 2 * np.pi, K)
    picked = rng.choice(K, 400, replace=False)
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.integers(2000, 60000)) / FS, profile=int(t % 2),
                   start_sample=int(rng.integers(0, n - 60000))) for t in picked[:300]]
    ramps = [dict(tone=int(t), amp_end=float(rng.uniform(0, 0.01)), duration=float(rng.integers(500, 40000)) / FS,
                  profile=int(t % 2), start_sample=int(rng.integers(0, n - 40000))) for t in picked[300:]]

    def make():
        s = awg.Synth(FS)
        s.set_tones(f, a, th)
        s.set_chirp_list(chirps)
        s.set_ramp_list(ramps)
        s.set_full_scale(0.5 * float(np.sum(a)))
        s.set_static_engine(awg.STATIC_GEMM_FP16)
        return s

    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    make().render(n, ref)
    s = make()
    got = torch.empty(n, dtype=torch.int16, device="cuda")
    c = 0
    for piece in (4095, 4097, 50_000, 12_345, 100_000):
        s.render(piece, got[c:])
        c += piece
    s.render_chunks(1 << 13, 7, got[c:])
    c += 7 << 13
    s.render(n - c, got[c:])
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.array_equal(r, got.cpu().numpy())
    w = oracle.add_ramps(oracle.make_waveform(FS, f, a, th, chirps), ramps)
    idx = np.unique(np.concatenate([rng.integers(0, n, 400), [0, n - 1]]))
    q_ref = oracle.quantize(oracle.render_at(w, idx, nthreads=NTHREADS), 0.5 * float(np.sum(a)))
    assert np.max(np.abs(r[idx].astype(np.int32) - q_ref)) <= 1


def test_ten_thousand_tone_comb(awg, oracle):
    """10,000 tones on the tensor-core engine over 2^20 samples: a contiguous window of 2^18 samples
    and sampled indices against the oracle (FP32 within FP32_BOUND_LSB, int16 within 1 LSB)."""
    rng = np.random.default_rng(11)
    K = 10_000
    f = 80e6 + 1e4 * rng.permutation(10_000)[:K].astype(np.float64) + rng.uniform(-3e3, 3e3, K)
    a = np.full(K, 1.0 / K)
    th = rng.uniform(0, 2 * np.pi, K)
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_static_engine(awg.STATIC_GEMM_FP16)
    n = 1 << 20
    q, x = render(s, n)
    w = oracle.make_waveform(FS, f, a, th)
    idx = np.unique(rng.integers(0, n, 300))
    x_idx = oracle.render_at(w, idx, nthreads=NTHREADS)
    w0, wn = 300_000, 1 << 18
    x_win = oracle.render(w, w0, wn, nthreads=NTHREADS)
    FSv = w.full_scale()
    assert fp32_lsb(x[idx], x_idx, FSv) <= FP32_BOUND_LSB
    assert fp32_lsb(x[w0:w0 + wn], x_win, FSv) <= FP32_BOUND_LSB
    assert np.max(np.abs(q[idx].astype(np.int32) - oracle.quantize(x_idx, FSv))) <= 1
    assert np.max(np.abs(q[w0:w0 + wn].astype(np.int32) - oracle.quantize(x_win, FSv))) <= 1


def test_engine_validation(awg):
    s = awg.Synth(FS)
    with pytest.raises(awg.AwgError):
        s.set_static_engine(3)
    assert s.static_engine == awg.STATIC_DIRECT


@pytest.mark.parametrize("with_ramps", [False, True])
def test_same_samples_for_long_and_short_calls(awg, with_ramps):
    """The engine's GEMM sums a sample the same way whatever the length of the call that renders
    it: one call of 2^21 samples and calls of 2^14 (and a ragged tail) give the same bits, for a
    static comb (two columns per tone) and with ramps (four)."""
    rng = np.random.default_rng(17)
    K = 3000
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    ramps = [dict(tone=int(t), amp_end=float(rng.uniform(0, 2.0 / K)), duration=float(rng.integers(5000, 100000)) / FS,
                  profile=int(t % 2), start_sample=int(rng.integers(0, 1_500_000))) for t in rng.choice(K, 40, replace=False)]

    def make():
        s = awg.Synth(FS)
        s.set_tones(f, a, th)
        if with_ramps:
            s.set_ramp_list(ramps)
            s.set_full_scale(2.0 * float(np.sum(a)))
        s.set_static_engine(awg.STATIC_GEMM_FP16)
        return s

    n = 1 << 21
    one = torch.empty(n, dtype=torch.int16, device="cuda")
    make().render(n, one)
    s = make()
    cut = torch.empty(n, dtype=torch.int16, device="cuda")
    c = 0
    while c < n:
        m = min(1 << 14, n - c) if c < n - 3000 else n - c
        s.render(m, cut[c:])
        c += m
    torch.cuda.synchronize()
    assert np.array_equal(one.cpu().numpy(), cut.cpu().numpy())


def test_every_tone_chirping_with_the_engine(awg, oracle):
    """Every tone holds a long linear or minimum-jerk chirp in the window, so the engine's render
    part takes all K tones without a tone list (chirps in linear and LOW6 form visited in their
    groups, without the lane-pair set-up sharing of the direct path): against the oracle at sampled
    indices and within one LSB of the direct render."""
    rng = np.random.default_rng(29)
    K, n, n0 = 64, 60_000, 1_000_000
    f = rng.uniform(20e6, 120e6, K)
    a = rng.uniform(0.2, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = [dict(tone=k, f_start=float(f[k]), f_end=float(rng.uniform(20e6, 120e6)), duration=20e-3,
                   profile=k % 2, start_sample=int(rng.integers(0, 4096))) for k in range(K)]

    def make(engine):
        s = awg.Synth(FS)
        s.set_tones(f, a, th)
        s.set_chirp_list(chirps)
        if engine:
            s.set_static_engine(awg.STATIC_GEMM_FP16)
        return s

    q_eng, _ = render(make(True), n, n0)
    q_dir, _ = render(make(False), n, n0)
    assert np.max(np.abs(q_eng.astype(np.int32) - q_dir)) <= 1
    w = oracle.make_waveform(FS, f, a, th, chirps)
    idx = np.unique(np.concatenate([rng.integers(0, n, 500), [0, n - 1]]))
    q_ref = oracle.quantize(oracle.render_at(w, idx + n0, nthreads=NTHREADS), w.full_scale())
    assert np.max(np.abs(q_eng[idx].astype(np.int32) - q_ref)) <= 1
    assert np.max(np.abs(q_dir[idx].astype(np.int32) - q_ref)) <= 1
