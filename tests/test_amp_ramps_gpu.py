"""Amplitude ramps (a_j[i] of Eq. dynamicandstatic) on the GPU against the oracle: every sample of
records where ramps (linear and minimum-jerk, up, down, to zero) overlap chirps; folding of a
finished ramp; chunking; the periodic hand-off after the ramps.

FP32 bound per tone-sample: the render's 5e-6 max(|A|, |A_end|) (sine, argument, cascade) plus
6e-7 |A_end - A| for the ramp's FP32 amplitude, plus FP32 summation as in the render tests."""
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


def _case(seed, K=40, n_ramps=20, n_chirps=10, span=60000):
    rng = np.random.default_rng(seed)
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(0, 2 * np.pi, K)
    ramps = []
    for i, t in enumerate(rng.choice(K, n_ramps, replace=False)):
        end = 0.0 if i % 5 == 0 else float(rng.uniform(0.1, 1.5))
        ramps.append(dict(tone=int(t), amp_end=end, duration=float(rng.integers(100, 20000)) / FS,
                          profile=int(i % 2), start_sample=int(rng.integers(0, span // 2))))
    chirps = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(1e6, 139e6)),
                   duration=float(rng.integers(3000, 25000)) / FS, profile=int(t % 2),
                   start_sample=int(rng.integers(0, span // 2)))
              for t in rng.choice(K, n_chirps, replace=False)]
    return f, a, th, ramps, chirps


def _bound(a, ramps, split):
    amax = np.abs(np.asarray(a, dtype=np.float64)).copy()
    dA = np.zeros_like(amax)
    for r in ramps:
        k = r["tone"]
        dA[k] = abs(r["amp_end"] - a[k])
        amax[k] = max(amax[k], abs(r["amp_end"]))
    K = len(a)
    return float(np.sum(5e-6 * amax + 6e-7 * dA) + np.sum(amax) * (K / split + split + 2) * 2.0**-24)


def _synth(awg, case, mode=0):
    f, a, th, ramps, chirps = case
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_chirp_list(chirps)
    s.set_ramp_list(ramps)
    s.set_sine_mode(mode)
    amax = np.abs(a).copy()
    for r in ramps:
        amax[r["tone"]] = max(amax[r["tone"]], abs(r["amp_end"]))
    s.set_full_scale(float(np.sum(amax)))
    return s


def _oracle_wave(oracle, case):
    f, a, th, ramps, chirps = case
    w = oracle.make_waveform(FS, f, a, th, chirps)
    return oracle.add_ramps(w, ramps)


@pytest.mark.parametrize("mode", [0, 1])
def test_every_sample_against_the_oracle(awg, oracle, mode):
    case = _case(1)
    s = _synth(awg, case, mode)
    n = 60000
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, q)
    torch.cuda.synchronize()
    assert s.device_status() == 0
    w = _oracle_wave(oracle, case)
    x_ref = oracle.render(w, 0, n, nthreads=NTHREADS)
    err = float(np.max(np.abs(x.cpu().numpy().astype(np.float64) - x_ref)))
    assert err <= _bound(case[1], case[3], s.tone_split), err
    q_ref = oracle.quantize(x_ref, s.full_scale)
    assert np.max(np.abs(q.cpu().numpy().astype(np.int32) - q_ref)) <= 1


def test_second_ramp_folds_the_first(awg, oracle):
    f, a, th = [30e6, 70.5e6], [0.8, 0.4], [0.1, 2.0]
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_full_scale(3.0)
    s.set_ramp_list([dict(tone=0, amp_end=0.1, duration=5000 / FS, profile=1, start_sample=1000)])
    q1 = torch.empty(8000, dtype=torch.int16, device="cuda")
    s.render(8000, q1)
    with pytest.raises(awg.AwgError):     # tone 1 ramp starting before the cursor
        s.set_ramp_list([dict(tone=1, amp_end=1.0, duration=1e-6, profile=0, start_sample=7000)])
    s.set_ramp_list([dict(tone=0, amp_end=1.2, duration=3000 / FS, profile=0, start_sample=9000)])
    q2 = torch.empty(6000, dtype=torch.int16, device="cuda")
    s.render(6000, q2)
    torch.cuda.synchronize()
    w = oracle.make_waveform(FS, f, [0.1, 0.4], th)          # after the first ramp A_0 = 0.1
    oracle.add_ramps(w, [dict(tone=0, amp_end=1.2, duration=3000 / FS, profile=0, start_sample=9000)])
    q_ref = oracle.quantize(oracle.render(w, 8000, 6000, nthreads=NTHREADS), 3.0)
    assert np.max(np.abs(q2.cpu().numpy().astype(np.int32) - q_ref)) <= 1


def test_chunking_bit_exact(awg):
    case = _case(2, K=300, n_ramps=60, n_chirps=30, span=200000)
    n = 200000
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    _synth(awg, case).render(n, ref)
    s = _synth(awg, case)
    got = torch.empty(n, dtype=torch.int16, device="cuda")
    s.render(12345, got)
    s.render_chunks(1 << 14, 11, got[12345:])
    rest = n - 12345 - 11 * (1 << 14)
    s.render(rest, got[n - rest:])
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy(), got.cpu().numpy())


def test_periodic_hand_off_after_ramps(awg):
    lg, N = 16, 1 << 16
    rng = np.random.default_rng(3)
    j = rng.choice(np.arange(N // 8, N // 2 - 100), 50, replace=False)
    f = j * FS / N
    a = rng.uniform(0.2, 1.0, 50)
    th = rng.uniform(0, 2 * np.pi, 50)
    ramps = [dict(tone=int(t), amp_end=float(rng.uniform(0, 1)), duration=float(rng.integers(1000, 30000)) / FS,
                  profile=int(t % 2), start_sample=int(rng.integers(0, 50000))) for t in range(0, 50, 3)]

    def make():
        s = awg.Synth(FS)
        s.set_tones(f, a, th, grid_log2=lg)
        s.set_ramp_list(ramps)
        s.set_full_scale(50.0)
        return s

    total = 120000 + 2 * N
    ref = torch.empty(total, dtype=torch.int16, device="cuda")
    make().render(total, ref)
    s = make()
    s.set_periodic(lg, awg.PERIODIC_DIRECT)
    assert s.periodic_start >= 50000
    got = torch.empty(total, dtype=torch.int16, device="cuda")
    s.render(total, got)
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy(), got.cpu().numpy())


def test_ramp_argument_errors(awg):
    s = awg.Synth(FS)
    s.set_tones([10e6, 20e6], [1.0, 1.0], [0.0, 0.0], grid_log2=16)
    bad = [dict(tone=2, amp_end=0.5, duration=1e-6, profile=0, start_sample=0),
           dict(tone=0, amp_end=float("nan"), duration=1e-6, profile=0, start_sample=0),
           dict(tone=0, amp_end=0.5, duration=0.0, profile=0, start_sample=0),
           dict(tone=0, amp_end=0.5, duration=1e-6, profile=7, start_sample=0)]
    for r in bad:
        with pytest.raises(awg.AwgError):
            s.set_ramp_list([r])
    with pytest.raises(awg.AwgError):     # two ramps for one tone in one call
        s.set_ramp_list([dict(tone=0, amp_end=0.5, duration=1e-6, profile=0, start_sample=0)] * 2)
    s.set_ramp_list([dict(tone=0, amp_end=0.5, duration=1e-3, profile=1, start_sample=10)])
    with pytest.raises(awg.AwgError):     # the first ramp has not been rendered past
        s.set_ramp_list([dict(tone=0, amp_end=0.9, duration=1e-6, profile=0, start_sample=500000)])
    q = torch.empty(1 << 16, dtype=torch.int16, device="cuda")
    with pytest.raises(awg.AwgError):     # the table GEMM needs constant amplitudes
        s.table_gemm(16, 1, q)
