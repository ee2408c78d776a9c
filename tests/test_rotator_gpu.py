"""GPU parity of the rotator sine variant (static tone segments: exact sin/cos at the start of each
32-sample run, then complex rotations by the per-sample step on the FP32 pipe) against the oracle.

Bound per tone-sample (written out in `rot_bound`): run-start phasor <= 7.4e-7 |A| (the 32-bit
turn to float, the 2 pi scaling and the SFU sine/cosine), then per rotation <= 4.2e-8 |A| from the
FP32 rounding of (cos, sin) of the step and <= 1.7e-7 |A| from the two roundings of each
component, over at most 31 rotations: <= 7.4e-6 |A|, taken as 1.2e-5 |A|; plus FP32 summation of
K/split + split terms.  Chirp segments keep the SFU form (`fp32_bound` of the render tests)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def rot_bound(amps, split):
    K = len(amps)
    S = float(np.sum(np.abs(amps)))
    return S * (1.2e-5 + (K / max(split, 1) + split + 2) * 2.0**-24)


def render(s, n, n0=None):
    if n0 is not None:
        s.seek(n0)
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, q)
    torch.cuda.synchronize()
    assert s.device_status() == 0
    return q.cpu().numpy(), x.cpu().numpy()


def check(q, x, w, oracle, x_ref, split):
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(q.astype(np.int32) - q_ref)) <= 1
    err = float(np.max(np.abs(x.astype(np.float64) - x_ref)))
    assert err <= rot_bound(w.A, split), (err, rot_bound(w.A, split))
    return err


def test_mode_switch_and_validation(awg):
    s = awg.Synth(280e6)
    assert s.sine_mode == awg.SINE_SFU
    s.set_sine_mode(awg.SINE_ROTATOR)
    assert s.sine_mode == awg.SINE_ROTATOR
    with pytest.raises(awg.AwgError):
        s.set_sine_mode(2)
    assert s.sine_mode == awg.SINE_ROTATOR


def test_static_100_full_record(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.static_100(seed=0)
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    s.set_sine_mode(awg.SINE_ROTATOR)
    q, x = render(s, wk.n_samples)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad)
    check(q, x, w, oracle, oracle.render(w, 0, wk.n_samples, nthreads=NTHREADS), s.tone_split)


@pytest.mark.parametrize("K", [1, 65, 1000])
def test_any_frequency(awg, oracle, K):
    """Frequencies over [0, f_s), including DC, Nyquist and just below f_s; a window far into the
    stream (phase words wrap many times)."""
    rng = np.random.default_rng(100 + K)
    fs = 280e6
    f = rng.uniform(0, fs, K)
    f[:min(K, 4)] = [0.0, fs / 2, fs - 1.0, 1.0][:min(K, 4)]
    a = rng.uniform(-1, 1, K)
    th = rng.uniform(0, 6.3, K)
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    s.set_sine_mode(awg.SINE_ROTATOR)
    n0 = 3_000_000_007
    q, x = render(s, 20000, n0)
    w = oracle.make_waveform(fs, f, a, th)
    check(q, x, w, oracle, oracle.render(w, n0, 20000, nthreads=NTHREADS), s.tone_split)


def test_chirps_with_static_segments(awg, oracle):
    """Tones that chirp inside the record: their static segments before and after the chirp
    rotate, the chirp segments keep the SFU form; the whole record against the oracle."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=3, K=24, n_samples=60000)
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    s.set_chirp_list(wk.chirps)
    s.set_sine_mode(awg.SINE_ROTATOR)
    q, x = render(s, wk.n_samples, 0)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps)
    check(q, x, w, oracle, oracle.render(w, 0, wk.n_samples, nthreads=NTHREADS), s.tone_split)


def test_chunking_and_pipelined_sequence_bit_exact(awg):
    rng = np.random.default_rng(7)
    K, fs, chunk = 500, 280e6, 1 << 16
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(0, 6.3, K)

    def make():
        s = awg.Synth(fs)
        s.set_tones(f, a, th)
        s.set_sine_mode(awg.SINE_ROTATOR)
        return s

    n = 5 * chunk
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    make().render(n, ref)
    s2 = make()
    got = torch.empty(n, dtype=torch.int16, device="cuda")
    s2.render(4097, got)
    s2.render(chunk - 4097, got[4097:])
    s2.render_chunks(chunk, 4, got[chunk:])
    torch.cuda.synchronize()
    assert np.array_equal(ref.cpu().numpy(), got.cpu().numpy())
