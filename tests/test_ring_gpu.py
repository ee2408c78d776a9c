"""Streaming ring: the sink plays what the render kernel wrote into pinned host slots; underruns
are counted when a chunk is late (provoked on the host by a slow producer -- no GPU fault)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _tones(fs, K, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.01 * fs, 0.45 * fs, K), rng.uniform(0.2, 1.0, K), rng.uniform(0, 6.28, K)


def test_ring_plays_exactly_what_render_writes(awg):
    from paper_2403_15582_gb300.stream import run_stream
    fs, K, chunk, n = 2e6, 40, 3 * 4096 + 5, 10          # 6 ms of playback per chunk
    f, a, th = _tones(fs, K, 1)
    chirps = [dict(tone=k, f_start=float(f[k]), f_end=float(f[k]) * 0.9, duration=20000 / fs, profile=k % 2,
                   start_sample=int(1000 + 7000 * k)) for k in range(0, K, 4)]
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    ring = awg.Ring(s, chunk, 3)
    cap = np.zeros(chunk * n, dtype=np.int16)
    st = run_stream(s, ring, chirps, n, capture=cap)
    assert st["played"] == n and st["underruns"] == 0
    ref = awg.Synth(fs)
    ref.set_tones(f, a, th)
    ref.set_chirp_list(chirps)
    out = torch.empty(chunk * n, dtype=torch.int16, device="cuda")
    ref.render(chunk * n, out)
    torch.cuda.synchronize()
    assert np.array_equal(cap, out.cpu().numpy())
    ring.close()


def test_ring_stream_matches_oracle_with_repeated_chirps(awg, oracle):
    from paper_2403_15582_gb300.stream import run_stream
    fs, K, chunk, n = 2e6, 30, 8192, 8
    f, a, th = _tones(fs, K, 2)
    chirps = []
    for k in range(K):   # every tone chirps twice, the second time from where the first ended
        f1 = float(f[k]) * 0.8
        chirps.append(dict(tone=k, f_start=float(f[k]), f_end=f1, duration=5000 / fs, profile=k % 2, start_sample=2000 + 97 * k))
        chirps.append(dict(tone=k, f_start=f1, f_end=float(f[k]), duration=9000 / fs, profile=(k + 1) % 2,
                           start_sample=30000 + 113 * k))
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    ring = awg.Ring(s, chunk, 4)
    cap = np.zeros(chunk * n, dtype=np.int16)
    st = run_stream(s, ring, chirps, n, capture=cap)
    assert st["played"] == n
    for c in range(n):
        w = oracle.make_waveform_window(fs, f, a, th, chirps, c * chunk, chunk)
        idx = c * chunk + np.arange(0, chunk, 37)
        q_ref = oracle.quantize(oracle.render_at(w, idx), w.full_scale())
        assert np.max(np.abs(cap[idx].astype(np.int32) - q_ref)) <= 1, c
    ring.close()


def test_ring_counts_underruns_of_a_slow_producer(awg):
    from paper_2403_15582_gb300.stream import run_stream
    fs, chunk, n = 1e6, 2048, 12                            # 2 ms per chunk, producer adds 5 ms
    f, a, th = _tones(fs, 8, 3)
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    ring = awg.Ring(s, chunk, 2)
    st = run_stream(s, ring, [], n, prefill=1, producer_delay_s=0.005)
    assert st["played"] == n
    assert st["underruns"] >= n // 2
    ring.close()


def test_ring_push_times_out_when_full(awg):
    fs, chunk = 1e6, 1024
    f, a, th = _tones(fs, 4, 4)
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    ring = awg.Ring(s, chunk, 2)
    ring.push(None, 100)
    ring.push(None, 100)
    with pytest.raises(awg.AwgError) as e:      # no sink running: the third slot never frees
        ring.push(None, 50)
    assert e.value.code == awg.AWG_ETIMEOUT
    ring.close()
