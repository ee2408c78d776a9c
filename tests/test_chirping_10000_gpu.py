"""10,000 tones that all chirp at once (the real-time target: every tone ramping along a linear or
minimum-jerk profile, Eq. freqchirp, continued segment after segment).  Two 33.7 ms segments are
rendered through the pipelined chunk loop; windows at the record's start, across the boundary
where every tone's first chirp ends and its second begins, inside the second segment and at its
end are compared element by element with the CPU oracle (int16 within 1 LSB).  The oracle folds
each tone's finished chirp into its static state before the window (Eq. freqchirp case 2)."""
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


def test_ten_thousand_chirping_tones_against_the_oracle(awg, oracle):
    from paper_2403_15582_gb300 import workloads as wl
    K, segs = 10_000, 2
    wk = wl.chirping_stream(seed=1, K=K, segments=segs)
    S = wk.n_samples // segs
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    assert s.tone_split == 16
    out = torch.empty(wk.n_samples, dtype=torch.int16, device="cuda")
    for g in range(segs):
        s.set_chirp_list([c for c in wk.chirps if c["start_sample"] == g * S])
        s.render_stream(S, 1 << 18, out[g * S:])
    torch.cuda.synchronize()
    assert s.device_status() == 0
    q = out.cpu().numpy()
    FS = float(np.sum(np.abs(wk.amp)))
    # a window holds at most one chirp per tone: the boundary is covered by one window on each side
    windows = [(0, 4096), (S - 6000, 6000), (S, 6000), (S + S // 2 + 777, 4096), (wk.n_samples - 4096, 4096)]
    for n0, n in windows:
        w = oracle.make_waveform_window(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, n0, n)
        q_ref = oracle.quantize(oracle.render(w, n0, n, nthreads=NTHREADS), FS)
        dq = np.abs(q[n0:n0 + n].astype(np.int32) - q_ref.astype(np.int32))
        assert dq.max() <= 1, (n0, int(dq.max()))


def test_rotating_stream_of_10000_tones_against_the_oracle(awg, oracle):
    """The continuous 10,000-tone stream at 280 MS/s (groups of 100 tones ramping linearly for 1 ms in
    turn) rendered as the stream driver does it: 2^20-sample chunks, each chunk's chirps handed to
    the library just before the chunk.  120 ms, so that group 0 ramps twice and every tone's first
    ramp is folded into its static state before its second; windows across group hand-overs, inside
    a ramp and after a second ramp are compared element by element with the oracle (int16 within
    1 LSB)."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.stream_rotating(seed=3, fs=280e6, seconds=0.12)
    chunk = wk.chunk
    n_chunks = -(-wk.n_samples // chunk)
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    out = torch.empty(n_chunks * chunk, dtype=torch.int16, device="cuda")
    order = sorted(wk.chirps, key=lambda c: c["start_sample"])
    nxt = 0
    for c in range(n_chunks):
        batch = []
        while nxt < len(order) and order[nxt]["start_sample"] < (c + 1) * chunk:
            batch.append(order[nxt])
            nxt += 1
        if batch:
            s.set_chirp_list(batch)
        s.render(chunk, out[c * chunk:])
    torch.cuda.synchronize()
    assert s.device_status() == 0
    q = out.cpu().numpy()
    FS = float(np.sum(np.abs(wk.amp)))
    L = 280000                                                 # one 1 ms ramp
    windows = [(0, 4096), (L - 2048, 4096), (37 * L + 140_001, 4096), (100 * L - 3000, 6000),
               (100 * L + L // 2, 4096), (119 * L + 12_345, 4096)]
    for n0, n in windows:
        w = oracle.make_waveform_window(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, n0, n)
        q_ref = oracle.quantize(oracle.render(w, n0, n, nthreads=NTHREADS), FS)
        dq = np.abs(q[n0:n0 + n].astype(np.int32) - q_ref.astype(np.int32))
        assert dq.max() <= 1, (n0, int(dq.max()))
