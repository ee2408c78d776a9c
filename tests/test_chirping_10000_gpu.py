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
