"""The allocation-free render (awg_render_noalloc).

It exists for callers that cannot allocate device memory while they stream: a real-time thread
feeding a DAC must not stall in the device allocator, and some host applications hand the
library a fixed memory budget.  It must produce the same samples as awg_render, call after call
(its fixed scratch keeps the previous call's contents), and refuse a window larger than that
scratch with a clear error.  This file is collected last so that a failure here cannot hide
another test's result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _synth(awg, wk):
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=wk.grid_log2)
    s.set_chirp_list(wk.chirps)
    return s


def _pair(awg, ref, alt, n):
    a = torch.empty(n, dtype=torch.int16, device="cuda")
    b = torch.full((n,), 12345, dtype=torch.int16, device="cuda")   # every sample must be written
    ref.render(n, a)
    alt.render_noalloc(n, b)
    torch.cuda.synchronize()
    return a.cpu().numpy().astype(np.int32), b.cpu().numpy().astype(np.int32)


def test_noalloc_matches_render_on_consecutive_calls(awg):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.chirp_1000(seed=2)          # 1000 chirping tones, 2^18-sample chunks
    ref, alt = _synth(awg, wk), _synth(awg, wk)
    for call in range(2):
        a, b = _pair(awg, ref, alt, wk.chunk)
        assert np.max(np.abs(a - b)) <= 1, call
        assert alt.cursor == ref.cursor == (call + 1) * wk.chunk
    assert alt.device_status() == 0


def test_noalloc_matches_render_with_chirps_starting_inside_windows(awg):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=4, K=12, n_samples=20000)
    ref, alt = _synth(awg, wk), _synth(awg, wk)
    for n in (7001, 9999):
        a, b = _pair(awg, ref, alt, n)
        assert np.max(np.abs(a - b)) <= 1, n


def test_noalloc_rejects_windows_beyond_its_scratch(awg):
    from paper_2403_15582_gb300 import workloads as wl
    from paper_2403_15582_gb300 import binding
    wk = wl.chirp_1000(seed=2)
    s = _synth(awg, wk)
    limit = 71493                                            # AWG_NOALLOC_MAX_RECORDS
    n = (limit // wk.K + 2) * 4096                           # 1000 chirps x 19 tiles > limit
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    with pytest.raises(awg.AwgError) as e:
        s.render_noalloc(n, out)
    assert e.value.code == binding.AWG_ENOMEM
    assert "AWG_NOALLOC_MAX_RECORDS" in str(e.value)
    assert s.cursor == 0
