"""The allocation-free render (awg_render_noalloc).

It exists for callers that cannot allocate device memory while they stream: a real-time thread
feeding a DAC must not stall in the device allocator, and some host applications hand the
library a fixed memory budget.  It must produce the same samples as awg_render, bit for bit, call
after call (its fixed scratch keeps the previous call's contents), leave the device's free memory
unchanged, and refuse a window larger than that scratch with a clear error.  This file is
collected last so that a failure here cannot hide another test's result."""
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
    return a.cpu().numpy(), b.cpu().numpy()


@pytest.mark.parametrize("K", [1000, 1500])
def test_noalloc_matches_render_on_consecutive_calls(awg, K):
    """1000 (tone split 11) and 1500 (split 16, the largest thread-block cluster) chirping tones,
    two consecutive chunks (2^18 and 2^16 samples: 1000 x 64 and 1500 x 16 tile records, within the
    fixed scratch): the same bits as awg_render, and the device's free memory unchanged over the
    noalloc calls."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.chirp_1000(seed=2, K=K)
    ref, alt = _synth(awg, wk), _synth(awg, wk)
    assert alt.tone_split == (11 if K == 1000 else 16)
    n = wk.chunk if K == 1000 else 1 << 16
    a = [torch.empty(n, dtype=torch.int16, device="cuda") for _ in range(2)]
    b = [torch.full((n,), 12345, dtype=torch.int16, device="cuda") for _ in range(2)]
    for c in range(2):
        ref.render(n, a[c])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for c in range(2):
        alt.render_noalloc(n, b[c])
        assert alt.cursor == (c + 1) * n
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for c in range(2):
        assert np.array_equal(a[c].cpu().numpy(), b[c].cpu().numpy()), c
    assert alt.device_status() == 0


@pytest.mark.parametrize("K", [12, 200])
def test_noalloc_matches_render_with_chirps_starting_inside_windows(awg, K):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=4, K=K, n_samples=20000)
    ref, alt = _synth(awg, wk), _synth(awg, wk)
    assert alt.tone_split == (1 if K == 12 else 3)
    for n in (7001, 9999):
        a, b = _pair(awg, ref, alt, n)
        assert np.array_equal(a, b), n


def test_noalloc_rejects_windows_beyond_its_scratch(awg):
    from paper_2403_15582_gb300 import workloads as wl
    from paper_2403_15582_gb300 import binding
    wk = wl.chirp_1000(seed=2)
    s = _synth(awg, wk)
    limit = binding.NOALLOC_MAX_RECORDS
    n = (limit // wk.K + 2) * 4096                           # 1000 chirps x 19 tiles > limit
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    with pytest.raises(awg.AwgError) as e:
        s.render_noalloc(n, out)
    assert e.value.code == binding.AWG_ENOMEM
    assert "AWG_NOALLOC_MAX_RECORDS" in str(e.value)
    assert s.cursor == 0
