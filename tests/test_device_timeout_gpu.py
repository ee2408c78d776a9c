"""Bounded waits on the device.  Every spin-wait in the library's kernels (mbarrier waits on bulk
copies, the join that ends a pipelined chunk sequence) gives up after a wall-time limit, sets the
handle's device status word to AWG_ETIMEOUT and returns, so a lost wake-up becomes an error code
instead of a hung GPU.  Here a join waits for a count that no kernel will reach, with a 1 ms limit:
the status reads AWG_ETIMEOUT once, is cleared by the read, and the same handle then renders
within 1 LSB of the oracle again."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _render_and_check(awg, oracle, s, w, n0, n):
    s.seek(n0)
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    s.render_chunks(4096, n // 4096, q)          # a pipelined sequence, closed by a join
    torch.cuda.synchronize()
    q_ref = oracle.quantize(oracle.render(w, n0, n), w.full_scale())
    assert np.max(np.abs(q.cpu().numpy().astype(np.int32) - q_ref)) <= 1


def test_join_wait_times_out_and_the_handle_stays_usable(awg, oracle):
    from paper_2403_15582_gb300 import binding
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=3, K=10, n_samples=5 * 4096)
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad)
    s.set_chirp_list(wk.chirps)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps)
    _render_and_check(awg, oracle, s, w, 0, wk.n_samples)
    assert s.device_status() == 0
    s.test_wait_timeout(1000)                    # 1 ms, on the current stream
    torch.cuda.synchronize()
    assert s.device_status() == binding.AWG_ETIMEOUT
    assert s.device_status() == 0                # the read cleared it
    _render_and_check(awg, oracle, s, w, 0, wk.n_samples)
    assert s.device_status() == 0
    with pytest.raises(awg.AwgError):
        s.test_wait_timeout(0)
