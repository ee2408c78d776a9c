"""Channel multiplexing fused into the render's store (the WM step of Sec. IV-C): interleaved
groups of one sample per channel.  Each de-interleaved channel is compared element by element with
the CPU oracle (int16 within 1 LSB) and with its own render (bit for bit)."""
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


def _channel(awg, seed, K, fs=280e6, chirps=0, oracle=None):
    rng = np.random.default_rng(seed)
    f = rng.uniform(80e6, 180e6, K)
    a = rng.uniform(0.5, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    ch = [dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(80e6, 180e6)),
               duration=float(rng.uniform(0.1e-3, 0.3e-3)), profile=int(t % 2), start_sample=int(rng.integers(0, 50000)))
          for t in rng.choice(K, chirps, replace=False)] if chirps else []

    def make():
        s = awg.Synth(fs)
        s.set_tones(f, a, th)
        if ch:
            s.set_chirp_list(ch)
        return s

    def reference(n):
        """The oracle's int16 codes of samples 0 .. n-1 (full scale sum |A|)."""
        w = oracle.make_waveform(fs, f, a, th, ch)
        return oracle.quantize(oracle.render(w, 0, n, nthreads=NTHREADS), w.full_scale())
    make.reference = reference
    return make


@pytest.mark.parametrize("n_ch", [1, 2, 4])
def test_interleaved_channels_equal_their_own_renders(awg, oracle, n_ch):
    makers = [_channel(awg, 10 + c, K, chirps=nc, oracle=oracle) for c, (K, nc) in
              enumerate([(100, 0), (700, 40), (37, 37), (2000, 10)][:n_ch])]
    n1, n2 = 70001, 50000
    chans = [m() for m in makers]
    out = torch.full(((n1 + n2) * n_ch,), -32768, dtype=torch.int16, device="cuda")
    awg.render_multiplexed(chans, n1, out)
    awg.render_multiplexed(chans, n2, out[n1 * n_ch:])
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(-1, n_ch)
    for c, m in enumerate(makers):
        s = m()
        ref = torch.empty(n1 + n2, dtype=torch.int16, device="cuda")
        s.render(n1 + n2, ref)
        torch.cuda.synchronize()
        assert np.array_equal(got[:, c], ref.cpu().numpy()), c
        assert chans[c].cursor == n1 + n2
        dq = np.abs(got[:, c].astype(np.int32) - m.reference(n1 + n2).astype(np.int32))
        assert dq.max() <= 1, (c, int(dq.max()))


def test_multiplex_argument_errors(awg):
    a, b = _channel(awg, 1, 10)(), _channel(awg, 2, 10)()
    out = torch.empty(1024, dtype=torch.int16, device="cuda")
    with pytest.raises(awg.AwgError):
        awg.render_multiplexed([a, a], 100, out)                  # one handle in two channels
    with pytest.raises(awg.AwgError):
        awg.render_multiplexed([], 100, out)
    c = awg.Synth(100e6)
    c.set_tones([1e6], [1.0], [0.0])
    with pytest.raises(awg.AwgError):
        awg.render_multiplexed([a, c], 100, out)                  # two sample rates
    assert a.cursor == 0 and b.cursor == 0 and c.cursor == 0
