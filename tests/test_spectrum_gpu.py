"""Digital spectral check of the int16 output (the paper measures SFDR with a spectrum analyser;
here it is computed from the samples): for tones on the record's frequency grid (Eq. freqapprox)
the 2^20-sample record is periodic, so an unwindowed FFT puts every tone in one bin and everything
else is spur.  The GPU output's spurious-free dynamic range matches that of the oracle's FP64 sum
quantised the same way, in both sine variants."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
LG = 20
N = 1 << LG
FS_HZ = 280e6


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def sfdr_dbc(x, bins):
    """Weakest tone power over the largest non-tone, non-DC bin power, in dB."""
    P = np.abs(np.fft.rfft(np.asarray(x, dtype=np.float64))) ** 2
    mask = np.ones(P.size, dtype=bool)
    mask[0] = False
    mask[bins] = False
    return 10 * np.log10(P[bins].min() / P[mask].max())


def _case(K, seed):
    rng = np.random.default_rng(seed)
    j = np.sort(rng.choice(np.arange(N // 20, N // 2 - N // 20), K, replace=False))
    f = j * FS_HZ / N
    a = np.full(K, 1.0 / K)
    th = rng.uniform(0, 2 * np.pi, K)
    return f, a, th, j


@pytest.mark.parametrize("K,floor_db", [(1, 90.0), (100, 45.0)])
@pytest.mark.parametrize("mode", [0, 1])
def test_sfdr_matches_oracle(awg, oracle, K, floor_db, mode):
    f, a, th, bins = _case(K, 40 + K)
    s = awg.Synth(FS_HZ)
    s.set_tones(f, a, th, grid_log2=LG)
    s.set_sine_mode(mode)
    q = torch.empty(N, dtype=torch.int16, device="cuda")
    s.render(N, q)
    torch.cuda.synchronize()
    g = q.cpu().numpy()
    w = oracle.make_waveform(FS_HZ, f, a, th, grid_log2=LG)
    r = oracle.quantize(oracle.render(w, 0, N, nthreads=NTHREADS), w.full_scale())
    s_gpu, s_ref = sfdr_dbc(g, bins), sfdr_dbc(r, bins)
    assert s_gpu >= floor_db, (s_gpu, s_ref)
    assert abs(s_gpu - s_ref) <= 3.0, (s_gpu, s_ref)
