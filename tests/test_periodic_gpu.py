"""Periodic hand-off after a chirp burst (the end state of the Playback pathway): once every chirp
is over and every final frequency sits on the record's grid (Eq. freqapprox), the output is a
periodic table replayed by a copy kernel.  With the table rendered by the render kernel the
replayed samples equal the rendered ones bit for bit; with the split-precision GEMM table they
are within 1 LSB of the oracle."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
FS = 280e6
LG = 16
N = 1 << LG


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _burst(seed, K=300, n_chirps=60):
    """Grid tones (2^16-sample grid); some chirp to other grid frequencies within ~0.5 ms."""
    rng = np.random.default_rng(seed)
    j = rng.choice(np.arange(N // 4, N // 2 - 100), K, replace=False)
    f = j * FS / N
    a = rng.uniform(0.5, 1.0, K) / K
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = []
    for t in rng.choice(K, n_chirps, replace=False):
        j_end = int(rng.integers(N // 4, N // 2 - 100))
        chirps.append(dict(tone=int(t), f_start=float(f[t]), f_end=float(j_end * FS / N),
                           duration=float(rng.uniform(0.05e-3, 0.5e-3)), profile=int(t % 2),
                           start_sample=int(rng.integers(0, 30000))))
    return f, a, th, chirps


def _make(awg, case, mode):
    f, a, th, chirps = case
    s = awg.Synth(FS)
    s.set_tones(f, a, th, grid_log2=LG)
    s.set_chirp_list(chirps)
    s.set_sine_mode(mode)
    return s


@pytest.mark.parametrize("mode", [0, 1])
def test_direct_table_replay_equals_rendering(awg, mode):
    case = _burst(1)
    total = 250_001 + 3 * N
    ref = torch.empty(total, dtype=torch.int16, device="cuda")
    _make(awg, case, mode).render(total, ref)
    s = _make(awg, case, mode)
    s.set_periodic(LG, awg.PERIODIC_DIRECT)
    n_p = s.periodic_start
    assert 0 < n_p < 250_001 and n_p % 4096 == 0
    got = torch.empty(total, dtype=torch.int16, device="cuda")
    c = 0
    for piece in (1000, 77_777, 4096 * 3, 100_003, total):
        m = min(piece, total - c)
        s.render(m, got[c:])
        c += m
    torch.cuda.synchronize()
    assert s.device_status() == 0
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.array_equal(r, g)
    assert np.array_equal(g[n_p:n_p + N], g[n_p + N:n_p + 2 * N])     # periodic from n_p on


def test_gemm_table_within_one_lsb(awg, oracle):
    case = _burst(2)
    f, a, th, chirps = case
    s = _make(awg, case, 0)
    s.set_periodic(LG, awg.PERIODIC_GEMM_FP16)
    n_p = s.periodic_start
    total = n_p + 2 * N + 333
    q = torch.empty(total, dtype=torch.int16, device="cuda")
    s.render(total, q)
    torch.cuda.synchronize()
    g = q.cpu().numpy()
    assert np.array_equal(g[n_p:n_p + N], g[n_p + N:n_p + 2 * N])
    w = oracle.make_waveform_window(FS, f, a, th, chirps, n_p, total - n_p)
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([rng.integers(n_p, total, 500), [n_p, total - 1]]))
    q_ref = oracle.quantize(oracle.render_at(w, idx, nthreads=NTHREADS), w.full_scale())
    assert np.max(np.abs(g[idx].astype(np.int32) - q_ref)) <= 1


def test_chunks_and_multiplexed_through_the_hand_off(awg):
    case = _burst(4, K=120, n_chirps=30)
    chunk, n_chunks = 1 << 15, 12
    ref = torch.empty(chunk * n_chunks, dtype=torch.int16, device="cuda")
    _make(awg, case, 0).render(chunk * n_chunks, ref)
    s = _make(awg, case, 0)
    s.set_periodic(LG, awg.PERIODIC_DIRECT)
    got = torch.empty(chunk * n_chunks, dtype=torch.int16, device="cuda")
    s.render_chunks(chunk, n_chunks, got)
    s2 = _make(awg, case, 0)
    s2.set_periodic(LG, awg.PERIODIC_DIRECT)
    other = _make(awg, _burst(5, K=50, n_chirps=0), 0)
    mux = torch.empty(2 * chunk * n_chunks, dtype=torch.int16, device="cuda")
    awg.render_multiplexed([s2, other], chunk * n_chunks, mux)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.array_equal(got.cpu().numpy(), r)
    assert np.array_equal(mux.cpu().numpy()[0::2], r)


def test_conditions_and_invalidation(awg):
    case = _burst(6, K=20, n_chirps=5)
    s = _make(awg, case, 0)
    with pytest.raises(awg.AwgError):
        s.set_periodic(11, awg.PERIODIC_DIRECT)            # period below 12
    with pytest.raises(awg.AwgError):
        s.set_periodic(14, awg.PERIODIC_GEMM_FP16)         # the GEMM needs 2^15
    with pytest.raises(awg.AwgError):
        s.set_periodic(LG, 3)
    assert s.periodic_start == -1
    off = awg.Synth(FS)
    off.set_tones([10.123456e6, 20e6], [1.0, 1.0], [0.0, 0.0])   # not on the 2^16 grid
    with pytest.raises(awg.AwgError):
        off.set_periodic(LG, awg.PERIODIC_DIRECT)
    s.set_periodic(LG, awg.PERIODIC_DIRECT)
    assert s.periodic_start > 0
    f, a, th, _ = case
    s.set_tones(f, a, th, grid_log2=LG)
    assert s.periodic_start == -1
    s.set_periodic(LG, awg.PERIODIC_DIRECT)
    s.clear_periodic()
    assert s.periodic_start == -1
