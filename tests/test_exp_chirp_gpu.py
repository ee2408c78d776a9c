"""Exponential chirps (Sec. II names them beside the minimum-jerk profile: the frequency moves
geometrically from f_start to f_end and the phase is its integral) on the GPU against the oracle:
phase words, the render's 32-bit phases and every sample, for long chirps (tile polynomials) and
short fast ones (per-sample tables), up and down, beside polynomial chirps; chunk invariance, the
static engine, and the argument rules.

Bounds: phase words within 2^36 words (2^-28 turn: FP64 evaluation of R(m) on both sides); the
32-bit run phases within 2600 units of 2^-32 turn (the minimum-jerk cascade bound of 2500 plus
the tile polynomial's dropped orders, <= 2^-26 turn = 64 units); samples as in the render tests."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
FS = 280e6
EXP = 2


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _case(seed, K=24, span=300_000, n_chirps=16):
    rng = np.random.default_rng(seed)
    f = rng.uniform(5e6, 135e6, K)
    a = rng.uniform(0.2, 1.0, K)
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = []
    for i, t in enumerate(rng.choice(K, n_chirps, replace=False)):
        L = (200_000, 100_000, 20_000, 3_000)[i % 4]
        f1 = float(rng.uniform(1e6, 139e6))
        if i == 0:      # a slow ratio: tile polynomials (the fast ones get per-sample tables)
            f1 = f[t] * 1.3 if f[t] * 1.3 < 139e6 else f[t] / 1.3
        chirps.append(dict(tone=int(t), f_start=float(f[t]), f_end=f1, duration=L / FS,
                           profile=EXP if i < 3 * n_chirps // 4 else int(i % 2),
                           start_sample=int(rng.integers(0, span - L))))
    return f, a, th, chirps


def _synth(awg, case, mode=0, engine=0):
    f, a, th, chirps = case
    s = awg.Synth(FS)
    s.set_tones(f, a, th)
    s.set_chirp_list(chirps)
    s.set_sine_mode(mode)
    s.set_static_engine(engine)
    return s


def _bound(a, split):
    K = len(a)
    S = float(np.sum(np.abs(a)))
    return S * (5e-6 + (K / max(split, 1) + split + 2) * 2.0**-24)


def _sdiff(a, b, bits):
    m = 1 << bits
    d = (np.asarray(a, dtype=object) - np.asarray(b, dtype=object)) % m
    return np.array([int(x) - m if x >= m // 2 else int(x) for x in d], dtype=np.float64)


@pytest.mark.parametrize("mode", [0, 1])
def test_every_sample_against_the_oracle(awg, oracle, mode):
    case = _case(1)
    f, a, th, chirps = case
    s = _synth(awg, case, mode)
    n = 300_000
    q = torch.empty(n, dtype=torch.int16, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    s.render_f32(n, x, q)
    torch.cuda.synchronize()
    assert s.device_status() == 0
    w = oracle.make_waveform(FS, f, a, th, chirps)
    x_ref = oracle.render(w, 0, n, nthreads=NTHREADS)
    err = float(np.max(np.abs(x.cpu().numpy().astype(np.float64) - x_ref)))
    assert err <= _bound(a, s.tone_split), err
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(q.cpu().numpy().astype(np.int32) - q_ref)) <= 1


def test_phase_words_and_run_phases(awg, oracle):
    case = _case(2)
    f, a, th, chirps = case
    s = _synth(awg, case)
    w = oracle.make_waveform(FS, f, a, th, chirps)
    exp_tones = [c["tone"] for c in chirps if c["profile"] == EXP]
    rng = np.random.default_rng(0)
    for n in [0, 1, 299_999] + [int(c["start_sample"]) + d for c in chirps for d in (0, 1, 4095, int(c["duration"] * FS))] \
            + list(rng.integers(0, 300_000, 20)):
        got = s.phase_words(int(n), w.K)
        ref = [int(oracle.phase_words_at(w, k, [int(n)])[0]) for k in range(w.K)]
        for k in range(w.K):
            if k in exp_tones:
                assert abs(_sdiff([int(got[k])], [ref[k]], 64)[0]) <= 2.0**36, (n, k)
            else:
                assert int(got[k]) == ref[k], (n, k)
    # the render's 32-bit phases over whole chirps (tile polynomials and per-sample tables)
    for c in chirps:
        if c["profile"] != EXP:
            continue
        k, n0 = c["tone"], max(0, int(c["start_sample"]) - 100)
        cnt = min(int(c["duration"] * FS) + 200, 300_000 - n0)
        got = s.render_phases(k, n0, cnt)
        words = oracle.phase_words_at(w, k, np.arange(n0, n0 + cnt, dtype=np.int64))
        ref = [((int(v) + (1 << 40)) >> 32) % (1 << 32) for v in words]
        d = np.abs(_sdiff(got.astype(np.int64), ref, 32))
        assert d.max() <= 2600, (k, int(d.max()))


def test_chunks_and_static_engine(awg, oracle):
    case = _case(3, K=200, span=400_000, n_chirps=40)
    f, a, th, chirps = case
    n = 400_000
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    _synth(awg, case).render(n, ref)
    s = _synth(awg, case)
    got = torch.empty(n, dtype=torch.int16, device="cuda")
    c = 0
    for piece in (4095, 123_457, 4097):
        s.render(piece, got[c:])
        c += piece
    s.render_chunks(1 << 15, 8, got[c:])
    c += 8 << 15
    s.render(n - c, got[c:])
    eng = torch.empty(n, dtype=torch.int16, device="cuda")
    se = _synth(awg, case, engine=awg.STATIC_GEMM_FP16)
    se.render(n, eng)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.array_equal(r, got.cpu().numpy())
    w = oracle.make_waveform(FS, f, a, th, chirps)
    idx = np.unique(np.concatenate([np.random.default_rng(4).integers(0, n, 500), [0, n - 1]]))
    q_ref = oracle.quantize(oracle.render_at(w, idx, nthreads=NTHREADS), w.full_scale())
    assert np.max(np.abs(r[idx].astype(np.int32) - q_ref)) <= 1
    assert np.max(np.abs(eng.cpu().numpy()[idx].astype(np.int32) - q_ref)) <= 1


def test_argument_rules(awg):
    s = awg.Synth(FS)
    s.set_tones([0.0, 50e6], [1.0, 1.0], [0.0, 0.0])
    with pytest.raises(awg.AwgError):       # from 0 Hz: no frequency ratio
        s.set_chirp_list([dict(tone=0, f_start=0.0, f_end=10e6, duration=1e-4, profile=EXP, start_sample=0)])
    with pytest.raises(awg.AwgError):
        s.set_chirp_list([dict(tone=1, f_start=50e6, f_end=0.0, duration=1e-4, profile=EXP, start_sample=0)])
    with pytest.raises(awg.AwgError):
        s.set_chirp_list([dict(tone=1, f_start=50e6, f_end=60e6, duration=1e-4, profile=3, start_sample=0)])
    # equal end frequencies: the same samples as the linear profile
    outs = []
    for prof in (EXP, 0):
        t = awg.Synth(FS)
        t.set_tones([40e6, 70e6], [0.5, 0.5], [0.3, 0.1])
        t.set_chirp_list([dict(tone=0, f_start=45e6, f_end=45e6, duration=2e-4, profile=prof, start_sample=1000)])
        q = torch.empty(80_000, dtype=torch.int16, device="cuda")
        t.render(80_000, q)
        outs.append(q)
    torch.cuda.synchronize()
    assert np.array_equal(outs[0].cpu().numpy(), outs[1].cpu().numpy())
