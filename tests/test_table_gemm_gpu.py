"""Periodic table as a split-precision tcgen05 GEMM, against the CPU oracle.

Error model (written out in `gemm_bound`): an operand x split into hi + lo halves with unit
roundoff u (BF16 2^-8, FP16 2^-11) is represented to u^2 |x|; the three products hi*hi + hi*lo +
lo*hi miss lo*lo, so each term a*b carries at most 3 u^2 |a b|; over the 2K terms of one sample
that is 3 u^2 * 2 sum|A|, plus the FP32 accumulation of 6K products (<= 6K 2^-24 of the running
magnitude, bounded by 2 sum|A|) and the operand sines: the A operand's SFU sine and cosine of the
phase word's top 32 bits (< 3.6e-7 from the SFU, < 1e-7 from the 24-bit rounding of the turn)
and the B operand's corrected sincospi (< 5e-8), so < 5.1e-7 per product term."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def gemm_bound(amps, precision):
    u = 2.0**-8 if precision == 0 else 2.0**-11
    S = float(np.sum(np.abs(amps)))
    K = len(amps)
    return 2 * S * (3 * u * u + 6 * K * 2.0**-24 + 5.1e-7)


def _grid_set(K, lg, seed, fs=280e6):
    rng = np.random.default_rng(seed)
    f = rng.uniform(1e6, 139e6, K)
    a = rng.uniform(0.5, 1.0, K)
    th = rng.uniform(0, 2 * np.pi, K)
    return fs, f, a, th


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lg,K", [(15, 100), (16, 37), (17, 300)])
def test_table_gemm_small_all_samples(awg, oracle, precision, lg, K):
    fs, f, a, th = _grid_set(K, lg, lg * 7 + K)
    s = awg.Synth(fs)
    s.set_tones(f, a, th, grid_log2=lg)
    N = 1 << lg
    xq = torch.empty(N, dtype=torch.int16, device="cuda")
    xf = torch.empty(N, dtype=torch.float32, device="cuda")
    s.table_gemm(lg, precision, xq, xf)
    torch.cuda.synchronize()
    assert s.device_status() == 0
    w = oracle.make_waveform(fs, f, a, th, grid_log2=lg)
    x_ref = oracle.render(w, 0, N, nthreads=8)
    err = np.max(np.abs(xf.cpu().numpy().astype(np.float64) - x_ref))
    assert err <= gemm_bound(a, precision), (err, gemm_bound(a, precision))
    q_ref = oracle.quantize(x_ref, w.full_scale())
    assert np.max(np.abs(xq.cpu().numpy().astype(np.int32) - q_ref)) <= 1


def test_table_gemm_10000_tones_2e24(awg, oracle):
    """10,000 grid tones, 2^24 samples: FP16 hi+lo within 1 LSB of the FP64 oracle at sampled
    indices (full scale = max |x| of the record); BF16 hi+lo error reported and bounded; both
    compared with the direct-sum render of the same record."""
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.table_10000(seed=0)
    lg = wk.grid_log2
    N = 1 << lg
    s = awg.Synth(wk.fs)
    s.set_tones(wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=lg)
    xf = torch.empty(N, dtype=torch.float32, device="cuda")
    s.table_gemm(lg, 1, None, xf)
    torch.cuda.synchronize()
    FS = float(xf.abs().max())
    s.set_full_scale(FS)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, grid_log2=lg)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, N, 300), [0, 1, 255, 256, N - 1]]))
    x_ref = oracle.render_at(w, idx, nthreads=8)
    q_ref = oracle.quantize(x_ref, FS)
    results = {}
    for prec in (1, 0):
        q = torch.empty(N, dtype=torch.int16, device="cuda")
        x = torch.empty(N, dtype=torch.float32, device="cuda")
        s.table_gemm(lg, prec, q, x)
        torch.cuda.synchronize()
        xe = np.abs(x.cpu().numpy()[idx].astype(np.float64) - x_ref)
        qe = np.abs(q.cpu().numpy()[idx].astype(np.int32) - q_ref)
        results[prec] = (float(xe.max()), int(qe.max()))
        assert xe.max() <= gemm_bound(wk.amp, prec)
    assert results[1][1] <= 1, results
    # the direct-sum render of the same periodic record agrees with the GEMM
    qd = torch.empty(N, dtype=torch.int16, device="cuda")
    s.seek(0)
    s.render(N, qd)
    torch.cuda.synchronize()
    assert np.max(np.abs(qd.cpu().numpy()[idx].astype(np.int32) - q_ref)) <= 1
    print("table GEMM 10k x 2^24: max |err| FP16 %.3g (%d LSB), BF16 %.3g (%d LSB)" %
          (results[1][0], results[1][1], results[0][0], results[0][1]))


def test_table_gemm_argument_errors(awg):
    s = awg.Synth(280e6)
    s.set_tones([10e6, 20.1234567e6], [1, 1], [0, 0])            # not on the 2^16 grid
    q = torch.empty(1 << 16, dtype=torch.int16, device="cuda")
    with pytest.raises(awg.AwgError):
        s.table_gemm(16, 0, q)
    s.set_tones([10e6, 20e6], [1, 1], [0, 0], grid_log2=16)
    with pytest.raises(awg.AwgError):
        s.table_gemm(14, 0, q)                                   # record shorter than one tile
    with pytest.raises(awg.AwgError):
        s.table_gemm(16, 2, q)                                   # unknown precision
    s.set_chirps([0], [10e6], [30e6], [1e-4], [0], [0])
    with pytest.raises(awg.AwgError):
        s.table_gemm(16, 0, q)                                   # a tone holds a chirp
