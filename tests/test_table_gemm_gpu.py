"""Periodic table as a split-precision tcgen05 GEMM, against the CPU oracle.

Error model, in int16 LSBs of the record's full scale (1 LSB = FS / 32767).  The FP32 sum of one
sample carries (a) the tensor cores' FP32 accumulation over 3 x 2K / 16 MMA steps, a random walk of
rounding errors of the running sum, and (b) per product term the residual of the hi + lo split
(about u^2 of the term, u = 2^-8 for BF16, 2^-11 for FP16; the dropped lo*lo product is of the
same order) and the operand sines (A operand: SFU sine/cosine of the phase's top 32 bits, below
4.6e-7; B operand below 5e-8).  Both add up as random walks: over 10,000 tones at 2^24 samples
(FS = max |x| of about 100, 1 LSB about 3e-3) they give a floor of about 0.3 LSB, measured at
1.0e-3 (FP16) and 9.5e-4 (BF16).  The tests bound the FP32 error by `FP32_BOUND_LSB` and the int16
codes by 1 LSB: a systematic error of one LSB (a dropped hi*lo product is 2^-8 of every term, tens of
LSB; a wrong sign or index, far more) breaks both."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
FP32_BOUND_LSB = 0.75     # the FP32 sum against the FP64 oracle, in LSB of the full scale


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def lsb_errors(x, q, x_ref, FS):
    """(FP32 error, int16 error) against the oracle, both in LSB of FS."""
    lsb = FS / 32767.0
    xe = float(np.max(np.abs(x.astype(np.float64) - x_ref))) / lsb
    qe = int(np.max(np.abs(q.astype(np.int32) - oracle_codes(x_ref, FS))))
    return xe, qe


def oracle_codes(x_ref, FS):
    import oracle
    return oracle.quantize(x_ref, FS).astype(np.int32)


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
    x_ref = oracle.render(w, 0, N, nthreads=NTHREADS)
    xe, qe = lsb_errors(xf.cpu().numpy(), xq.cpu().numpy(), x_ref, w.full_scale())
    print(f"table GEMM {K} tones x 2^{lg} prec {precision}: FP32 {xe:.3f} LSB, int16 {qe} LSB")
    assert xe <= FP32_BOUND_LSB and qe <= 1, (xe, qe)


def test_table_gemm_10000_tones_2e24(awg, oracle):
    """10,000 grid tones, 2^24 samples, full scale FS = max |x| of the record: FP16 and BF16 hi+lo
    both within FP32_BOUND_LSB (FP32 sum) and 1 LSB (int16) of the FP64 oracle on a contiguous
    window of 2^20 samples (rows of 256 samples, n1 from 20480) and at sampled indices across the
    record; the direct-sum render of the same record within 1 LSB at the same samples."""
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
    w0, wn = 20480 * 256, 1 << 20
    x_idx = oracle.render_at(w, idx, nthreads=NTHREADS)
    x_win = oracle.render(w, w0, wn, nthreads=NTHREADS)
    results = {}
    for prec in (1, 0):
        q = torch.empty(N, dtype=torch.int16, device="cuda")
        x = torch.empty(N, dtype=torch.float32, device="cuda")
        s.table_gemm(lg, prec, q, x)
        torch.cuda.synchronize()
        xh, qh = x.cpu().numpy(), q.cpu().numpy()
        e_idx = lsb_errors(xh[idx], qh[idx], x_idx, FS)
        e_win = lsb_errors(xh[w0:w0 + wn], qh[w0:w0 + wn], x_win, FS)
        results["fp16" if prec else "bf16"] = (e_idx, e_win)
        assert max(e_idx[0], e_win[0]) <= FP32_BOUND_LSB, results
        assert max(e_idx[1], e_win[1]) <= 1, results
    print("table GEMM 10k x 2^24 (FP32 LSB, int16 LSB) at samples / on the window:", results)
    # the direct-sum render of the same periodic record agrees with the GEMM
    qd = torch.empty(N, dtype=torch.int16, device="cuda")
    s.seek(0)
    s.render(N, qd)
    torch.cuda.synchronize()
    assert np.max(np.abs(qd.cpu().numpy()[idx].astype(np.int32) - oracle_codes(x_idx, FS))) <= 1


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
