"""Accounting of a half-precision (FP16 / half2) sine, the speed-up the paper's Appendix describes,
against the <= 1 LSB bar of the int16 output.

FP16 carries 11 significant bits.  A phase held in FP16 turns (in [-1/2, 1/2)) is off by up to
2^-13 turn, and a sine rounded to FP16 by up to 2^-12; per unit amplitude that is at most
2 pi 2^-13 + 2^-12 = 1.01e-3, against 1 LSB = 3.05e-5 of a full scale sum |A|.  So one tone alone
can miss by up to 33 LSB; K tones with random phases add their errors like noise, about
3e-4 sqrt(sum A^2) rms, which shrinks against sum |A| as 1/sqrt(K).  The test evaluates the sum
that way (phase and sine in FP16, accumulation in FP32) on the oracle's phase words and checks
the error against that bound: above 1 LSB for one tone and for the 100-tone comb (about 2.5 LSB),
about 1 LSB at the tails for 1000 chirping tones.  That is why the library keeps its sines in
FP32 (SFU or rotator), which hold the bar at every K."""
import numpy as np

FS_HZ = 280e6


def _half_sum(words, amps):
    """sum_k A_k sin(2 pi u_k) with u_k the signed turn in FP16 and the sine rounded to FP16."""
    u = (words.astype(np.int64).astype(np.float64) * 2.0**-64).astype(np.float16)
    s = np.sin(2 * np.pi * u.astype(np.float64)).astype(np.float16).astype(np.float32)
    return (s * np.asarray(amps, dtype=np.float32)[:, None]).sum(axis=0, dtype=np.float32)


def _case(oracle, f, a, th, chirps, n0, n):
    w = oracle.make_waveform(FS_HZ, f, a, th, chirps)
    words = np.stack([oracle.phase_words_seq(w, k, n0, n) for k in range(w.K)])
    x_half = _half_sum(words, a).astype(np.float64)
    x_ref = oracle.render(w, n0, n)
    FS = w.full_scale()
    err_lsb = float(np.max(np.abs(x_half - x_ref))) * 32767.0 / FS
    bound_lsb = (2 * np.pi * 2.0**-13 + 2.0**-12 + 2.0**-20) * float(np.sum(np.abs(a))) * 32767.0 / FS
    return err_lsb, bound_lsb


def test_half_precision_sine_misses_one_lsb(oracle):
    rng = np.random.default_rng(0)
    # one tone, the 100-tone static comb (80-179 MHz, A = 1/100), 1000 tones chirping 80-180 MHz
    err, bound = _case(oracle, [97.3e6], [1.0], [0.4], [], 0, 4096)
    assert 4.0 < err <= bound, (err, bound)
    f = 80e6 + 1e6 * np.arange(100)
    err, bound = _case(oracle, f, np.full(100, 0.01), rng.uniform(0, 2 * np.pi, 100), [], 0, 4096)
    assert 1.0 < err <= bound, (err, bound)
    K = 1000
    f0, f1 = rng.uniform(80e6, 180e6, K), rng.uniform(80e6, 180e6, K)
    a = rng.uniform(0.5, 1.0, K) / K
    chirps = [dict(tone=k, f_start=float(f0[k]), f_end=float(f1[k]), duration=35e-3, profile=k % 2, start_sample=0)
              for k in range(K)]
    err, bound = _case(oracle, f0, a, rng.uniform(0, 2 * np.pi, K), chirps, 4_000_000, 1024)
    assert 0.3 < err <= bound, (err, bound)
