"""Pins for the CPU oracle: closed forms, the paper's own equations in exact rationals,
invariants and brute force.  None of these re-types the oracle's cascade arithmetic; each pin
reaches the answer by an independent route, chosen so that a dropped term, a wrong sign or a
transposed operand in the oracle fails at least one of them (see the planted-mistake tests)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TWO64 = 1 << 64


def _golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _sdiff(a, b):
    """signed difference of two words mod 2^64"""
    d = (int(a) - int(b)) % TWO64
    return d - TWO64 if d >= TWO64 // 2 else d


# ---------------------------------------------------------------------------------------------
# a1: words
# ---------------------------------------------------------------------------------------------
def test_freq_word_identities(oracle):
    fs = 280e6
    assert oracle.freq_word(fs / 4, fs) == 1 << 62
    assert oracle.freq_word(fs / 2, fs) == 1 << 63
    assert oracle.freq_word(0.0, fs) == 0
    # dyadic fractions of f_s are exact
    for k in (1, 3, 12345, (1 << 20) - 1):
        assert oracle.freq_word(fs * k / (1 << 20), fs) == k << 44
    # the word is within (half an ulp of the IEEE quotient f/fs) + 1/2 word of the exact f/fs 2^64
    rng = np.random.default_rng(1)
    for f in rng.uniform(0, fs, 200):
        exact = Fraction(float(f)) / Fraction(fs) * TWO64
        bound = Fraction(TWO64) * Fraction(math.ulp(float(f) / fs)) / 2 + Fraction(1, 2)
        assert abs(oracle.freq_word(f, fs) - exact) <= bound


def test_phase_word_identities(oracle):
    assert oracle.phase_word(0.0) == 0
    assert oracle.phase_word(math.pi) == 1 << 63
    assert oracle.phase_word(math.pi / 2) == 1 << 62
    assert oracle.phase_word(-math.pi / 2) == 3 << 62
    assert oracle.phase_word(2 * math.pi) == 0
    rng = np.random.default_rng(2)
    for th in rng.uniform(-10, 10, 100):
        w = oracle.phase_word(th)
        # back to radians: within one word of the input modulo 2 pi
        back = 2 * math.pi * w / TWO64
        assert abs(math.remainder(back - th, 2 * math.pi)) < 1e-12


def test_grid_snap_bound_from_paper(oracle):
    g = _golden("freq_grid_280MSps.txt")
    fs, lg = g["fs_hz"], int(g["log2_Ls"])
    Ls = 1 << lg
    half = fs / (2 * Ls)
    assert half < g["stated_max_error_hz"] + 0.06          # 534.0576 Hz, which the paper rounds to 534
    rng = np.random.default_rng(3)
    worst = 0.0
    for f in rng.uniform(1e6, fs / 2, 2000):
        j = oracle.grid_index(f, fs, lg)
        worst = max(worst, abs(f - j * fs / Ls))
        # the grid word is exactly j cycles per L_s samples
        assert oracle.grid_word(j, lg) == (j << (64 - lg)) % TWO64
    assert worst <= half * (1 + 1e-12)


def test_grid_tone_is_periodic(oracle):
    lg = 12
    w = oracle.make_waveform(280e6, [10e6, 33.3e6, 101.7e6], [1, 1, 1], [0.3, 1.0, -2.0], grid_log2=lg)
    for k in range(3):
        a = oracle.phase_words_seq(w, k, 0, 64)
        b = oracle.phase_words_seq(w, k, 1 << lg, 64)
        assert np.array_equal(a, b)
        c = oracle.phase_words_seq(w, k, 5 * (1 << lg) + 17, 64)
        assert np.array_equal(a[17:], c[:-17])


# ---------------------------------------------------------------------------------------------
# static phase: closed form == sequential stepping, brute force up to 2^20
# ---------------------------------------------------------------------------------------------
def test_static_phase_closed_equals_sequential(oracle):
    rng = np.random.default_rng(4)
    for _ in range(3):
        F = int(rng.integers(0, 1 << 62)) * 4 + int(rng.integers(0, 4))
        ph = int(rng.integers(0, 1 << 63)) * 2 + 1
        w = oracle.Waveform(fs=1.0, F=[F], phi_ref=[ph], A=[1.0], has_chirp=[0], n_s=[0], L=[0],
                            d=[[0] * 7], F_end=[0])
        n0 = int(rng.integers(0, 1 << 40))
        seq = oracle.phase_words_seq(w, 0, n0, 1 << 20)
        idx = n0 + np.arange(1 << 20, dtype=np.int64)
        closed = oracle.phase_words_at(w, 0, idx)
        assert np.array_equal(seq, closed)
        # and both are (phi + n F) mod 2^64 computed with Python integers
        for i in (0, 1, 777, (1 << 20) - 1):
            assert int(seq[i]) == (ph + (n0 + i) * F) % TWO64


# ---------------------------------------------------------------------------------------------
# a2: chirp phase against Eq. freqchirp evaluated in exact rationals
# ---------------------------------------------------------------------------------------------
def paper_chirp_turns(i, fs, f_start, f_fin, L, profile):
    """Eq. freqchirp as printed (cases 1 and 2), in turns, exact.  T = L / fs.
    The linear profile is the integral of a linear frequency ramp (the paper names it, Sec. II,
    without printing a formula)."""
    T = Fraction(L) / fs
    if i <= L:
        tau = Fraction(i, L)
        if profile == 1:
            p = (f_fin - f_start) * (Fraction(5, 2) * tau**3 - 3 * tau**4 + tau**5)
        else:
            p = (f_fin - f_start) * tau / 2
        return Fraction(i) / fs * (f_start + p)
    return f_fin * Fraction(i) / fs + T * (f_start - f_fin) / 2


def _chirp_max_word_error(oracle, fs_hz, f0, f1, L, profile, ms, use_closed):
    fs = Fraction(fs_hz)
    F0 = oracle.freq_word(float(f0), fs_hz)
    F1 = oracle.freq_word(float(f1), fs_hz)
    # the frequencies the words actually represent
    fe0 = Fraction(F0) * fs / TWO64
    fe1 = Fraction(F1) * fs / TWO64
    w = oracle.make_waveform(fs_hz, [float(f0)], [1.0], [0.0],
                             chirps=[dict(tone=0, f_start=float(f0), f_end=float(f1), duration=L / fs_hz,
                                          profile=profile, start_sample=0)])
    assert w.L[0] == L
    ms = np.asarray(ms, dtype=np.int64)
    words = oracle.phase_words_at(w, 0, ms) if use_closed else oracle.phase_words_seq(w, 0, 0, int(ms.max()) + 1)[ms]
    worst = 0
    for m, wd in zip(ms, words):
        exact = paper_chirp_turns(int(m), fs, fe0, fe1, L, profile) * TWO64
        worst = max(worst, abs(_sdiff(wd, round(exact))))
    return worst


@pytest.mark.parametrize("profile", [0, 1])
def test_chirp_matches_paper_equation_brute_force(oracle, profile):
    # exact dyadic set-up: every sample 0..L+500 checked through the sequential cascade
    fs = 2.0**28
    for f0, f1 in ((50331648.0, 83886080.0), (83886080.0, 1234567.0), (3.0, 2.0**27 - 5)):
        err = _chirp_max_word_error(oracle, fs, f0, f1, 4096, profile, np.arange(0, 4096 + 500), False)
        assert err <= 1, (f0, f1, err)


@pytest.mark.parametrize("profile", [0, 1])
def test_chirp_matches_paper_equation_long(oracle, profile):
    # 35 ms at 280 MS/s (9.8M samples), sampled through the closed form; the 192-bit words stay
    # within a few 2^-64 turns of the exact rational phase over the whole chirp
    rng = np.random.default_rng(5 + profile)
    L = 9_800_000
    ms = np.concatenate([[0, 1, 2, L - 1, L, L + 1, L + 1000], rng.integers(0, L, 60)])
    err = _chirp_max_word_error(oracle, 280e6, 80.5e6, 179.25e6, L, profile, ms, True)
    assert err <= 4, err
    err = _chirp_max_word_error(oracle, 280e6, 179.9e6, 80.1e6, L, profile, ms, True)
    assert err <= 4, err


def test_chirp_end_phase_golden(oracle):
    g = _golden("chirp_end_phase.txt")
    fs, f0, f1, L = g["fs_hz"], g["f_start_hz"], g["f_fin_hz"], int(g["L"])
    for profile in (0, 1):
        w = oracle.make_waveform(fs, [f0], [1.0], [0.0], chirps=[dict(tone=0, f_start=f0, f_end=f1, duration=L / fs,
                                                                        profile=profile, start_sample=0)])
        end = oracle.chirp_end_word(w, 0)
        expected = int(g["end_phase_turns"] * TWO64) % TWO64
        assert abs(_sdiff(end, expected)) <= 1


@pytest.mark.parametrize("profile", [0, 1])
def test_chirp_frequency_ends(oracle, profile):
    # instantaneous frequency (first difference) starts at F_start and ends at F_end; with the
    # minimum-jerk profile the frequency is flat at both ends (zero slope and curvature)
    fs = 280e6
    L = 28000
    w = oracle.make_waveform(fs, [90e6], [1.0], [0.4], chirps=[dict(tone=0, f_start=90e6, f_end=150e6, duration=L / fs,
                                                                     profile=profile, start_sample=1000)])
    ph = oracle.phase_words_seq(w, 0, 0, 1000 + L + 50).astype(object)
    df = [(int(ph[i + 1]) - int(ph[i])) % TWO64 for i in range(len(ph) - 1)]
    F0, F1 = oracle.freq_word(90e6, fs), oracle.freq_word(150e6, fs)
    assert all(x == F0 for x in df[:1000])
    assert all(x == F1 for x in df[1000 + L:])
    D = F1 - F0
    if profile == 1:
        assert abs(df[1000] - F0) < 1e-6 * abs(D)
        assert abs(df[1000 + L - 1] - F1) < 1e-6 * abs(D)
        mid = df[1000 + L // 2]
        assert abs(mid - (F0 + D / 2)) < 1e-3 * abs(D)
    else:
        slope = (df[1000 + 20001] - df[1000 + 20000])
        assert abs(slope - D / L) <= 2


def test_chirp_closed_equals_sequential_and_exact_integers(oracle):
    rng = np.random.default_rng(6)
    for profile in (0, 1):
        for F0, F1 in ((0, TWO64 - 1), (TWO64 - 1, 0), (int(rng.integers(0, 1 << 63)), int(rng.integers(0, 1 << 63)))):
            L = 3000
            d = oracle.chirp_coefficients(F0, F1, L, profile)
            w = oracle.Waveform(fs=1.0, F=[F0], phi_ref=[12345], A=[1.0], has_chirp=[1], n_s=[700], L=[L], d=[d], F_end=[F1])
            seq = oracle.phase_words_seq(w, 0, 0, 700 + L + 300)
            closed = oracle.phase_words_at(w, 0, np.arange(700 + L + 300))
            assert np.array_equal(seq, closed)
            for m in (0, 1, 2, 5, 999, L):
                py = oracle.cascade_state(d, m)
                assert oracle.cascade_state_c(d, m) == py
                assert int(seq[700 + m]) == (12345 + 700 * F0 + (py[0] >> 128)) % TWO64


# ---------------------------------------------------------------------------------------------
# single tone, Dirichlet kernel, Parseval, brute force at tiny K
# ---------------------------------------------------------------------------------------------
def test_single_tone_special_points(oracle):
    fs = 280e6
    w = oracle.make_waveform(fs, [fs / 4], [0.7], [0.0])
    x = oracle.render(w, 0, 8)
    assert np.allclose(x, 0.7 * np.array([0, 1, 0, -1, 0, 1, 0, -1]), atol=1e-15)
    th = 0.3
    w = oracle.make_waveform(fs, [fs / 2], [1.3], [th])
    x = oracle.render(w, 5, 6)
    expect = 1.3 * np.array([(-1) ** n for n in range(5, 11)]) * math.sin(th)
    assert np.allclose(x, expect, atol=1e-14)


def test_dirichlet_closed_form(oracle):
    # K equal-amplitude, equally spaced, zero-phase tones:
    # sum_k sin((w0 + k dw) n) = sin((w0 + (K-1) dw / 2) n) sin(K dw n / 2) / sin(dw n / 2)
    K = 50
    F0 = 0x1234_5678_9ABC_DE00
    dF = 1 << 52                      # the centre word F0 + (K-1) dF / 2 is an integer
    A = 1.0 / K
    w = oracle.Waveform(fs=1.0, F=[(F0 + k * dF) % TWO64 for k in range(K)], phi_ref=[0] * K, A=[A] * K,
                        has_chirp=[0] * K, n_s=[0] * K, L=[0] * K, d=[[0] * 7] * K, F_end=[0] * K)
    N = 4095
    x = oracle.render(w, 1, N)
    Fc = F0 + (K - 1) * dF // 2

    def sin_turn(num, den_bits):
        # sin(2 pi num / 2^den_bits), with the argument reduced exactly first
        r = num % (1 << den_bits)
        if r >= 1 << (den_bits - 1):
            r -= 1 << den_bits
        return math.sin(2 * math.pi * r / (1 << den_bits))

    ref = np.empty(N)
    for i in range(N):
        n = i + 1
        ref[i] = A * sin_turn(Fc * n, 64) * sin_turn(K * dF * n, 65) / sin_turn(dF * n, 65)
    assert np.max(np.abs(x - ref)) < 1e-12


def test_parseval_over_whole_period(oracle):
    lg = 12
    Ls = 1 << lg
    rng = np.random.default_rng(7)
    js = rng.choice(np.arange(1, Ls // 2), size=20, replace=False)
    A = rng.uniform(0.1, 1.0, 20)
    w = oracle.Waveform(fs=1.0, F=[oracle.grid_word(int(j), lg) for j in js],
                        phi_ref=[oracle.phase_word(t) for t in rng.uniform(0, 6.28, 20)], A=list(A),
                        has_chirp=[0] * 20, n_s=[0] * 20, L=[0] * 20, d=[[0] * 7] * 20, F_end=[0] * 20)
    x = oracle.render(w, 123, Ls)
    assert abs(np.mean(x * x) - np.sum(A * A) / 2) < 1e-12


def _brute_force_turns(oracle, w, k, n, fs_hz):
    """Exact rational turn of tone k at sample n from Eq. freqchirp (no cascade, no words)."""
    fs = Fraction(fs_hz)
    phi0 = Fraction(w.phi_ref[k], TWO64)
    f_static = Fraction(w.F[k]) * fs / TWO64
    if not w.has_chirp[k] or n < w.n_s[k]:
        return phi0 + f_static * n / fs
    # the chirp starts from the tone's phase at n_s
    start = phi0 + f_static * w.n_s[k] / fs
    # the chirp's own start frequency is the d_1-consistent word of f_start; recover it from the
    # waveform description the test built
    return start + paper_chirp_turns(n - w.n_s[k], fs, w._f0[k], w._f1[k], w.L[k], w._prof[k])


def test_brute_force_tiny_waveforms(oracle):
    from paper_2403_15582_gb300 import workloads as wl
    for seed in (0, 1, 2):
        wk = wl.tiny(seed=seed, K=3, n_samples=3000)
        w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps)
        # remember the word-exact chirp frequencies for the brute-force phase
        w._f0, w._f1, w._prof = {}, {}, {}
        for c in wk.chirps:
            k = c["tone"]
            w._f0[k] = Fraction(oracle.freq_word(c["f_start"], wk.fs)) * Fraction(wk.fs) / TWO64
            w._f1[k] = Fraction(oracle.freq_word(c["f_end"], wk.fs)) * Fraction(wk.fs) / TWO64
            w._prof[k] = c["profile"]
        x = oracle.render(w, 0, wk.n_samples)
        ref = np.zeros(wk.n_samples)
        for k in range(w.K):
            for n in range(wk.n_samples):
                t = _brute_force_turns(oracle, w, k, n, wk.fs)
                t = t - math.floor(t)
                if t >= Fraction(1, 2):
                    t -= 1
                ref[n] += w.A[k] * math.sin(2 * math.pi * float(t))
        assert np.max(np.abs(x - ref)) < 1e-13, seed


def test_quantize_rounding_and_clamp(oracle):
    x = np.array([0.0, 2.5, 3.5, -2.5, -3.5, 0.49999, 40000.0, -40000.0, 32766.5, -32766.5])
    q = oracle.quantize(x, 32767.0)
    assert q.tolist() == [0, 2, 4, -2, -4, 0, 32767, -32767, 32766, -32766]
    # default full scale never clips: FS = sum |A|
    w = oracle.make_waveform(280e6, [10e6, 20e6], [0.5, -0.25], [0.0, 0.0])
    assert w.full_scale() == 0.75


def test_threads_and_sampled_paths_agree(oracle):
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.tiny(seed=3, K=7, n_samples=5000)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps)
    a = oracle.render(w, 100, 5000, nthreads=1)
    b = oracle.render(w, 100, 5000, nthreads=4)
    assert np.array_equal(a, b)
    idx = np.array([100, 101, 2500, 5099])
    c = oracle.render_at(w, idx)
    assert np.array_equal(c, a[idx - 100])


# ---------------------------------------------------------------------------------------------
# planted mistakes: each plausible error in the oracle's chirp derivation fails a pin
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mistake", ["sign", "drop_m5", "transpose", "linear_half"])
def test_pins_catch_planted_mistakes(oracle, monkeypatch, mistake):
    good = oracle.chirp_phase_poly

    def bad(F_start, F_end, L, profile):
        D = int(F_end) - int(F_start)
        if mistake == "sign":
            D = -D
        if mistake == "transpose":
            F_start, D = F_end, -D
        if profile == 1:
            if mistake == "drop_m5":
                return lambda m: int(F_start) * m + Fraction(D * (5 * m**4 * L**2 + 2 * m**6), 2 * L**5)
            return lambda m: int(F_start) * m + Fraction(D * (5 * m**4 * L**2 - 6 * m**5 * L + 2 * m**6), 2 * L**5)
        if mistake == "linear_half":
            return lambda m: int(F_start) * m + Fraction(D * m * m, L)
        return lambda m: int(F_start) * m + Fraction(D * m * m, 2 * L)

    monkeypatch.setattr(oracle, "chirp_phase_poly", bad)
    profile = 0 if mistake == "linear_half" else 1
    err = _chirp_max_word_error(oracle, 2.0**28, 50331648.0, 83886080.0, 4096, profile, np.arange(0, 4200, 7), False)
    assert err > 1 << 40
    monkeypatch.setattr(oracle, "chirp_phase_poly", good)


def test_repeated_chirps_fold_continuously(oracle):
    """A tone chirped twice: inside and after the second chirp, the folded oracle state follows
    the exact rational phase of Eq. freqchirp applied twice in a row (case 2 between them)."""
    fs = 2.0**28
    f0, f1, f2 = 50331648.0, 83886080.0, 16777216.0
    L1, L2, n1, n2 = 4096, 2048, 100, 9000
    chirps = [dict(tone=0, f_start=f0, f_end=f1, duration=L1 / fs, profile=1, start_sample=n1),
              dict(tone=0, f_start=f1, f_end=f2, duration=L2 / fs, profile=0, start_sample=n2)]
    Fr = Fraction(fs)
    e0, e1, e2 = (Fraction(oracle.freq_word(x, fs)) * Fr / TWO64 for x in (f0, f1, f2))
    th = 0.7
    start1 = Fraction(oracle.phase_word(th), TWO64) + e0 * n1 / Fr
    end1 = start1 + paper_chirp_turns(L1, Fr, e0, e1, L1, 1)

    def exact_turns(n):
        if n <= n1 + L1:
            return start1 + paper_chirp_turns(n - n1, Fr, e0, e1, L1, 1)
        if n < n2:
            return end1 + e1 * (n - n1 - L1) / Fr
        start2 = end1 + e1 * (n2 - n1 - L1) / Fr
        return start2 + paper_chirp_turns(n - n2, Fr, e1, e2, L2, 0)

    for n0 in (n2 - 50, n2 + 1000, n2 + L2 - 5):
        w = oracle.make_waveform_window(fs, [f0], [1.0], [th], chirps, n0, 64)
        words = oracle.phase_words_seq(w, 0, n0, 64)
        for i, wd in enumerate(words):
            assert abs(_sdiff(wd, round(exact_turns(n0 + i) * TWO64))) <= 3, (n0, i)


# ---------------------------------------------------------------------------------------------
# amplitude ramps a_j[i] (Eq. dynamicandstatic): A -> A_end along the linear or minimum-jerk
# profile s(tau) (10 tau^3 - 15 tau^4 + 6 tau^5, the minimum-jerk trajectory of Eq. freqchirp)
# ---------------------------------------------------------------------------------------------
def _check_amp_pins(amp, A0, A1, ns, L, profile):
    """Pins of a ramp sampler amp(samples) -> values: constant outside, exact ends, midpoint
    (A0 + A1)/2, point symmetry s(tau) + s(1 - tau) = 1, and the slopes the profile fixes."""
    dA = A1 - A0
    m = np.arange(0, L + 1)
    a = amp(ns + m)
    assert np.all(amp(np.array([ns - 5, ns - 1, ns])) == A0)
    assert np.all(amp(np.array([ns + L, ns + L + 1, ns + 10 * L])) == A1)
    assert abs(a[L // 2] - 0.5 * (A0 + A1)) <= 1e-12 * abs(dA)
    assert np.max(np.abs(a + a[::-1] - (A0 + A1))) <= 1e-12 * abs(dA)
    d = np.diff(a)
    if profile == 0:
        assert np.max(np.abs(d - dA / L)) <= 1e-12 * abs(dA)
    else:
        assert abs(d[0]) <= 11 * abs(dA) / L**3 and abs(d[-1]) <= 11 * abs(dA) / L**3
        assert abs(d[L // 2] / (dA / L) - 1.875) <= 2e-3       # s'(1/2) = 30/16


@pytest.mark.parametrize("profile", [0, 1])
def test_amp_ramp_pins(oracle, profile):
    for A0, A1, ns, L in [(0.25, 1.0, 1000, 4000), (1.0, 0.0, 0, 1000), (-0.5, 0.75, 123456789, 20000)]:
        _check_amp_pins(lambda n: oracle.amp_at(A0, profile, ns, L, A1, n), A0, A1, ns, L, profile)


@pytest.mark.parametrize("mutant", ["swapped_coeffs", "profile_swap", "missing_cube", "length_plus_one"])
def test_amp_pins_catch_planted_mistakes(oracle, mutant):
    A0, A1, ns, L = 0.25, 1.0, 1000, 4000

    def amp(n):
        n = np.asarray(n, dtype=np.float64)
        tau = np.clip((n - ns) / (L + 1 if mutant == "length_plus_one" else L), 0.0, 1.0)
        if mutant == "swapped_coeffs":
            s = tau**3 * (6 - 15 * tau + 10 * tau**2)
        elif mutant == "profile_swap":
            s = tau
        elif mutant == "missing_cube":
            s = np.where((tau > 0) & (tau < 1), 10 - 15 * tau + 6 * tau**2, tau)
        else:
            s = tau**3 * (10 - 15 * tau + 6 * tau**2)
        return A0 + (A1 - A0) * s

    with pytest.raises(AssertionError):
        _check_amp_pins(amp, A0, A1, ns, L, 1)


def test_amp_ramp_seen_through_the_render(oracle):
    """A tone at f_s/4 with phase pi/2 reads sin = 1 exactly at every fourth sample, so the
    rendered sum there is the amplitude itself: the ramp enters x[n] as a_j[i] sin(phi_j[i])."""
    fs = 2.0**28
    w = oracle.make_waveform(fs, [fs / 4], [0.3], [np.pi / 2])
    oracle.add_ramps(w, [dict(tone=0, amp_end=0.9, duration=4000 / fs, profile=1, start_sample=800)])
    x = oracle.render(w, 0, 6000)
    n = np.arange(0, 6000, 4)
    assert np.array_equal(x[n], oracle.amp_at(0.3, 1, 800, 4000, 0.9, n))


# ---------------------------------------------------------------------------------------------
# exponential chirps (named in Sec. II, formula not printed): the frequency moves geometrically
# from F_start to F_end, the phase is its integral
# ---------------------------------------------------------------------------------------------
EXP = 2


def _exp_wave(oracle, fs, f0, f1, L, n_s=0, phase=0.0):
    return oracle.make_waveform(fs, [f0], [1.0], [phase], chirps=[dict(tone=0, f_start=f0, f_end=f1, duration=L / fs,
                                                                        profile=EXP, start_sample=n_s)])


def _exp_checks(oracle, fs=280e6, cases=((90e6, 150e6, 100_000), (179e6, 81e6, 60_000), (1e6, 60e6, 200_000))):
    """Worst violation of each exponential-chirp pin, relative to its tolerance (<= 1 passes)."""
    worst = {"law": 0.0, "reversal": 0.0, "taylor": 0.0, "ends": 0.0}
    for f0, f1, L in cases:
        F0, F1 = oracle.freq_word(f0, fs), oracle.freq_word(f1, fs)
        r = F1 / F0
        alpha = math.log(r) / L
        w = _exp_wave(oracle, fs, f0, f1, L)
        ph0 = int(w.phi_ref[0])
        ms = np.array(sorted({0, 1, L // 3, L // 2, L - 2, L - 1} | set(range(0, L, L // 7))), dtype=np.int64)
        a = oracle.phase_words_at(w, 0, ms)
        b = oracle.phase_words_at(w, 0, ms + 1)
        # (1) per-sample increments follow the geometric law: the integral of F0 r^(t/L) over one
        # sample is F(m + 1/2) sinh(alpha/2) / (alpha/2) = F(m + 1/2) (1 + alpha^2/24 + ...)
        for m, x, y in zip(ms, a, b):
            delta = (int(y) - int(x)) % TWO64
            Fm = F0 * r ** ((m + 0.5) / L)
            worst["law"] = max(worst["law"], abs(delta / Fm - 1 - alpha * alpha / 24) / (alpha**4 + 2e-13))
        # (2) time reversal: R_{0->1}(m) + R_{1->0}(L - m) = R_{0->1}(L) (the same frequency curve
        # read backwards covers the rest of the phase)
        wr = _exp_wave(oracle, fs, f1, f0, L)
        phr = int(wr.phi_ref[0])
        total = (int(oracle.phase_words_at(w, 0, [L])[0]) - ph0) % TWO64
        rev = oracle.phase_words_at(wr, 0, L - ms)
        for x, y in zip(a, rev):
            s = ((int(x) - ph0) + (int(y) - phr)) % TWO64
            worst["reversal"] = max(worst["reversal"], abs(_sdiff(s, total)) / 2**20)
        # (4) the end: Phi(L) is the post-chirp anchor, then steps of exactly F_end
        tail = oracle.phase_words_seq(w, 0, L - 1, 4)
        inc = [(int(tail[i + 1]) - int(tail[i])) % TWO64 for i in range(3)]
        ok = inc[1] == F1 and inc[2] == F1 and abs(inc[0] / (F1 * r ** (-0.5 / L)) - 1 - alpha * alpha / 24) < alpha**4 + 2e-13
        ok = ok and int(tail[1]) == oracle.chirp_end_word(w, 0)
        worst["ends"] = max(worst["ends"], 0.0 if ok else 2.0)
    # (3) near r = 1 the exponential chirp is the (exactly pinned) linear chirp plus the Taylor
    # terms of the exponential in x = D / F_start: R_exp - R_lin = F_s L [x^2 (u^3/6 - u^2/4) +
    # x^3 (u^2/6 - u^3/6 + u^4/24)] + O(x^4), u = m / L
    fs, L = 280e6, 100_000
    for f0, f1 in ((100e6, 100.003e6), (120e6, 119.9955e6)):
        F0, F1 = oracle.freq_word(f0, fs), oracle.freq_word(f1, fs)
        x = Fraction(F1 - F0, F0)
        we = _exp_wave(oracle, fs, f0, f1, L)
        wl = oracle.make_waveform(fs, [f0], [1.0], [0.0], chirps=[dict(tone=0, f_start=f0, f_end=f1, duration=L / fs,
                                                                        profile=0, start_sample=0)])
        ms = np.arange(0, L + 1, L // 10, dtype=np.int64)
        pe, pl = oracle.phase_words_at(we, 0, ms), oracle.phase_words_at(wl, 0, ms)
        for m, e, l in zip(ms, pe, pl):
            u = Fraction(int(m), L)
            corr = F0 * L * (x**2 * (u**3 / 6 - u**2 / 4) + x**3 * (u**2 / 6 - u**3 / 6 + u**4 / 24))
            worst["taylor"] = max(worst["taylor"], abs(_sdiff(e, (int(l) + round(corr)) % TWO64)) / 2**22)
    return worst


def test_exp_chirp_pins(oracle):
    worst = _exp_checks(oracle)
    assert all(v <= 1 for v in worst.values()), worst
    # r = 1: the static tone's words exactly
    fs = 280e6
    w = _exp_wave(oracle, fs, 77e6, 77e6, 5000, n_s=300, phase=1.1)
    s = oracle.make_waveform(fs, [77e6], [1.0], [1.1])
    assert np.array_equal(oracle.phase_words_seq(w, 0, 0, 6000), oracle.phase_words_seq(s, 0, 0, 6000))
    # sequential and closed-form paths agree, and a zero frequency is refused
    w = _exp_wave(oracle, fs, 30e6, 90e6, 7000, n_s=123, phase=0.7)
    assert np.array_equal(oracle.phase_words_seq(w, 0, 0, 7500), oracle.phase_words_at(w, 0, np.arange(7500)))
    with pytest.raises(ValueError):
        _exp_wave(oracle, fs, 0.0, 90e6, 7000)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_exp_pins_catch_planted_mistakes(oracle, mutant):
    import ctypes
    knob = ctypes.c_int.in_dll(oracle.lib(), "oracle_exp_plant")
    knob.value = mutant
    try:
        worst = _exp_checks(oracle)
    finally:
        knob.value = 0
    assert max(worst.values()) > 1, worst
