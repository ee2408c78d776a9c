"""Host-side logic of the library, checked without a GPU: the exported symbols match the header,
and the set-up words the library computes (its own exact-integer code) equal the oracle's
(exact rationals), bit for bit."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "awg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(awg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(awglib):
    import ctypes
    from paper_2403_15582_gb300 import binding
    declared = _header_symbols()
    assert len(declared) >= 20
    lib = ctypes.CDLL(binding.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    bound = sorted(n for n, _, _ in binding.SIGNATURES)
    assert bound == declared


def test_header_limits_match_the_binding(awglib):
    """The noalloc limits the binding exposes are the #defines of include/awg.h (the library itself
    ties those to its fixed scratch with static_asserts)."""
    import os
    import re
    from paper_2403_15582_gb300 import binding
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "awg.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(AWG_\w+)\s+(\d+)", hdr)}
    assert defs["AWG_NOALLOC_MAX_RECORDS"] == binding.NOALLOC_MAX_RECORDS
    assert defs["AWG_NOALLOC_MAX_SLOTS"] == binding.NOALLOC_MAX_SLOTS


def test_version_and_error_string(awglib):
    assert awglib.lib().awg_version() >= 10000
    with pytest.raises(awglib.AwgError) as e:
        awglib.freq_word(300e6, 280e6)
    assert e.value.code == awglib.AWG_EINVAL
    assert "fs" in awglib.lib().awg_last_error().decode()


def test_freq_and_phase_words_match_oracle(awglib, oracle):
    rng = np.random.default_rng(11)
    for fs in (280e6, 50e6, 2.0**28, 1.0):
        for f in np.concatenate([rng.uniform(0, fs, 300), [0.0, fs / 4, fs / 2, np.nextafter(fs, 0)]]):
            assert awglib.freq_word(f, fs) == oracle.freq_word(f, fs)
    for th in np.concatenate([rng.uniform(-100, 100, 300), [0.0, math.pi, -math.pi, 2 * math.pi, -1e-300]]):
        assert awglib.phase_word(th) == oracle.phase_word(th)


def test_grid_words_match_oracle(awglib, oracle):
    rng = np.random.default_rng(12)
    for lg in (12, 18, 24):
        for f in rng.uniform(0, 280e6, 200):
            w, j = awglib.grid_word(f, 280e6, lg)
            assert j == oracle.grid_index(f, 280e6, lg)
            assert w == oracle.grid_word(j, lg)


def test_chirp_length_rule(awglib, oracle):
    for dur in (35e-3, 1e-3, 0.1e-3, 2e-3, 1 / 280e6, 0.5 / 280e6 * 3):
        assert awglib.chirp_length(dur, 280e6) == oracle.chirp_length(dur, 280e6)
    for bad in (0.0, -1.0, float("nan"), 1e3, 0.4 / 280e6):
        with pytest.raises(awglib.AwgError):
            awglib.chirp_length(bad, 280e6)


@pytest.mark.parametrize("profile", [0, 1])
def test_chirp_coefficients_match_oracle_bitwise(awglib, oracle, profile):
    rng = np.random.default_rng(13 + profile)
    M = 1 << 64
    cases = [(0, M - 1, 1), (M - 1, 0, 2), (123, 456, 3), (1 << 63, (1 << 63) + 1, 7), (0, M - 1, (1 << 28) - 1),
             (M - 1, 0, (1 << 28) - 1), (5, 5, 1000)]
    for _ in range(40):
        cases.append((int(rng.integers(0, M, dtype=np.uint64)), int(rng.integers(0, M, dtype=np.uint64)),
                      int(rng.integers(1, 1 << 28))))
    for F0, F1, L in cases:
        assert awglib.chirp_coeffs(F0, F1, L, profile) == oracle.chirp_coefficients(F0, F1, L, profile), (F0, F1, L)



def test_chirp_coefficients_round_exact_ties_to_even(awglib, oracle):
    """Power-of-two lengths make some minimum-jerk c_k 2^128 land exactly on a half (L^5 = 2^130
    for L = 2^26): the library's quotient rounding must send those to even, as the oracle's exact
    fractions do.  The cases are checked to contain such ties.  (Linear coefficients never tie:
    their denominator 2L holds at most 2^29.)"""
    profile = 1
    import math
    from fractions import Fraction
    rng = np.random.default_rng(5)
    M = 1 << 64
    ties = 0
    for L in (1 << 26, 1 << 27, 1 << 25, 1 << 24, 3 << 24):
        for _ in range(10):
            F0, F1 = int(rng.integers(0, M, dtype=np.uint64)), int(rng.integers(0, M, dtype=np.uint64))
            P = oracle.chirp_phase_poly(F0, F1, L, profile)
            vals = [P(m) for m in range(7)]
            for k in range(1, 7):
                ck = sum(((-1) ** (k - j)) * math.comb(k, j) * vals[j] for j in range(k + 1))
                ties += (Fraction(ck) * (1 << 128)).denominator == 2
            assert awglib.chirp_coeffs(F0, F1, L, profile) == oracle.chirp_coefficients(F0, F1, L, profile), (F0, F1, L)
    assert ties >= 2, ties

def test_chirp_coefficient_errors(awglib):
    with pytest.raises(awglib.AwgError):
        awglib.chirp_coeffs(1, 2, 0, 0)
    with pytest.raises(awglib.AwgError):
        awglib.chirp_coeffs(1, 2, 1 << 28, 1)
    with pytest.raises(awglib.AwgError):
        awglib.chirp_coeffs(1, 2, 100, 3)
    with pytest.raises(awglib.AwgError):       # exponential chirps need both ends > 0
        awglib.chirp_coeffs(0, 2, 100, 2)
    with pytest.raises(awglib.AwgError):
        awglib.chirp_coeffs(5, 0, 100, 2)


def test_exponential_chirp_parameters(awglib):
    """The exponential profile's words: F_start, F_end and the doubles alpha = ln(F_end/F_start)/L,
    C = F_start/alpha and e^alpha - 1 (bit patterns); equal ends give the linear profile's words."""
    import math
    import struct
    M = 1 << 64
    for F0, F1, L in ((1 << 62, 3 << 61, 100_000), (M - 1, 12345678901234, 7), (1 << 40, (1 << 40) + 1, (1 << 28) - 1)):
        w = awglib.chirp_coeffs(F0, F1, L, 2)
        limbs = [(w[k] >> (64 * j)) & (M - 1) for k in range(7) for j in range(3)]
        assert limbs[0] == F0 and limbs[1] == F1 and not any(limbs[5:])
        alpha, C, q = (struct.unpack("<d", struct.pack("<Q", v))[0] for v in limbs[2:5])
        lam = math.log(F1 / F0) if abs(F1 / F0 - 1) > 1e-3 else math.log1p((F1 - F0) / F0)
        assert abs(alpha * L / lam - 1) < 1e-13
        assert abs(C * alpha / F0 - 1) < 1e-15
        assert abs(q / math.expm1(alpha) - 1) < 1e-15
    assert awglib.chirp_coeffs(777, 777, 500, 2) == awglib.chirp_coeffs(777, 777, 500, 0)


def test_bad_arguments_rejected_without_gpu(awglib):
    L = awglib.lib()
    assert L.awg_create(float("nan")) is None
    assert L.awg_create(-1.0) is None
    for f in (-1.0, float("inf"), float("nan"), 280e6):
        with pytest.raises(awglib.AwgError):
            awglib.freq_word(f, 280e6)
    with pytest.raises(awglib.AwgError):
        awglib.phase_word(float("nan"))
    with pytest.raises(awglib.AwgError):
        awglib.grid_word(1e6, 280e6, 0)


def test_null_handles_rejected_without_gpu(awglib):
    """Entry points given no handle fail with AWG_EINVAL (or -1 for counters) instead of touching
    the device."""
    L = awglib.lib()
    assert L.awg_render_stream(None, 100, 10, None, None) == awglib.AWG_EINVAL
    assert L.awg_render_chunks(None, 10, 2, None, None) == awglib.AWG_EINVAL
    assert L.awg_render(None, 100, None, None) == awglib.AWG_EINVAL
    assert L.awg_launch_count(None) == -1
    assert L.awg_set_static_engine(None, 1) == awglib.AWG_EINVAL
