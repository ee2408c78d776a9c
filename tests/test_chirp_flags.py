"""Host logic: the flags the render gives a chirp (awg_chirp_render_flags), which decide its run
set-up.  Checked against what the bounds state (the third unit difference of a minimum-jerk chirp
is at most 5.77 |D| / L^2 words by the mean value theorem, taken as 6 |D| / L^2; a lane pair may
share the set-up of a linear chirp always and of a LOW6 chirp while C(63, 3) times that bound stays
below 512 units of 2^-32 turn), and for the orderings the set-up relies on: LOW3 implies LOW6
implies FLAT3, LOW6 implies a shared set-up, a tabled chirp never shares one, and a longer chirp
of the same frequency change never loses a flag it had."""
import numpy as np
import pytest

FS = 280e6
UNIT = 2.0**32          # words per unit of 2^-32 turn


def flags(awg, f0, f1, L, profile):
    return awg.chirp_render_flags(awg.freq_word(f0, FS), awg.freq_word(f1, FS), L, profile)


def test_linear_chirps_share_their_set_up(awglib):
    awg = awglib
    rng = np.random.default_rng(3)
    for _ in range(100):
        f0, f1 = rng.uniform(1e6, 139e6, 2)
        L = int(rng.integers(100, 20_000_000))
        fl = flags(awg, f0, f1, L, awg.PROFILE_LINEAR)
        assert fl & awg.CHIRP_LINEAR and fl & awg.CHIRP_PAIR, (f0, f1, L, fl)
        assert not fl & (awg.CHIRP_FLAT3 | awg.CHIRP_LOW6 | awg.CHIRP_LOW3 | awg.CHIRP_TABLE | awg.CHIRP_EXP)


def test_the_benchmark_chirps_take_the_shortest_set_up(awglib):
    """1000 tones chirped 35 ms at 280 MS/s between 80 and 180 MHz: every minimum-jerk chirp takes
    the LOW3 set-up, shared in lane pairs."""
    from paper_2403_15582_gb300 import workloads as wl
    awg = awglib
    wk = wl.chirp_1000(seed=0)
    for c in wk.chirps:
        fl = flags(awg, c["f_start"], c["f_end"], wk.n_samples, c["profile"])
        if c["profile"] == awg.PROFILE_MINJERK:
            want = awg.CHIRP_FLAT3 | awg.CHIRP_LOW6 | awg.CHIRP_LOW3 | awg.CHIRP_PAIR
            assert fl == want, (c, fl)


@pytest.mark.parametrize("profile", [1, 2])
def test_orderings_and_monotone_in_length(awglib, profile):
    awg = awglib
    rng = np.random.default_rng(7 + profile)
    lengths = np.unique(np.round(np.geomspace(2, 5e7, 80)).astype(np.int64))
    kept = (awg.CHIRP_FLAT3, awg.CHIRP_LOW6, awg.CHIRP_LOW3, awg.CHIRP_PAIR)
    for _ in range(12):
        f0, f1 = rng.uniform(1e6, 139e6, 2)
        prev = None
        for L in lengths:
            fl = flags(awg, f0, f1, int(L), profile)
            if fl & awg.CHIRP_LOW3:
                assert fl & awg.CHIRP_LOW6
            if fl & awg.CHIRP_LOW6:
                assert fl & awg.CHIRP_FLAT3 and fl & awg.CHIRP_PAIR
            if fl & awg.CHIRP_TABLE:
                assert not fl & awg.CHIRP_PAIR
            assert bool(fl & awg.CHIRP_EXP) == (profile == awg.PROFILE_EXPONENTIAL)
            if prev is not None:
                for bit in kept:
                    assert not (prev & bit) or (fl & bit), (f0, f1, int(L), prev, fl)
                assert not (fl & awg.CHIRP_TABLE) or (prev & awg.CHIRP_TABLE)
            prev = fl


def test_thresholds_of_the_minimum_jerk_bounds(awglib):
    """FLAT3 where 6 |D| / L^2 < 2^30 words, checked 3 % on either side of the threshold length; a
    minimum-jerk chirp shares its run set-up only in LOW6 form, whose bound (the fourth to sixth
    derivatives over a run) needs longer chirps than the pair bound C(63, 3) 6 |D| / L^2 < 512
    units does."""
    awg = awglib
    F0, F1 = awg.freq_word(60e6, FS), awg.freq_word(140e6, FS)
    D = float(F1 - F0)
    L_flat3 = (6.0 * D / 2.0**30) ** 0.5
    assert flags(awg, 60e6, 140e6, int(L_flat3 * 1.03), 1) & awg.CHIRP_FLAT3
    assert not flags(awg, 60e6, 140e6, int(L_flat3 * 0.97), 1) & awg.CHIRP_FLAT3
    L_pair = (39711.0 * 6.0 * D / (512.0 * UNIT)) ** 0.5
    assert not flags(awg, 60e6, 140e6, int(L_pair * 0.97), 1) & (awg.CHIRP_PAIR | awg.CHIRP_LOW6)
    L_low6 = next(L for L in np.geomspace(L_pair, 100 * L_pair, 400).astype(np.int64)
                  if flags(awg, 60e6, 140e6, int(L), 1) & awg.CHIRP_LOW6)
    assert L_low6 > L_pair and flags(awg, 60e6, 140e6, int(L_low6), 1) & awg.CHIRP_PAIR


def test_validation(awglib):
    awg = awglib
    F = awg.freq_word(100e6, FS)
    assert flags(awg, 100e6, 100e6, 1000, awg.PROFILE_EXPONENTIAL) & awg.CHIRP_LINEAR   # same phase
    for args in ((F, F, 0, 1), (F, F, 100, 7), (0, F, 100, awg.PROFILE_EXPONENTIAL)):
        with pytest.raises(awg.AwgError):
            awg.chirp_render_flags(*args)
