"""GB300 (sm_103a) multi-tone additive synthesis: Python binding of the C ABI in include/awg.h.

The binding marshals arguments only; every step of the synthesis runs in the CUDA library
(libawg.so, built in-tree by ``paper_2403_15582_gb300.build``).  There is no CPU fallback: if the
library is missing, importing the binding's entry points raises.
"""
from __future__ import annotations

from .binding import (AWG_EDEADLINE, AWG_EINVAL, AWG_ENOMEM, AWG_ECUDA, AWG_ESTATE, AWG_ETIMEOUT, AWG_OK,
                      PERIODIC_DIRECT, PERIODIC_GEMM_BF16, PERIODIC_GEMM_FP16, PREC_BF16, PREC_FP16, PROFILE_EXPONENTIAL, PROFILE_LINEAR, PROFILE_MINJERK, SINE_ROTATOR, SINE_SFU, STATIC_DIRECT, STATIC_GEMM_BF16, STATIC_GEMM_FP16, AwgError, Ring, Server,
                      Synth, chirp_coeffs, chirp_length, freq_word, grid_word, lib, phase_word, render_multiplexed,
                      sfu_rate_probe, chirp_rate_probe, chirp_render_flags,
                      CHIRP_TABLE, CHIRP_LINEAR, CHIRP_EXP, CHIRP_FLAT3, CHIRP_LOW6, CHIRP_PAIR, CHIRP_LOW3)

__all__ = ["Synth", "Ring", "Server", "AwgError", "lib", "freq_word", "phase_word", "grid_word", "chirp_length", "chirp_coeffs",
           "PROFILE_LINEAR", "PROFILE_MINJERK", "PROFILE_EXPONENTIAL", "AWG_OK", "AWG_EINVAL", "AWG_ENOMEM", "AWG_ECUDA", "AWG_ETIMEOUT",
           "AWG_EDEADLINE", "AWG_ESTATE", "PREC_BF16", "PREC_FP16", "SINE_SFU", "SINE_ROTATOR", "render_multiplexed",
           "PERIODIC_DIRECT", "PERIODIC_GEMM_BF16", "PERIODIC_GEMM_FP16",
           "STATIC_DIRECT", "STATIC_GEMM_FP16", "STATIC_GEMM_BF16", "sfu_rate_probe", "chirp_rate_probe", "chirp_render_flags",
           "CHIRP_TABLE", "CHIRP_LINEAR", "CHIRP_EXP", "CHIRP_FLAT3", "CHIRP_LOW6", "CHIRP_PAIR", "CHIRP_LOW3"]
