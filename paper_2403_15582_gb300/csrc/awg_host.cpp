// Host side of the C ABI (include/awg.h): tone and chirp set-up in exact integer arithmetic,
// device-resident state, and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/awg.h"
#include "awg_internal.h"

using awgk::ChirpRec;
using awgk::TileRec;
using awgk::ToneRec;

// The public limits of awg_render_noalloc are the sizes of its fixed scratch.
static_assert(awgk::NOALLOC_MAX_RECORDS == AWG_NOALLOC_MAX_RECORDS, "awg.h: AWG_NOALLOC_MAX_RECORDS");
static_assert(awgk::NOALLOC_MAX_SLOTS == AWG_NOALLOC_MAX_SLOTS, "awg.h: AWG_NOALLOC_MAX_SLOTS");
static_assert(AWG_CHIRP_TABLE == awgk::TONE_EXACT && AWG_CHIRP_LINEAR == awgk::TONE_LINEAR && AWG_CHIRP_EXP == awgk::TONE_EXP &&
                  AWG_CHIRP_FLAT3 == awgk::TONE_FLAT3 && AWG_CHIRP_LOW6 == awgk::TONE_LOW6 &&
                  AWG_CHIRP_PAIR == awgk::TONE_PAIR && AWG_CHIRP_LOW3 == awgk::TONE_LOW3,
              "awg.h: AWG_CHIRP_* flags");

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

namespace awgk {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace awgk

namespace {
int cuda_fail(cudaError_t e, const char* what) {
  return fail(AWG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

typedef unsigned __int128 u128;
typedef __int128 s128;

// ------------------------------------------------------------------------------------------
// 192-bit words (mod 2^192) and a small unsigned bigint for exact set-up
// ------------------------------------------------------------------------------------------
struct W192 {
  uint64_t w[3];
};

W192 w_add(W192 a, W192 b) {
  W192 r;
  u128 c = 0;
  for (int i = 0; i < 3; ++i) {
    c += (u128)a.w[i] + b.w[i];
    r.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}
W192 w_neg(W192 a) {
  W192 r;
  u128 c = 1;
  for (int i = 0; i < 3; ++i) {
    c += (u128)(~a.w[i]);
    r.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}
W192 w_mul(W192 a, W192 b) {
  W192 r = {{0, 0, 0}};
  for (int i = 0; i < 3; ++i) {
    u128 c = 0;
    for (int j = 0; i + j < 3; ++j) {
      c += (u128)a.w[i] * b.w[j] + r.w[i + j];
      r.w[i + j] = (uint64_t)c;
      c >>= 64;
    }
  }
  return r;
}
W192 w_from_u64(uint64_t v) { return W192{{v, 0, 0}}; }

// Unsigned little-endian multi-limb integer (up to 8 limbs).
struct Big {
  uint64_t l[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};
Big big_from_u128(u128 v) {
  Big b;
  b.l[0] = (uint64_t)v;
  b.l[1] = (uint64_t)(v >> 64);
  return b;
}
Big big_mul_u128(const Big& a, u128 m) {   // a * m, m < 2^128
  Big r;
  uint64_t m0 = (uint64_t)m, m1 = (uint64_t)(m >> 64);
  for (int part = 0; part < 2; ++part) {
    uint64_t mm = part ? m1 : m0;
    if (!mm) continue;
    u128 c = 0;
    for (int i = 0; i + part < 8; ++i) {
      c += (u128)a.l[i] * mm + r.l[i + part];
      r.l[i + part] = (uint64_t)c;
      c >>= 64;
    }
  }
  return r;
}
Big big_shl(const Big& a, int s) {   // s < 512
  Big r;
  int q = s / 64, b = s % 64;
  for (int i = 7; i >= 0; --i) {
    uint64_t v = 0;
    if (i - q >= 0) v = a.l[i - q] << b;
    if (b && i - q - 1 >= 0) v |= a.l[i - q - 1] >> (64 - b);
    r.l[i] = v;
  }
  return r;
}
// Division of n < 2^64 by an invariant divisor d < 2^32 through its reciprocal inv = floor((2^64 -
// 1) / d): the estimate floor(n inv / 2^64) is below n / d by less than n / 2^64 + 1 < 2, so at
// most two corrections give the exact quotient and remainder.
struct Div32 {
  uint64_t d, inv;
  explicit Div32(uint64_t dd) : d(dd), inv(~0ull / dd) {}
  uint64_t divmod(uint64_t n, uint64_t* r) const {
    uint64_t q = (uint64_t)(((u128)n * inv) >> 64);
    uint64_t rem = n - q * d;
    while (rem >= d) {
      rem -= d;
      ++q;
    }
    *r = rem;
    return q;
  }
};

uint64_t big_divmod_u64(Big& a, uint64_t d) {   // a /= d, returns remainder
  int top = 7;
  while (top > 0 && a.l[top] == 0) --top;         // leading zero limbs stay zero
  if (d < (1ull << 32)) {
    // 32-bit halves: every partial dividend is below 2^64, divided through the reciprocal of d
    const Div32 dv(d);
    uint64_t rem = 0;
    for (int i = top; i >= 0; --i) {
      const uint64_t qh = dv.divmod((rem << 32) | (a.l[i] >> 32), &rem);
      const uint64_t ql = dv.divmod((rem << 32) | (a.l[i] & 0xFFFFFFFFull), &rem);
      a.l[i] = (qh << 32) | ql;
    }
    return rem;
  }
  u128 rem = 0;
  for (int i = top; i >= 0; --i) {
    u128 cur = (rem << 64) | a.l[i];
    a.l[i] = (uint64_t)(cur / d);
    rem = cur % d;
  }
  return (uint64_t)rem;
}
Big big_add(const Big& a, const Big& b) {
  Big r;
  u128 c = 0;
  for (int i = 0; i < 8; ++i) {
    c += (u128)a.l[i] + b.l[i];
    r.l[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}

// Delta^k [m^p] at m = 0 = sum_j (-1)^(k-j) C(k,j) j^p  (k! S(p,k), Stirling numbers of the 2nd kind)
s128 power_difference_sum(int p, int k) {
  s128 s = 0;
  s128 binom = 1;   // C(k, j)
  for (int j = 0; j <= k; ++j) {
    if (j > 0) binom = binom * (k - j + 1) / j;
    s128 pw = 1;
    for (int e = 0; e < p; ++e) pw *= j;
    s += (((k - j) & 1) ? -1 : 1) * binom * pw;
  }
  return s;
}

// The same values, tabulated once (p, k <= 6): they are constants of every chirp's set-up.
s128 power_difference(int p, int k) {
  static const struct Table {
    s128 v[7][7];
    Table() {
      for (int pp = 0; pp <= 6; ++pp)
        for (int kk = 0; kk <= 6; ++kk) v[pp][kk] = power_difference_sum(pp, kk);
    }
  } table;
  return table.v[p][k];
}

Big big_shr1(const Big& a) {
  Big r;
  for (int i = 0; i < 8; ++i) r.l[i] = (a.l[i] >> 1) | (i < 7 ? a.l[i + 1] << 63 : 0);
  return r;
}

// round_half_even( sign * mag * 2^127 / L^pw ), returned mod 2^192.  Successive divisions by L
// give q2 = floor(mag 2^128 / L^pw) (floor(floor(x / a) / b) = floor(x / (a b))); the quotient
// rounds up when q2 is odd (fraction >= 1/2), except on an exact tie (every remainder 0) with
// floor(q2 / 2) even.
W192 rounded_quotient(bool negative, const Big& mag, uint64_t L, int pw) {
  Big q2 = big_shl(mag, 128);
  bool exact = true;
  for (int i = 0; i < pw; ++i) exact &= big_divmod_u64(q2, L) == 0;
  Big q = big_shr1(q2);
  if ((q2.l[0] & 1) && (!exact || (q.l[0] & 1))) q = big_add(q, big_from_u128(1));
  W192 r = {{q.l[0], q.l[1], q.l[2]}};
  return negative ? w_neg(r) : r;
}

// C(m, k), k = 0..6, for 0 <= m < 2^28 as exact 192-bit values: C(m, k) = C(m, k-1) (m - k + 1) / k,
// every product below 6 C(m, 6) < 2^168 and every quotient exact.
void binomials_w(int64_t m, W192 c[7]) {
  c[0] = w_from_u64(1);
  for (int k = 1; k <= 6; ++k) {
    if (m < k) {
      c[k] = w_from_u64(0);
      continue;
    }
    const W192 p = w_mul(c[k - 1], w_from_u64((uint64_t)(m - k + 1)));
    const Div32 dv((uint64_t)k);   // 32-bit halves, as in big_divmod_u64
    uint64_t rem = 0;
    for (int i = 2; i >= 0; --i) {
      const uint64_t qh = dv.divmod((rem << 32) | (p.w[i] >> 32), &rem);
      const uint64_t ql = dv.divmod((rem << 32) | (p.w[i] & 0xFFFFFFFFull), &rem);
      c[k].w[i] = (qh << 32) | ql;
    }
  }
}

W192 w_inverse_odd(uint64_t o) {   // o^-1 mod 2^192 by Newton's iteration
  W192 x = w_from_u64(o);           // correct to 3 bits for odd o
  W192 two = w_from_u64(2);
  for (int it = 0; it < 8; ++it) x = w_mul(x, w_add(two, w_neg(w_mul(w_from_u64(o), x))));
  return x;
}

// ------------------------------------------------------------------------------------------
// set-up rules (a1, a2)
// ------------------------------------------------------------------------------------------
bool is_fin(double v) { return std::isfinite(v); }

int freq_word_impl(double f, double fs, uint64_t* out) {
  if (!(is_fin(fs) && fs > 0)) return fail(AWG_EINVAL, "sample rate must be finite and > 0");
  if (!is_fin(f) || f < 0 || f >= fs) return fail(AWG_EINVAL, "tone frequency must lie in [0, fs)");
  double r = std::ldexp(f / fs, 64);
  double w = std::rint(r);
  *out = (w >= 18446744073709551616.0) ? 0 : (uint64_t)w;
  return AWG_OK;
}

int phase_word_impl(double theta, uint64_t* out) {
  if (!is_fin(theta)) return fail(AWG_EINVAL, "phase must be finite");
  double t = theta / (2.0 * M_PI);
  double frac = t - std::floor(t);
  double w = std::rint(std::ldexp(frac, 64));
  *out = (w >= 18446744073709551616.0) ? 0 : (uint64_t)w;
  return AWG_OK;
}

int chirp_length_impl(double dur, double fs, int64_t* L) {
  if (!(is_fin(fs) && fs > 0)) return fail(AWG_EINVAL, "sample rate must be finite and > 0");
  if (!is_fin(dur) || dur <= 0) return fail(AWG_EINVAL, "chirp duration must be finite and > 0");
  double l = std::rint(dur * fs);
  if (!(l >= 1 && l <= (double)((1 << 28) - 1))) return fail(AWG_EINVAL, "chirp length must be 1 .. 2^28-1 samples");
  *L = (int64_t)l;
  return AWG_OK;
}

// d_k, k = 0..6 (see awg.h).  With D = F_end - F_start:
//   min-jerk  P(m) = F_start m + D (5 L^2 m^4 - 6 L m^5 + 2 m^6) / (2 L^5)
//   linear    P(m) = F_start m + D m^2 / (2 L)
// Delta^k P(0) = F_start [k = 1] + D N_k / (2 L^pw) with N_k built from Delta^k[m^p](0).
uint64_t bits_of(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
}

// x rounded to the nearest word, mod 2^64: the double's exact value M 2^sh (M its 53-bit integer
// mantissa) reduced by shifting.
uint64_t word_of_double(double x) {
  int e;
  const double fr = std::frexp(std::fabs(x), &e);   // |x| = fr 2^e, fr in [1/2, 1)
  if (fr == 0 || !std::isfinite(x)) return 0;
  const uint64_t M = (uint64_t)std::ldexp(fr, 53);
  const int sh = e - 53;
  uint64_t v = 0;
  if (sh >= 64) v = 0;
  else if (sh >= 0) v = M << sh;
  else if (sh > -54) v = (M + (1ull << (-sh - 1))) >> (-sh);
  return x < 0 ? (uint64_t)0 - v : v;
}

// Exponential chirp from F0 to F1 (both > 0, F0 != F1) over L samples: the frequency
// F0 e^(alpha t) with alpha = ln(F1/F0) / L, phase offset R(m) = C (e^(alpha m) - 1), C = F0 / alpha.
struct ExpParams {
  double alpha, C, q;   // q = e^alpha - 1
};
ExpParams exp_params(uint64_t F0, uint64_t F1, int64_t L) {
  const double diff = F1 >= F0 ? (double)(F1 - F0) : -(double)(F0 - F1);   // exact difference, rounded once
  ExpParams p;
  p.alpha = std::log1p(diff / (double)F0) / (double)L;
  p.C = (double)F0 / p.alpha;
  p.q = std::expm1(p.alpha);
  return p;
}

int chirp_coeffs_impl(uint64_t F0, uint64_t F1, int64_t L, int profile, W192 d[7]) {
  if (L < 1 || L > (1 << 28) - 1) return fail(AWG_EINVAL, "chirp length must be 1 .. 2^28-1 samples");
  if (profile == AWG_PROFILE_EXPONENTIAL) {
    if (F0 == 0 || F1 == 0) return fail(AWG_EINVAL, "an exponential chirp needs f_start, f_end > 0");
    if (F0 == F1) return chirp_coeffs_impl(F0, F1, L, AWG_PROFILE_LINEAR, d);   // the same phase
    const ExpParams e = exp_params(F0, F1, L);
    for (int k = 0; k < 7; ++k) d[k] = W192{{0, 0, 0}};
    d[0] = W192{{F0, F1, bits_of(e.alpha)}};
    d[1] = W192{{bits_of(e.C), bits_of(e.q), 0}};
    return AWG_OK;
  }
  if (profile != AWG_PROFILE_LINEAR && profile != AWG_PROFILE_MINJERK) return fail(AWG_EINVAL, "unknown chirp profile");
  const s128 D = (s128)F1 - (s128)F0;
  d[0] = W192{{0, 1ull << 63, 0}};   // 2^127: rounding offset of the top 64 bits
  for (int k = 1; k <= 6; ++k) {
    s128 N;
    int pw;
    if (profile == AWG_PROFILE_MINJERK) {
      N = 5 * (s128)L * L * power_difference(4, k) - 6 * (s128)L * power_difference(5, k) + 2 * power_difference(6, k);
      pw = 5;
    } else {
      N = power_difference(2, k);
      pw = 1;
    }
    W192 v = {{0, 0, 0}};
    if (N != 0 && D != 0) {
      bool neg = (N < 0) != (D < 0);
      u128 aD = (u128)(D < 0 ? -D : D);
      u128 aN = (u128)(N < 0 ? -N : N);
      Big mag = big_mul_u128(big_from_u128(aD), aN);
      v = rounded_quotient(neg, mag, (uint64_t)L, pw);
    }
    if (k == 1) v = w_add(v, W192{{0, 0, F0}});   // F_start * 2^128
    d[k] = v;
  }
  return AWG_OK;
}

// top64 of sum_k d_k C(m, k): the chirp phase in words at offset m (d_0 holds the rounding offset)
uint64_t chirp_offset_word(const W192 d[7], int64_t m) {
  W192 c[7];
  binomials_w(m, c);
  W192 s = {{0, 0, 0}};
  for (int k = 0; k < 7; ++k)
    if (d[k].w[0] | d[k].w[1] | d[k].w[2]) s = w_add(s, w_mul(d[k], c[k]));
  return s.w[2];
}

// Chirps whose neglected 4th..6th-order phase terms over one 32-sample run could exceed 512 units
// of 2^-32 turn (1.2e-7 turn) are rendered from a per-sample table of exact phases instead.
// Bound on |Delta^3 P| (words) over the whole chirp, or -1 for profiles without one (linear chirps
// have Delta^3 P = 0 exactly and take their own path).  Minimum-jerk: by the mean value theorem
// |Delta^3 P| <= max |P'''| = 5.77 |D| / L^2 (60 max |t - 3 t^2 + 2 t^3| = 5.77 over t in [0, 1]),
// taken as 6 |D| / L^2.  Exponential: exactly Delta^3 R(m) = C e^(alpha m) q^3 with C = F_start /
// alpha and q = e^alpha - 1, i.e. F(m) q^3 / alpha, at most F_max |q|^3 / |alpha| (1 + |q|)^3 over
// the differences that reach past the end.
double third_difference_bound(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  const double l = (double)L;
  if (profile == AWG_PROFILE_MINJERK) return 6.0 * std::fabs((double)F1 - (double)F0) / (l * l);
  if (profile == AWG_PROFILE_EXPONENTIAL && F0 != F1) {
    const ExpParams e = exp_params(F0, F1, L);
    const double q = std::fabs(e.q), a = std::fabs(e.alpha);
    return (double)std::max(F0, F1) * q * q * q / a * (1.0 + q) * (1.0 + q) * (1.0 + q) * 1.01;
  }
  return -1.0;
}

// Whether the third unit difference of the chirp phase stays below 2^30 words over the whole
// chirp, so that the render's run cascade rounds h to 0 in every run (TONE_FLAT3).

bool flat_third_difference(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  const double bound = third_difference_bound(F0, F1, L, profile);
  return bound >= 0 && bound < 1073741824.0;   // 2^30
}

// Whether a TONE_FLAT3 chirp may also drop the stride-32 differences B_6, E_5 and G_2..G_4 of its
// run set-up (TONE_LOW6): each is bounded through the mean value theorem by 32^q max |P^(k)| (B_q:
// k = q, E_q: k = q + 1, G_q: k = q + 2), with max |P^(k)| = 60, 360, 720 |D| / L^(k-1) for
// k = 4, 5, 6 on the minimum-jerk profile and F_max |alpha|^(k-1) on the exponential one.  Their
// largest effect on a run's phase, through C(127, q) and the 31 / 465 steps the run takes f and g
// through, must stay below 64 units of 2^-32 turn (the cascade's own bound is 2500).
bool low_order_negligible(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  const double l = (double)L;
  double d4, d5, d6;
  if (profile == AWG_PROFILE_MINJERK) {
    const double D = std::fabs((double)F1 - (double)F0);
    d4 = 60.0 * D / (l * l * l);
    d5 = 360.0 * D / (l * l * l * l);
    d6 = 720.0 * D / (l * l * l * l * l);
  } else if (profile == AWG_PROFILE_EXPONENTIAL && F0 != F1) {
    const double a = std::fabs(exp_params(F0, F1, L).alpha) * 1.01;
    const double Fm = (double)std::max(F0, F1) * 1.01;
    d4 = Fm * a * a * a;
    d5 = d4 * a;
    d6 = d5 * a;
  } else {
    return false;
  }
  const double s32 = 32.0, c2 = 8001.0, c3 = 333375.0, c4 = 10334625.0, c5 = 254231775.0, c6 = 5169379425.0;
  const double B6 = std::pow(s32, 6) * d6, E5 = std::pow(s32, 5) * d6;
  const double G2 = s32 * s32 * d4, G3 = std::pow(s32, 3) * d5, G4 = std::pow(s32, 4) * d6;
  const double words = B6 * c6 + 31.0 * E5 * c5 + 465.0 * (G2 * c2 + G3 * c3 + G4 * c4);
  return words < 64.0 * 4294967296.0;
}

// Whether a TONE_LOW6 chirp may also drop B_5, E_3 and E_4 of its run set-up (TONE_LOW3): every
// left-out stride difference, bounded as in low_order_negligible (B_q: 32^q max |P^(q)|, E_q: with
// P^(q+1), G_q: with P^(q+2)), weighted by C(127, q) and by the 63 / 1953 steps a cascade that
// spans two runs (a lane pair's moved state) takes f and g through, must stay below 256 units of
// 2^-32 turn: with the rounding (1008.5) and the third differences (512) of such a cascade, below
// the 2500 of an unshared minimum-jerk run.
bool low3_negligible(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  const double l = (double)L;
  double d4, d5, d6;
  if (profile == AWG_PROFILE_MINJERK) {
    const double D = std::fabs((double)F1 - (double)F0);
    d4 = 60.0 * D / (l * l * l);
    d5 = 360.0 * D / (l * l * l * l);
    d6 = 720.0 * D / (l * l * l * l * l);
  } else if (profile == AWG_PROFILE_EXPONENTIAL && F0 != F1) {
    const double a = std::fabs(exp_params(F0, F1, L).alpha) * 1.01;
    const double Fm = (double)std::max(F0, F1) * 1.01;
    d4 = Fm * a * a * a;
    d5 = d4 * a;
    d6 = d5 * a;
  } else {
    return false;
  }
  const double c2 = 8001.0, c3 = 333375.0, c4 = 10334625.0, c5 = 254231775.0, c6 = 5169379425.0;
  const double p2 = 1024.0, p3 = 32768.0, p4 = 1048576.0, p5 = 33554432.0, p6 = 1073741824.0;   // 32^q
  const double B = p5 * d5 * c5 + p6 * d6 * c6;
  const double E = p3 * d4 * c3 + p4 * d5 * c4 + p5 * d6 * c5;
  const double G = p2 * d4 * c2 + p3 * d5 * c3 + p4 * d6 * c4;
  return B + 63.0 * E + 1953.0 * G < 256.0 * 4294967296.0;
}

// Whether two lanes may share the chirp's run set-up (TONE_PAIR): the render then takes a run's
// cascade state from the neighbouring run's exact set-up, moved by 32 samples with the cascade's
// integer steps, so a cascade spans up to 63 steps instead of 31.  Linear chirps: the third
// difference is exactly zero, the bound is the rounding of p, f, g over 63 steps (0.5 + 31.5 +
// 976.5 units of 2^-32 turn).  LOW6 chirps: in addition the neglected third differences over 63
// steps, C(63, 3) max |Delta^3 P|, must stay below 512 units, and LOW6's left-out stride terms
// grow from 64 to at most 64 x 1953 / 465 = 269 units: at most 1790 units against the 2500 of an
// unshared minimum-jerk run.
bool pair_setup_ok(uint64_t F0, uint64_t F1, int64_t L, int profile, bool low6) {
  if (profile == AWG_PROFILE_LINEAR) return true;
  if (!low6) return false;
  const double bound = third_difference_bound(F0, F1, L, profile);
  return bound >= 0 && 39711.0 * bound < 512.0 * 4294967296.0;
}

bool needs_exact(uint64_t F0, uint64_t F1, int64_t L, int profile);

// The render's flags of a chirp (ChirpRec::flags; the low bits of ToneRec::flags): its profile
// (TONE_LINEAR, TONE_EXP), a per-sample table (TONE_EXACT), and the run set-up it takes (TONE_FLAT3,
// TONE_LOW6, TONE_LOW3, TONE_PAIR), from the bounds above.
int32_t chirp_render_flags(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  const bool exact = needs_exact(F0, F1, L, profile);
  const bool flat3 = flat_third_difference(F0, F1, L, profile);
  const bool low6 = flat3 && low_order_negligible(F0, F1, L, profile);
  const bool pair = !exact && pair_setup_ok(F0, F1, L, profile, low6);
  const bool low3 = low6 && low3_negligible(F0, F1, L, profile);
  return (exact ? awgk::TONE_EXACT : 0) | (profile == AWG_PROFILE_LINEAR ? awgk::TONE_LINEAR : 0) |
         (profile == AWG_PROFILE_EXPONENTIAL ? awgk::TONE_EXP : 0) | (flat3 ? awgk::TONE_FLAT3 : 0) |
         (low6 ? awgk::TONE_LOW6 : 0) | (low3 ? awgk::TONE_LOW3 : 0) | (pair ? awgk::TONE_PAIR : 0);
}

// Phase offset at the end of an exponential chirp, R(L), the same FP64 formula as the render's.
uint64_t exp_end_offset(uint64_t F0, uint64_t F1, int64_t L) {
  const ExpParams e = exp_params(F0, F1, L);
  return word_of_double(e.C * std::expm1(e.alpha * (double)L));
}

// Whether a chirp takes the per-sample table: the render's 32-bit run cascade drops the phase
// differences of order 4..6 inside a run of 32 samples; above 2^-23 turn the table is used.
// Exponential chirps: the tile polynomial also drops orders >= 7 over a tile of 4096 samples,
// C(4095, 7) |Delta^7 R| <= 3.8e21 F_max |q|^6 (twice that for the tail of the series), with a
// budget of 2^-26 turn.
bool needs_exact(uint64_t F0, uint64_t F1, int64_t L, int profile) {
  if (profile == AWG_PROFILE_EXPONENTIAL && F0 != F1) {
    const double q = std::fabs(exp_params(F0, F1, L).q);
    const double Fm = (double)std::max(F0, F1) * (1.0 + q);
    const double tile = 2.0 * 3.8e21 * Fm * q * q * q * q * q * q;
    const double run = 31465.0 * Fm * q * q * q + 169911.0 * Fm * q * q * q * q + 736281.0 * Fm * q * q * q * q * q;
    return tile > 274877906944.0 /* 2^38 */ || run > 512.0 * 4294967296.0 || 4096.0 * q > 1.0;
  }
  if (profile == AWG_PROFILE_LINEAR || profile == AWG_PROFILE_EXPONENTIAL) return false;
  double D = std::fabs((double)F1 - (double)F0);
  double l = (double)L;
  double bound = 31465.0 * 60.0 * D / (l * l * l) + 169911.0 * 360.0 * D / (l * l * l * l) +
                 736281.0 * 720.0 * D / (l * l * l * l * l);
  return bound > 512.0 * 4294967296.0;
}

}  // namespace

// cos and sin of the per-sample phase step 2 pi F / 2^64, rounded to float (rotator variant).
void rotation_of(uint64_t F, float* c, float* s) {
  const double turn = (double)(F >> 11) * 0x1p-53;
  const double ang = 6.283185307179586476925 * turn;
  *c = (float)std::cos(ang);
  *s = (float)std::sin(ang);
}

// Tone split per tile: about 96 tones per CTA, at most MAX_SPLIT CTAs per cluster.  A function of
// the tone count only, so that every sample is summed in the same order whatever the window.
int awgk::tone_split_for(int K) {
  int s = (K + 95) / 96;
  return std::max(1, std::min(s, awgk::MAX_SPLIT));
}

// ==========================================================================================
// handle
// ==========================================================================================
struct awg {
  double fs = 0;
  int device = 0;
  int32_t K = 0;
  std::vector<ToneRec> tones;
  std::vector<double> amp;
  std::vector<ChirpRec> chirps;       // slot pool (tone < 0: free)
  std::vector<int32_t> free_slots;
  ToneRec* d_tones = nullptr;
  size_t cap_tones = 0;
  ChirpRec* d_chirps = nullptr;
  int32_t* d_act = nullptr;
  size_t cap_chirps = 0;
  TileRec* d_recs = nullptr;          // chirp tile records of the current render window
  size_t cap_recs = 0;
  // pipelined chunk sequences (awg_render_chunks): the tile records of a group of chunks, and a
  // device counter of the render CTAs that have stored their samples
  TileRec* d_seq_recs = nullptr;
  size_t cap_seq_recs = 0;
  int32_t* d_seq_act = nullptr;
  size_t cap_seq_act = 0;
  unsigned long long* d_seq_exit = nullptr;
  unsigned long long seq_exit_target = 0;
  int32_t* d_status = nullptr;
  uint64_t* d_words = nullptr;
  size_t cap_words = 0;
  uint32_t* d_trace = nullptr;
  size_t cap_trace = 0;
  uint32_t* d_tab = nullptr;           // exact per-sample phases of TONE_EXACT chirps
  size_t cap_tab = 0;
  uint16_t* d_gemm = nullptr;          // table GEMM B operand: hi, lo (A is generated in the kernel)
  size_t cap_gemm = 0;
  int64_t cursor = 0;
  double full_scale = 0;
  bool fs_explicit = false;
  int split = 1;
  int32_t sine_mode = AWG_SINE_SFU;
  int32_t static_engine = AWG_STATIC_DIRECT;
  float* d_base = nullptr;             // tensor-core engine: FP32 sum of the window's static tones
  size_t cap_base = 0;
  // split sums without clusters: two scratch buffers (alternating between consecutive launches)
  // of part_tiles x part_split partial tiles each, and a 64-bit counter per tile per buffer
  float* d_part = nullptr;
  unsigned long long* d_tctr = nullptr;
  int32_t part_tiles = 0, part_split = 0, ctr_split = 0;
  int64_t n_launches = 0;              // kernels this handle has launched
  int32_t* d_list = nullptr;           // tensor-core engine: tones not static in some tile of the window
  size_t cap_list = 0;
  std::vector<int32_t> list;
  // tones that hold a chirp or an amplitude ramp, ascending (the static engine's render part);
  // rebuilt on demand after tones, chirps or ramps change
  std::vector<int32_t> flagged;
  double amax = 0;                     // largest |amplitude| (ramp targets included), with `flagged`
  bool flagged_ok = false;
  // periodic hand-off: from sample periodic_start on, x[n] = periodic table[n mod 2^periodic_log2]
  int16_t* d_periodic = nullptr;
  size_t cap_periodic = 0;
  int32_t periodic_log2 = 0;
  int64_t periodic_start = -1;
  cudaStream_t priv = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
  // stream-ordered uploads of changed records (awg_set_chirps): pinned staging, copied on the
  // private stream after the last render issued (ev_done); later launches wait for ev_upload
  unsigned char* stage = nullptr;
  size_t cap_stage = 0;
  cudaEvent_t ev_upload = nullptr;
  bool upload_pending = false;
  bool timed = false, have_done = false;
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;   // 4 per recorded render call
  size_t prof_calls = 0;
  int64_t prof_launches = 0;
  uint32_t W[7][7];
  uint64_t inv_odd[3][3];
};

namespace {

void fill_constants(awg_t* h) {
  // W[q][i] = Delta^q_j C(j RUN, i) at j = 0
  for (int q = 0; q < 7; ++q)
    for (int i = 0; i < 7; ++i) {
      s128 s = 0, bq = 1;
      for (int l = 0; l <= q; ++l) {
        if (l > 0) bq = bq * (q - l + 1) / l;
        s128 c = 1;   // C(l RUN, i)
        int64_t m = (int64_t)l * awgk::RUN;
        if (i > m) c = 0;
        else
          for (int t = 0; t < i; ++t) c = c * (m - t) / (t + 1);
        s += (((q - l) & 1) ? -1 : 1) * bq * c;
      }
      if (s < 0 || s > (s128)UINT32_MAX) std::abort();   // RUN = 32: every entry lies in [0, 2^32)
      h->W[q][i] = (uint32_t)s;
    }
  const uint64_t odd[3] = {3, 15, 45};
  for (int i = 0; i < 3; ++i) {
    W192 x = w_inverse_odd(odd[i]);
    for (int j = 0; j < 3; ++j) h->inv_odd[i][j] = x.w[j];
  }
}

// A kernel launch of the handle, counted (awg_launch_count).
inline cudaError_t counted(awg_t* h, cudaError_t e) {
  ++h->n_launches;
  return e;
}

int wait_idle(awg_t* h) {
  if (h->have_done) {
    cudaError_t e = cudaEventSynchronize(h->ev_done);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the last render");
  }
  if (h->upload_pending) {
    cudaError_t e = cudaEventSynchronize(h->ev_upload);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the last upload");
    h->upload_pending = false;
  }
  return AWG_OK;
}

// Device work on stream s that reads the handle's tone, chirp or table records is issued after
// the copies of the last stream-ordered upload.
cudaError_t order_after_uploads(awg_t* h, cudaStream_t s) {
  if (!h->upload_pending) return cudaSuccess;
  if (cudaEventQuery(h->ev_upload) == cudaSuccess) {
    h->upload_pending = false;
    return cudaSuccess;
  }
  cudaGetLastError();   // cudaErrorNotReady is not an error here
  return cudaStreamWaitEvent(s, h->ev_upload, 0);
}

template <class T>
int ensure(T** ptr, size_t* cap, size_t need, awg_t* h, const char* what) {
  if (need <= *cap) return AWG_OK;
  int st = wait_idle(h);
  if (st) return st;
  size_t ncap = std::max(need, *cap * 2);
  T* p = nullptr;
  cudaError_t e = cudaMalloc((void**)&p, ncap * sizeof(T));
  if (e != cudaSuccess) return fail(AWG_ENOMEM, std::string("cudaMalloc ") + what);
  if (*ptr) cudaFree(*ptr);
  *ptr = p;
  *cap = ncap;
  return AWG_OK;
}

// Host worker threads for the set-up arithmetic of large chirp batches, started once per process
// (starting threads per call cost more than the work at 1000 chirps).  parallel_for(n, fn) runs
// fn(lo, hi) over [0, n) in `parts` ranges, which the calling thread and the workers claim one at
// a time (so a worker that wakes late delays nothing but the range it takes), and returns when all
// are done.  Calls are serialised.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  size_t threads() const { return workers_.size() + 1; }
  void parallel_for(size_t n, size_t parts, const std::function<void(size_t, size_t)>& fn) {
    parts = std::max<size_t>(1, std::min(parts, 8 * threads()));
    if (parts == 1 || threads() == 1) {
      fn(0, n);
      return;
    }
    std::lock_guard<std::mutex> call(call_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      n_ = n;
      parts_ = parts;
      next_ = 0;
      pending_ = parts;
      ++gen_;
    }
    cv_.notify_all();
    for (;;) {   // the calling thread claims ranges too
      size_t part;
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (next_ >= parts_) break;
        part = next_++;
      }
      fn(n * part / parts, n * (part + 1) / parts);
      std::lock_guard<std::mutex> lk(mu_);
      --pending_;
    }
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return pending_ == 0; });
    fn_ = nullptr;
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread& t : workers_) t.join();
  }

 private:
  HostPool() {
    const size_t n = std::min<size_t>(15, std::max(1u, std::thread::hardware_concurrency()) - 1);
    for (size_t i = 0; i < n; ++i) workers_.emplace_back([this] { run(); });
  }
  void run() {
    uint64_t seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] { return stop_ || (gen_ != seen && next_ < parts_); });
      if (stop_) return;
      const size_t part = next_++;
      if (next_ >= parts_) seen = gen_;
      const std::function<void(size_t, size_t)>* fn = fn_;
      const size_t n = n_, parts = parts_;
      lk.unlock();
      (*fn)(n * part / parts, n * (part + 1) / parts);
      lk.lock();
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex mu_, call_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t, size_t)>* fn_ = nullptr;
  size_t n_ = 0, parts_ = 0, next_ = 0, pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// Scratch for launches of up to `tiles` tiles with tone split `split` (> 1): two buffers of
// part_tiles x part_split partial tiles (capacities) and part_tiles tile counters each.  The
// counters count every CTA of every launch, and a CTA is the last of its tile when its count is
// split - 1 mod split; so they are zeroed when allocated and whenever the split changes.
constexpr int32_t SPLIT_LAUNCH_TILES = 512;   // tiles per render launch when the split sums in scratch
int ensure_split_scratch(awg_t* h, int32_t tiles, int32_t split) {
  if (tiles <= h->part_tiles && split <= h->part_split && split == h->ctr_split) return AWG_OK;
  int st = wait_idle(h);
  if (st) return st;
  cudaError_t e = cudaSuccess;
  if (tiles > h->part_tiles || split > h->part_split) {
    const int32_t nt = std::max(tiles, h->part_tiles), ns = std::max(split, h->part_split);
    cudaFree(h->d_part);
    cudaFree(h->d_tctr);
    h->d_part = nullptr;
    h->d_tctr = nullptr;
    h->part_tiles = h->part_split = 0;
    e = cudaMalloc((void**)&h->d_part, (size_t)2 * nt * ns * awgk::TILE * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_tctr, (size_t)2 * nt * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AWG_ENOMEM, "cudaMalloc split scratch");
    }
    h->part_tiles = nt;
    h->part_split = ns;
  }
  if ((e = cudaMemset(h->d_tctr, 0, (size_t)2 * h->part_tiles * sizeof(unsigned long long))) != cudaSuccess)
    return cuda_fail(e, "split counters");
  h->ctr_split = split;
  return AWG_OK;
}

// Scratch buffer b (0 or 1) of the split sums.
float* split_part(awg_t* h, int b) {
  return h->d_part + (size_t)b * (size_t)h->part_tiles * (size_t)h->part_split * awgk::TILE;
}
unsigned long long* split_ctr(awg_t* h, int b) { return h->d_tctr + (size_t)b * (size_t)h->part_tiles; }

int upload_tones(awg_t* h) {
  int st = ensure(&h->d_tones, &h->cap_tones, std::max<size_t>(1, h->tones.size()), h, "tones");
  if (st) return st;
  if (!h->tones.empty()) {
    cudaError_t e = cudaMemcpy(h->d_tones, h->tones.data(), h->tones.size() * sizeof(ToneRec), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload tones");
  }
  return AWG_OK;
}

int upload_chirps(awg_t* h) {
  size_t n = std::max<size_t>(1, h->chirps.size());
  if (n > h->cap_chirps) {
    int st = wait_idle(h);
    if (st) return st;
    size_t ncap = std::max(n, h->cap_chirps * 2);
    ChirpRec* p = nullptr;
    int32_t* q = nullptr;
    if (cudaMalloc((void**)&p, ncap * sizeof(ChirpRec)) != cudaSuccess) return fail(AWG_ENOMEM, "cudaMalloc chirps");
    if (cudaMalloc((void**)&q, ncap * sizeof(int32_t)) != cudaSuccess) {
      cudaFree(p);
      return fail(AWG_ENOMEM, "cudaMalloc chirp map");
    }
    if (h->d_chirps) cudaFree(h->d_chirps);
    if (h->d_act) cudaFree(h->d_act);
    h->d_chirps = p;
    h->d_act = q;
    h->cap_chirps = ncap;
  }
  if (!h->chirps.empty()) {
    cudaError_t e = cudaMemcpy(h->d_chirps, h->chirps.data(), h->chirps.size() * sizeof(ChirpRec), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload chirps");
  }
  return AWG_OK;
}

// Upload the records at the given (sorted, unique) indices, one copy per run of adjacent indices.
template <class T>
int upload_runs(T* dev, const std::vector<T>& host, const std::vector<int32_t>& idx, const char* what) {
  size_t i = 0;
  while (i < idx.size()) {
    size_t j = i + 1;
    while (j < idx.size() && idx[j] == idx[j - 1] + 1) ++j;
    const size_t first = (size_t)idx[i], count = (size_t)(idx[j - 1] - idx[i] + 1);
    cudaError_t e = cudaMemcpy(dev + first, host.data() + first, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, what);
    i = j;
  }
  return AWG_OK;
}

// Largest |amplitude| any tone takes (its ramp target included), in FP32 as the kernels hold it.
double max_amplitude_scan(const awg_t* h) {
  double m = 0;
  for (const ToneRec& t : h->tones) {
    m = std::max(m, (double)std::fabs(t.A));
    if (t.flags & awgk::TONE_AMP_RAMP) m = std::max(m, (double)std::fabs(t.A_end));
  }
  return m;
}
const std::vector<int32_t>& flagged_tones(awg_t* h);
double max_amplitude(awg_t* h) {
  (void)flagged_tones(h);   // refreshes the cached maximum with the flagged tones
  return h->amax;
}

double default_full_scale(const awg_t* h) {
  double s = 0;
  for (double a : h->amp) s += std::fabs(a);
  return s;
}

int set_tones_common(awg_t* h, const double* f, const double* amp, const double* ph, int32_t n, int32_t log2_len) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0) return fail(AWG_EINVAL, "tone count must be >= 0");
  if (n > 0 && (!f || !amp || !ph)) return fail(AWG_EINVAL, "null tone array");
  std::vector<ToneRec> tones((size_t)n);
  std::vector<double> a((size_t)n);
  for (int32_t k = 0; k < n; ++k) {
    uint64_t F, P;
    int st;
    if (log2_len > 0) {
      int64_t j;
      st = awg_grid_word(f[k], h->fs, log2_len, &F, &j);
    } else {
      st = freq_word_impl(f[k], h->fs, &F);
    }
    if (st) return st;
    if (!is_fin(amp[k])) return fail(AWG_EINVAL, "amplitude must be finite");
    st = phase_word_impl(ph[k], &P);
    if (st) return st;
    ToneRec& t = tones[(size_t)k];
    std::memset(&t, 0, sizeof(t));
    t.phi_ref = P;
    t.F = F;
    rotation_of(F, &t.rot_c, &t.rot_s);
    t.n_s = awgk::NO_CHIRP;
    t.n_e = awgk::NO_CHIRP;
    t.A = (float)amp[k];
    t.slot = -1;
    a[(size_t)k] = amp[k];
  }
  int st = wait_idle(h);
  if (st) return st;
  h->tones.swap(tones);
  h->amp.swap(a);
  h->K = n;
  h->flagged_ok = false;
  h->periodic_start = -1;
  h->chirps.clear();
  h->free_slots.clear();
  h->fs_explicit = false;
  h->full_scale = default_full_scale(h);
  h->split = awgk::tone_split_for(n);
  st = upload_tones(h);
  if (st) return st;
  return upload_chirps(h);
}

// Per-sample exact 32-bit phases for every live TONE_EXACT chirp (very short, fast chirps),
// packed one after another; the tone records get their offsets.  Chirp records must already be
// on the device.
int build_exact_tables(awg_t* h, bool sync = true) {
  size_t total = 0;
  for (const ChirpRec& c : h->chirps)
    if (c.tone >= 0 && (c.flags & awgk::TONE_EXACT)) total += (size_t)c.L + 1;
  if (total == 0) return AWG_OK;
  int st = ensure(&h->d_tab, &h->cap_tab, total, h, "exact phase tables");
  if (st) return st;
  size_t off = 0;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    const ChirpRec& c = h->chirps[sl];
    if (c.tone < 0 || !(c.flags & awgk::TONE_EXACT)) continue;
    awgk::TableArgs ta;
    ta.chirps = h->d_chirps;
    ta.slot = (int32_t)sl;
    ta.out = h->d_tab + off;
    std::memcpy(ta.inv_odd, h->inv_odd, sizeof(ta.inv_odd));
    cudaError_t e = counted(h, awgk::launch_exact_table(ta, c.L, h->priv));
    if (e != cudaSuccess) return cuda_fail(e, "exact table launch");
    h->tones[(size_t)c.tone].tab_off = (int32_t)off;
    off += (size_t)c.L + 1;
  }
  if (!sync) return AWG_OK;
  cudaError_t e = cudaStreamSynchronize(h->priv);
  if (e != cudaSuccess) return cuda_fail(e, "exact tables");
  return AWG_OK;
}

// Stream-ordered upload through the pinned staging buffer: stage_begin makes room for `bytes`
// (after the previous upload's copies have read the buffer) and orders the private stream after
// the last render issued; stage_runs queues the copies of the records at the given sorted unique
// indices; stage_end marks the upload's completion (ev_upload) for later launches to wait on.
int stage_begin(awg_t* h, size_t bytes) {
  cudaError_t e;
  if (h->upload_pending) {
    if ((e = cudaEventSynchronize(h->ev_upload)) != cudaSuccess) return cuda_fail(e, "waiting for the last upload");
    h->upload_pending = false;
  }
  if (bytes > h->cap_stage) {
    const size_t ncap = std::max(bytes, 2 * h->cap_stage);
    unsigned char* p = nullptr;
    if (cudaHostAlloc((void**)&p, ncap, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return fail(AWG_ENOMEM, "cudaHostAlloc upload staging");
    }
    if (h->stage) cudaFreeHost(h->stage);
    h->stage = p;
    h->cap_stage = ncap;
  }
  if (h->have_done && (e = cudaStreamWaitEvent(h->priv, h->ev_done, 0)) != cudaSuccess)
    return cuda_fail(e, "upload ordering");
  return AWG_OK;
}

template <class T>
int stage_runs(awg_t* h, T* dev, const std::vector<T>& host, const std::vector<int32_t>& idx, size_t* off) {
  size_t i = 0;
  while (i < idx.size()) {
    size_t j = i + 1;
    while (j < idx.size() && idx[j] == idx[j - 1] + 1) ++j;
    const size_t first = (size_t)idx[i], count = (size_t)(idx[j - 1] - idx[i] + 1);
    const size_t bytes = count * sizeof(T);
    std::memcpy(h->stage + *off, host.data() + first, bytes);
    cudaError_t e = cudaMemcpyAsync(dev + first, h->stage + *off, bytes, cudaMemcpyHostToDevice, h->priv);
    if (e != cudaSuccess) return cuda_fail(e, "staged upload");
    *off += bytes;
    i = j;
  }
  return AWG_OK;
}

int stage_end(awg_t* h) {
  cudaError_t e = cudaEventRecord(h->ev_upload, h->priv);
  if (e != cudaSuccess) return cuda_fail(e, "upload event");
  h->upload_pending = true;
  return AWG_OK;
}

int render_direct(awg_t* h, int64_t n, float* out_f, int16_t* out_q, void* stream, int32_t q_stride,
                  const float* base, int32_t skip_static, const int32_t* tone_list = nullptr, int32_t n_list = 0,
                  int32_t list_split = 0, const int32_t* list_bounds = nullptr);
int render_engine(awg_t* h, int64_t n, float* out_f, int16_t* out_q, void* stream, int32_t q_stride);

int render_impl(awg_t* h, int64_t n, float* out_f, int16_t* out_q, void* stream, int32_t q_stride = 1) {
  if (h && h->static_engine != AWG_STATIC_DIRECT && n > 0 && (out_f || out_q) &&
      !(h->periodic_start >= 0 && !out_f && h->cursor + n > h->periodic_start))
    return render_engine(h, n, out_f, out_q, stream, q_stride);
  return render_direct(h, n, out_f, out_q, stream, q_stride, nullptr, 0);
}

int render_direct(awg_t* h, int64_t n, float* out_f, int16_t* out_q, void* stream, int32_t q_stride,
                  const float* base, int32_t skip_static, const int32_t* tone_list, int32_t n_list,
                  int32_t list_split, const int32_t* list_bounds) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0) return fail(AWG_EINVAL, "sample count must be >= 0");
  if (n == 0) return AWG_OK;
  if (!out_f && !out_q) return fail(AWG_EINVAL, "no output buffer");
  if (h->cursor > INT64_MAX - n) return fail(AWG_EINVAL, "sample index overflow");
  cudaStream_t s = (cudaStream_t)stream;
  if (h->periodic_start >= 0 && !out_f && h->cursor + n > h->periodic_start) {
    // periodic hand-off: render up to the start of the periodic part, replay the table after it
    const int64_t n1 = std::max<int64_t>(0, h->periodic_start - h->cursor);
    if (n1 > 0) {
      const int st = render_impl(h, n1, nullptr, out_q, stream, q_stride);
      if (st) return st;
    }
    const int64_t c = h->cursor, n2 = n - n1;
    cudaError_t e;
    if ((e = cudaEventRecord(h->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = counted(h, awgk::launch_replay(h->d_periodic, h->periodic_log2, c, n2, out_q + (size_t)n1 * (size_t)q_stride,
                                 q_stride, s))) != cudaSuccess)
      return cuda_fail(e, "replay launch");
    if ((e = cudaEventRecord(h->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = cudaEventRecord(h->ev_done, s)) != cudaSuccess) return cuda_fail(e, "event");
    h->timed = true;
    h->have_done = true;
    h->cursor = c + n2;
    return AWG_OK;
  }
  const int64_t c = h->cursor;
  const int64_t tile0 = c / awgk::TILE;
  const int64_t tile_last = (c + n - 1) / awgk::TILE;
  const int64_t n_tiles64 = tile_last - tile0 + 1;
  if (n_tiles64 > (int64_t)(INT32_MAX / awgk::MAX_SPLIT)) return fail(AWG_EINVAL, "render window too long");
  const int32_t n_tiles = (int32_t)n_tiles64;
  const int64_t span0 = tile0 * awgk::TILE, span1 = (tile_last + 1) * awgk::TILE - 1;

  std::vector<int32_t> active;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    const ChirpRec& cr = h->chirps[sl];
    if (cr.tone < 0 || (cr.flags & awgk::TONE_EXACT)) continue;
    const int64_t ne = cr.n_s + cr.L;
    if (cr.n_s <= span1 && ne >= span0) active.push_back((int32_t)sl);
  }
  int st = ensure(&h->d_recs, &h->cap_recs, std::max<size_t>(1, active.size() * (size_t)n_tiles), h, "tile records");
  if (st) return st;
  // With a split, the window goes out in launches of at most SPLIT_LAUNCH_TILES tiles, chained by
  // programmatic dependent launch, on alternating scratch buffers.
  const int32_t split_used = tone_list ? list_split : h->split;
  const bool scratch = split_used > 1;
  const int32_t per_launch = scratch ? std::min(n_tiles, SPLIT_LAUNCH_TILES) : n_tiles;
  if (scratch && (st = ensure_split_scratch(h, per_launch, split_used))) return st;

  // The chirp tile set-up runs in stream order right before the render.  (Running it on a second
  // stream, overlapped with the previous render, takes SM slots from the render and pushes its
  // grid into a second wave; measured slower.)
  cudaError_t e;
  cudaEvent_t pe[4] = {nullptr, nullptr, nullptr, nullptr};
  if (h->profiling) {
    while (h->prof_ev.size() < 4 * (h->prof_calls + 1)) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "profiling event");
      h->prof_ev.push_back(ev);
    }
    for (int i = 0; i < 4; ++i) pe[i] = h->prof_ev[4 * h->prof_calls + (size_t)i];
  }
  int64_t launches = 0;
  if ((e = order_after_uploads(h, s)) != cudaSuccess) return cuda_fail(e, "upload ordering");
  if ((e = cudaEventRecord(h->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
  if (pe[0] && (e = cudaEventRecord(pe[0], s)) != cudaSuccess) return cuda_fail(e, "event");
  for (size_t b = 0; b < active.size(); b += awgk::MAX_ACTIVE_PER_LAUNCH) {
    awgk::PrepArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.chirps = h->d_chirps;
    pa.recs = h->d_recs;
    pa.act_of_slot = h->d_act;
    pa.tile0 = tile0;
    pa.n_tiles = n_tiles;
    pa.n_active = (int32_t)std::min<size_t>(awgk::MAX_ACTIVE_PER_LAUNCH, active.size() - b);
    pa.act_base = (int32_t)b;
    std::memcpy(pa.W, h->W, sizeof(pa.W));
    std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
    for (int i = 0; i < pa.n_active; ++i) pa.slots[i] = active[b + (size_t)i];
    if ((e = counted(h, awgk::launch_prep(pa, s))) != cudaSuccess) return cuda_fail(e, "prep launch");
    ++launches;
  }
  if (pe[1] && (e = cudaEventRecord(pe[1], s)) != cudaSuccess) return cuda_fail(e, "event");
  if (pe[2] && (e = cudaEventRecord(pe[2], s)) != cudaSuccess) return cuda_fail(e, "event");
  awgk::RenderArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.tones = h->d_tones;
  ra.exact_tab = h->d_tab;
  ra.chirps = h->d_chirps;
  ra.recs = h->d_recs;
  ra.act_of_slot = h->d_act;
  ra.K = h->K;
  ra.split = h->split;
  ra.sine_mode = h->sine_mode;
  ra.q_stride = q_stride;
  ra.base = base;
  ra.skip_static = skip_static;
  ra.tone_list = tone_list;
  ra.n_list = n_list;
  if (tone_list) {
    ra.split = list_split;
    for (int r = 0; r <= list_split; ++r) ra.bounds[r] = list_bounds[r];
  }
  ra.scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
  ra.status = h->d_status;
  std::memcpy(ra.inv_odd, h->inv_odd, sizeof(ra.inv_odd));
  for (int32_t t0 = 0, i = 0; t0 < n_tiles; t0 += per_launch, ++i) {
    awgk::RenderArgs rs = ra;
    const int32_t nt = std::min(per_launch, n_tiles - t0);
    const int64_t w0 = std::max(c, (tile0 + t0) * (int64_t)awgk::TILE);
    const int64_t w1 = std::min(c + n, (tile0 + t0 + nt) * (int64_t)awgk::TILE);
    rs.tile0 = tile0 + t0;
    rs.n_tiles = nt;
    rs.rec_stride = n_tiles;
    rs.rec_tile0 = t0;
    rs.win_start = w0;
    rs.win_end = w1;
    rs.out_q = out_q ? out_q + (size_t)(w0 - c) * (size_t)(q_stride ? q_stride : 1) : nullptr;
    rs.out_f = out_f ? out_f + (w0 - c) : nullptr;
    rs.base = base ? base + (w0 - c) : nullptr;
    if (scratch) {
      rs.part = split_part(h, i & 1);
      rs.tile_ctr = split_ctr(h, i & 1);
      rs.pdl = n_tiles > per_launch ? (i == 0 ? 1 : 2) : 0;
    }
    if ((e = counted(h, awgk::launch_render(rs, s))) != cudaSuccess) return cuda_fail(e, "render launch");
    ++launches;
  }
  if (pe[3]) {
    if ((e = cudaEventRecord(pe[3], s)) != cudaSuccess) return cuda_fail(e, "event");
    ++h->prof_calls;
    h->prof_launches += launches;
  }
  if ((e = cudaEventRecord(h->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
  if ((e = cudaEventRecord(h->ev_done, s)) != cudaSuccess) return cuda_fail(e, "event");
  h->timed = true;
  h->have_done = true;
  h->cursor = c + n;
  return AWG_OK;
}

}  // namespace

namespace {

// Tensor-core static engine: in every 4096-sample tile, the tones that are static there
// (tile_segment_static, either segment of the tone) are summed by the table GEMM over 256-sample
// rows aligned to absolute sample indices, two column pairs per tone (before and after its
// chirp); the others by the render kernel, which skips the static ones and adds the GEMM's FP32
// sum before quantising.  The split depends on the tile and the tone state only, so a sample's
// value does not depend on how the stream is cut into calls.  Pieces of at most 2^26 samples.

// The render part's tone split: the tones that hold a chirp or a ramp at all (they change only when
// chirps, ramps or tones are set, never while rendering), about the same number of them in each of
// the split's tone ranges.  With every tone holding one this is the plain split.
struct EngineSplit {
  int32_t n_flagged = 0, split = 1;
  int32_t bounds[awgk::MAX_SPLIT + 1];
};
const std::vector<int32_t>& flagged_tones(awg_t* h) {
  if (!h->flagged_ok) {
    h->amax = max_amplitude_scan(h);
    h->flagged.clear();
    for (size_t k = 0; k < h->tones.size(); ++k)
      if (h->tones[k].slot >= 0 || (h->tones[k].flags & awgk::TONE_AMP_RAMP)) h->flagged.push_back((int32_t)k);
    h->flagged_ok = true;
  }
  return h->flagged;
}
EngineSplit engine_split(awg_t* h) {
  EngineSplit es;
  const std::vector<int32_t>& fl = flagged_tones(h);
  es.n_flagged = (int32_t)fl.size();
  es.split = awgk::tone_split_for(es.n_flagged);
  es.bounds[0] = 0;
  es.bounds[es.split] = h->K;
  // range r starts at the flagged tone at position floor(n_flagged r / split)
  for (int32_t r = 1; r < es.split; ++r) es.bounds[r] = fl[(size_t)((int64_t)es.n_flagged * r / es.split)];
  return es;
}

// The tones that are not static (tile_segment_static) in some tile of the window [c, c + m): a
// chirp or an amplitude ramp meets the tile span.  The render visits only these, in ascending
// order, and still skips them in the tiles where they are static.
void engine_list(awg_t* h, int64_t c, int64_t m, std::vector<int32_t>* list) {
  const int64_t t_first = c / awgk::TILE, t_last = (c + m - 1) / awgk::TILE;
  const int64_t s0 = t_first * awgk::TILE, s1 = (t_last + 1) * awgk::TILE - 1;
  list->clear();
  for (int32_t k : flagged_tones(h)) {
    const ToneRec& t = h->tones[(size_t)k];
    if ((t.slot >= 0 && !(s1 < t.n_s || s0 > t.n_e)) ||
        ((t.flags & awgk::TONE_AMP_RAMP) && !(s1 <= t.a_ns || s0 >= t.a_ns + t.a_L)))
      list->push_back(k);
  }
}

// GEMM arguments of the window [c, c + m) into out_q (every tone static there) or the FP32 sum
// out_f.  two_segments: some tone of the handle has held a chirp or a ramp (four columns per tone).
awgk::TableArgs2 engine_gemm_args(awg_t* h, int64_t c, int64_t m, bool two_segments, int16_t* out_q, float* out_f) {
  const size_t Kp = two_segments ? awgk::table_kp_window(std::max(h->K, 1)) : awgk::table_kp(std::max(h->K, 1));
  const size_t b_elems = (size_t)256 * Kp;
  awgk::TableArgs2 t;
  std::memset(&t, 0, sizeof(t));
  t.tones = h->d_tones;
  t.K = h->K;
  t.nb_log2 = 8;
  t.row_base = c >> 8;
  t.M = ((c + m - 1) >> 8) - t.row_base + 1;
  t.win_start = c;
  t.win_end = c + m;
  t.window_mode = two_segments ? 1 : 0;
  t.invariant = 1;
  t.precision = h->static_engine == AWG_STATIC_GEMM_FP16 ? AWG_PREC_FP16 : AWG_PREC_BF16;
  t.b_hi = h->d_gemm;
  t.b_lo = h->d_gemm + b_elems;
  t.out_q = out_q;
  t.out_f = out_f;
  t.scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
  t.a_scale = awgk::table_amp_scale(max_amplitude(h));
  t.status = h->d_status;
  return t;
}

// B operand of the handle's GEMM (cos, sin of 2 pi n2 F / 2^64 per tone and segment, hi + lo).
int engine_operand(awg_t* h, bool two_segments, cudaStream_t s) {
  const size_t Kp = two_segments ? awgk::table_kp_window(std::max(h->K, 1)) : awgk::table_kp(std::max(h->K, 1));
  int st = ensure(&h->d_gemm, &h->cap_gemm, 2 * (size_t)256 * Kp, h, "table GEMM operands");
  if (st) return st;
  const awgk::TableArgs2 t = engine_gemm_args(h, h->cursor, awgk::TILE, two_segments, nullptr, nullptr);
  cudaError_t e;
  if ((e = counted(h, awgk::launch_table_prep(t, s))) != cudaSuccess) return cuda_fail(e, "static operand launch");
  return AWG_OK;
}

int render_engine(awg_t* h, int64_t n, float* out_f, int16_t* out_q, void* stream, int32_t q_stride) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t PIECE = (int64_t)1 << 26;
  const EngineSplit es = engine_split(h);
  // no tone has ever held a chirp or a ramp: every tone is static in one segment everywhere, and
  // the GEMM takes the table's two columns per tone instead of four (half the work)
  const bool two_segments = es.n_flagged > 0;
  for (int64_t off = 0; off < n; off += PIECE) {
    const int64_t m = std::min(PIECE, n - off), c = h->cursor;
    engine_list(h, c, m, &h->list);
    const bool all_static = q_stride == 1 && h->K > 0 && h->list.empty();
    int16_t* oq = out_q ? out_q + (size_t)off * (size_t)q_stride : nullptr;
    float* of = out_f ? out_f + off : nullptr;
    int st;
    if (h->K == 0) {
      if ((st = render_direct(h, m, of, oq, stream, q_stride, nullptr, 0))) return st;
      continue;
    }
    if (!all_static && (st = ensure(&h->d_base, &h->cap_base, (size_t)m, h, "static sum"))) return st;
    cudaError_t e;
    if ((e = order_after_uploads(h, s)) != cudaSuccess) return cuda_fail(e, "upload ordering");
    if ((e = cudaEventRecord(h->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
    if ((st = engine_operand(h, two_segments, s))) return st;
    const awgk::TableArgs2 t = engine_gemm_args(h, c, m, two_segments, all_static ? oq : nullptr, all_static ? of : h->d_base);
    if ((e = counted(h, awgk::launch_table_gemm(t, s))) != cudaSuccess) return cuda_fail(e, "static GEMM launch");
    if (all_static) {
      if ((e = cudaEventRecord(h->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
      if ((e = cudaEventRecord(h->ev_done, s)) != cudaSuccess) return cuda_fail(e, "event");
      h->timed = true;
      h->have_done = true;
      h->cursor = c + m;
      continue;
    }
    // (a list of all K tones is left out: one bulk copy per stage instead of one per tone)
    const int32_t n_list = (int32_t)h->list.size();
    const bool use_list = n_list < h->K;
    if (use_list) {
      if ((st = ensure(&h->d_list, &h->cap_list, std::max<size_t>(1, (size_t)n_list), h, "tone list"))) return st;
      if (n_list > 0 &&
          (e = cudaMemcpyAsync(h->d_list, h->list.data(), (size_t)n_list * sizeof(int32_t), cudaMemcpyHostToDevice,
                               s)) != cudaSuccess)
        return cuda_fail(e, "tone list upload");
    }
    if ((st = render_direct(h, m, of, oq, stream, q_stride, h->d_base, 1, use_list ? h->d_list : nullptr, n_list,
                            es.split, es.bounds)))
      return st;
  }
  return AWG_OK;
}

}  // namespace

size_t awgk::render_recs_needed(const awg_t* h, int64_t n) {
  if (!h || n <= 0) return 0;
  const int64_t c = h->cursor;
  const int64_t tile0 = c / awgk::TILE, tile_last = (c + n - 1) / awgk::TILE;
  const int64_t span0 = tile0 * awgk::TILE, span1 = (tile_last + 1) * awgk::TILE - 1;
  size_t active = 0;
  for (const ChirpRec& cr : h->chirps)
    if (cr.tone >= 0 && !(cr.flags & awgk::TONE_EXACT) && cr.n_s <= span1 && cr.n_s + cr.L >= span0) ++active;
  return active * (size_t)(tile_last - tile0 + 1);
}

size_t awgk::render_slots(const awg_t* h) { return h ? h->chirps.size() : 0; }

int awgk::engine_setup(awg_t* h, int32_t engine, cudaStream_t s, int32_t* render_split) {
  if (!h || (engine != AWG_STATIC_GEMM_FP16 && engine != AWG_STATIC_GEMM_BF16))
    return fail(AWG_EINVAL, "engine_setup: bad arguments");
  h->static_engine = engine;
  const EngineSplit es = engine_split(h);
  cudaError_t e = order_after_uploads(h, s);
  if (e != cudaSuccess) return cuda_fail(e, "upload ordering");
  const int st = engine_operand(h, es.n_flagged > 0, s);
  if (st) return st;
  if (render_split) *render_split = es.split;
  return AWG_OK;
}

size_t awgk::engine_list_needed(awg_t* h, int64_t n) {
  if (!h || n <= 0) return 0;
  std::vector<int32_t> list;
  engine_list(h, h->cursor, n, &list);
  return list.size();
}

int awgk::prepare_render_engine(awg_t* h, int64_t n, int16_t* out_q, cudaStream_t s, awgk::RenderArgs* ra,
                                awgk::TileRec* recs, size_t recs_cap, int32_t* act, float* base, int32_t* d_list,
                                int32_t* h_list, size_t list_cap, bool* need_render) {
  if (!h || n <= 0 || !out_q || !ra || !base || !need_render || h->K == 0 || h->static_engine == AWG_STATIC_DIRECT)
    return fail(AWG_EINVAL, "prepare_render_engine: bad arguments");
  const int64_t c = h->cursor;
  const EngineSplit es = engine_split(h);
  std::vector<int32_t> list;
  engine_list(h, c, n, &list);
  const bool all_static = list.empty();
  cudaError_t e = order_after_uploads(h, s);
  if (e != cudaSuccess) return cuda_fail(e, "upload ordering");
  const awgk::TableArgs2 t = engine_gemm_args(h, c, n, es.n_flagged > 0, all_static ? out_q : nullptr, all_static ? nullptr : base);
  if ((e = counted(h, awgk::launch_table_gemm(t, s))) != cudaSuccess) return cuda_fail(e, "static GEMM launch");
  if (all_static) {
    *need_render = false;
    std::memset(ra, 0, sizeof(*ra));
    h->cursor = c + n;
    return AWG_OK;
  }
  // the listed tones through the render kernel, with the GEMM's sum added before quantising
  const int32_t n_list = (int32_t)list.size();
  const bool use_list = n_list < h->K;
  if (use_list) {
    if ((size_t)n_list > list_cap || !d_list || !h_list) return fail(AWG_ENOMEM, "prepare_render_engine: list arena too small");
    std::memcpy(h_list, list.data(), (size_t)n_list * sizeof(int32_t));
    if ((e = cudaMemcpyAsync(d_list, h_list, (size_t)n_list * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "tone list upload");
  }
  const int st = awgk::prepare_render(h, n, out_q, nullptr, s, ra, recs, recs_cap, act);
  if (st) {
    h->cursor = c;
    return st;
  }
  ra->base = base;
  ra->skip_static = 1;
  ra->tone_list = use_list ? d_list : nullptr;
  ra->n_list = n_list;
  ra->split = es.split;
  for (int r = 0; r <= es.split; ++r) ra->bounds[r] = es.bounds[r];
  *need_render = true;
  return AWG_OK;
}

int awgk::prepare_render(awg_t* h, int64_t n, int16_t* out_q, float* out_f, cudaStream_t s, awgk::RenderArgs* ra,
                         awgk::TileRec* recs, size_t recs_cap, int32_t* act, size_t* recs_need) {
  if (!h || n <= 0 || (!out_q && !out_f) || !ra) return fail(AWG_EINVAL, "prepare_render: bad arguments");
  const int64_t c = h->cursor;
  const int64_t tile0 = c / awgk::TILE, tile_last = (c + n - 1) / awgk::TILE;
  const int32_t n_tiles = (int32_t)(tile_last - tile0 + 1);
  const int64_t span0 = tile0 * awgk::TILE, span1 = (tile_last + 1) * awgk::TILE - 1;
  std::vector<int32_t> active;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    const ChirpRec& cr = h->chirps[sl];
    if (cr.tone < 0 || (cr.flags & awgk::TONE_EXACT)) continue;
    if (cr.n_s <= span1 && cr.n_s + cr.L >= span0) active.push_back((int32_t)sl);
  }
  const size_t need = active.size() * (size_t)n_tiles;
  if (recs_need) *recs_need = need;
  if (recs || act) {
    if (need > recs_cap || (!recs && need) || (!act && need)) return fail(AWG_ENOMEM, "prepare_render: arena too small");
  } else {
    int st = ensure(&h->d_recs, &h->cap_recs, std::max<size_t>(1, need), h, "tile records");
    if (st) return st;
    recs = h->d_recs;
    act = h->d_act;
  }
  {
    const cudaError_t e = order_after_uploads(h, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload ordering");
  }
  for (size_t b = 0; b < active.size(); b += awgk::MAX_ACTIVE_PER_LAUNCH) {
    awgk::PrepArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.chirps = h->d_chirps;
    pa.recs = recs;
    pa.act_of_slot = act;
    pa.tile0 = tile0;
    pa.n_tiles = n_tiles;
    pa.n_active = (int32_t)std::min<size_t>(awgk::MAX_ACTIVE_PER_LAUNCH, active.size() - b);
    pa.act_base = (int32_t)b;
    std::memcpy(pa.W, h->W, sizeof(pa.W));
    std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
    for (int i = 0; i < pa.n_active; ++i) pa.slots[i] = active[b + (size_t)i];
    cudaError_t e = counted(h, awgk::launch_prep(pa, s));
    if (e != cudaSuccess) return cuda_fail(e, "prep launch");
  }
  std::memset(ra, 0, sizeof(*ra));
  ra->tones = h->d_tones;
  ra->exact_tab = h->d_tab;
  ra->chirps = h->d_chirps;
  ra->recs = recs;
  ra->act_of_slot = act;
  ra->K = h->K;
  ra->split = h->split;
  ra->sine_mode = h->sine_mode;
  ra->tile0 = tile0;
  ra->n_tiles = n_tiles;
  ra->win_start = c;
  ra->win_end = c + n;
  ra->out_q = out_q;
  ra->out_f = out_f;
  ra->scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
  ra->status = h->d_status;
  std::memcpy(ra->inv_odd, h->inv_odd, sizeof(ra->inv_odd));
  h->cursor = c + n;
  return AWG_OK;
}

namespace {

// Chirp slots active in the window [c, c + n) (tile-aligned span), excluding exact-table chirps.
std::vector<int32_t> active_slots(const awg_t* h, int64_t c, int64_t n, int64_t* tile0, int32_t* n_tiles) {
  const int64_t t0 = c / awgk::TILE, t1 = (c + n - 1) / awgk::TILE;
  const int64_t span0 = t0 * awgk::TILE, span1 = (t1 + 1) * awgk::TILE - 1;
  std::vector<int32_t> active;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    const ChirpRec& cr = h->chirps[sl];
    if (cr.tone < 0 || (cr.flags & awgk::TONE_EXACT)) continue;
    if (cr.n_s <= span1 && cr.n_s + cr.L >= span0) active.push_back((int32_t)sl);
  }
  *tile0 = t0;
  *n_tiles = (int32_t)(t1 - t0 + 1);
  return active;
}

// n_chunks consecutive chunk renders, pipelined.  The chunks are taken in groups whose chirp tile
// records fit a fixed budget; for each group one set-up launch computes the records of every
// chunk of the group (in stream order: it waits for everything before it), then the chunk renders
// follow with programmatic dependent launch: the first waits for the set-up, and each later one
// may start as soon as every CTA of the one before has started, so a render's tail overlaps the
// next render's start (a chunk is one wave of the device or less at typical sizes).  A join kernel
// (stream order, then a bounded wait on a device counter of render CTAs that stored their
// samples) ends each group, so the next group's set-up and later work on the stream see every
// chunk complete.
constexpr size_t SEQ_RECORD_BUDGET = (size_t)1 << 22;   // 4M records (704 MiB) per group

// The device counter of render CTAs that stored their samples (pipelined sequences), zero at
// allocation; every sequence's join waits for its own running total.
int ensure_seq_counter(awg_t* h) {
  if (h->d_seq_exit) return AWG_OK;
  if (cudaMalloc((void**)&h->d_seq_exit, sizeof(unsigned long long)) != cudaSuccess)
    return fail(AWG_ENOMEM, "cudaMalloc sequence counter");
  cudaError_t e = cudaMemset(h->d_seq_exit, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "sequence counter");
  return AWG_OK;
}

int render_chunks_impl(awg_t* h, int64_t chunk, int32_t n_chunks, int16_t* out, cudaStream_t s, int64_t tail = 0) {
  // chunks 0 .. n_chunks - 1 of `chunk` samples, then (tail > 0) one of `tail` samples
  const int64_t n_total = (int64_t)n_chunks * chunk + tail;
  if (tail > 0) ++n_chunks;
  auto span = [&](int32_t a, int32_t b) {   // samples of chunks a .. b - 1
    return std::min((int64_t)b * chunk, n_total) - (int64_t)a * chunk;
  };
  cudaError_t e;
  int st0 = ensure_seq_counter(h);
  if (st0) return st0;
  const int64_t c0 = h->cursor;
  struct Group {
    int32_t g0, g1;
    int64_t tile0;
    int32_t n_tiles;
    std::vector<int32_t> active;
  };
  std::vector<Group> groups;
  size_t max_recs = 1;
  for (int32_t g0 = 0; g0 < n_chunks;) {
    // the largest group from g0 whose records fit the budget (at least one chunk)
    Group g;
    g.g0 = g0;
    g.g1 = g0 + 1;
    g.active = active_slots(h, c0 + (int64_t)g0 * chunk, span(g0, g0 + 1), &g.tile0, &g.n_tiles);
    while (g.g1 < n_chunks) {
      int64_t t0;
      int32_t nt;
      std::vector<int32_t> a2 = active_slots(h, c0 + (int64_t)g0 * chunk, span(g0, g.g1 + 1), &t0, &nt);
      if (a2.size() * (size_t)nt > SEQ_RECORD_BUDGET || nt > INT32_MAX / awgk::MAX_SPLIT) break;
      g.active.swap(a2);
      g.tile0 = t0;
      g.n_tiles = nt;
      ++g.g1;
    }
    max_recs = std::max(max_recs, g.active.size() * (size_t)g.n_tiles);
    g0 = g.g1;
    groups.push_back(std::move(g));
  }
  int st = ensure(&h->d_seq_recs, &h->cap_seq_recs, max_recs, h, "tile records");
  if (st) return st;
  if (h->split > 1 && (st = ensure_split_scratch(h, (int32_t)(chunk / awgk::TILE + 2), h->split))) return st;
  st = ensure(&h->d_seq_act, &h->cap_seq_act, std::max<size_t>(1, h->chirps.size()), h, "slot map");
  if (st) return st;
  // profiling: events at the start, after the first group's set-up (twice: the set-up's end and the
  // renders' start) and after the last join; the first render then starts in plain stream order
  cudaEvent_t pe[4] = {nullptr, nullptr, nullptr, nullptr};
  if (h->profiling) {
    while (h->prof_ev.size() < 4 * (h->prof_calls + 1)) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "profiling event");
      h->prof_ev.push_back(ev);
    }
    for (int i = 0; i < 4; ++i) pe[i] = h->prof_ev[4 * h->prof_calls + (size_t)i];
  }
  const int64_t launches0 = h->n_launches;
  if ((e = order_after_uploads(h, s)) != cudaSuccess) return cuda_fail(e, "upload ordering");
  if ((e = cudaEventRecord(h->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
  if (pe[0] && (e = cudaEventRecord(pe[0], s)) != cudaSuccess) return cuda_fail(e, "event");
  for (const Group& grp : groups) {
    const int32_t g0 = grp.g0, g1 = grp.g1;
    const int64_t tile0 = grp.tile0;
    const int32_t n_tiles = grp.n_tiles;
    const std::vector<int32_t>& active = grp.active;
    for (size_t b = 0; b < active.size(); b += awgk::MAX_ACTIVE_PER_LAUNCH) {
      awgk::PrepArgs pa;
      std::memset(&pa, 0, sizeof(pa));
      pa.chirps = h->d_chirps;
      pa.recs = h->d_seq_recs;
      pa.act_of_slot = h->d_seq_act;
      pa.tile0 = tile0;
      pa.n_tiles = n_tiles;
      pa.n_active = (int32_t)std::min<size_t>(awgk::MAX_ACTIVE_PER_LAUNCH, active.size() - b);
      pa.act_base = (int32_t)b;
      std::memcpy(pa.W, h->W, sizeof(pa.W));
      std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
      for (int i = 0; i < pa.n_active; ++i) pa.slots[i] = active[b + (size_t)i];
      if ((e = counted(h, awgk::launch_prep(pa, s))) != cudaSuccess) return cuda_fail(e, "prep launch");
    }
    if (pe[1] && g0 == 0) {
      if ((e = cudaEventRecord(pe[1], s)) != cudaSuccess) return cuda_fail(e, "event");
      if ((e = cudaEventRecord(pe[2], s)) != cudaSuccess) return cuda_fail(e, "event");
    }
    for (int32_t c = g0; c < g1; ++c) {
      const int64_t wc = c0 + (int64_t)c * chunk, len = span(c, c + 1);
      const int64_t t_first = wc / awgk::TILE, t_last = (wc + len - 1) / awgk::TILE;
      awgk::RenderArgs ra;
      std::memset(&ra, 0, sizeof(ra));
      ra.tones = h->d_tones;
      ra.exact_tab = h->d_tab;
      ra.chirps = h->d_chirps;
      ra.recs = h->d_seq_recs;
      ra.act_of_slot = h->d_seq_act;
      ra.rec_stride = n_tiles;
      ra.rec_tile0 = (int32_t)(t_first - tile0);
      ra.K = h->K;
      ra.split = h->split;
      ra.sine_mode = h->sine_mode;
      ra.tile0 = t_first;
      ra.n_tiles = (int32_t)(t_last - t_first + 1);
      ra.win_start = wc;
      ra.win_end = wc + len;
      ra.out_q = out + (size_t)c * (size_t)chunk;
      ra.scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
      ra.status = h->d_status;
      std::memcpy(ra.inv_odd, h->inv_odd, sizeof(ra.inv_odd));
      ra.pdl = c == g0 ? 1 : 2;
      ra.exit_ctr = h->d_seq_exit;
      if (h->split > 1) {   // alternating scratch (see tile_epilogue_split)
        ra.part = split_part(h, c & 1);
        ra.tile_ctr = split_ctr(h, c & 1);
      }
      if ((e = counted(h, awgk::launch_render(ra, s))) != cudaSuccess) return cuda_fail(e, "render launch");
      h->seq_exit_target += (unsigned long long)ra.n_tiles * (unsigned long long)h->split;
    }
    if ((e = counted(h, awgk::launch_join(h->d_seq_exit, h->seq_exit_target, h->d_status, awgk::JOIN_LIMIT_NS, s))) !=
        cudaSuccess)
      return cuda_fail(e, "join launch");
  }
  if (pe[3]) {
    if ((e = cudaEventRecord(pe[3], s)) != cudaSuccess) return cuda_fail(e, "event");
    ++h->prof_calls;
    h->prof_launches += h->n_launches - launches0;
  }
  if ((e = cudaEventRecord(h->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
  if ((e = cudaEventRecord(h->ev_done, s)) != cudaSuccess) return cuda_fail(e, "event");
  h->timed = true;
  h->have_done = true;
  h->cursor = c0 + n_total;
  return AWG_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

int awg_version(void) { return 10000; }

const char* awg_last_error(void) { return g_err.c_str(); }

int awg_freq_word(double f_hz, double fs_hz, uint64_t* out_word) {
  if (!out_word) return fail(AWG_EINVAL, "null output");
  return freq_word_impl(f_hz, fs_hz, out_word);
}

int awg_phase_word(double theta_rad, uint64_t* out_word) {
  if (!out_word) return fail(AWG_EINVAL, "null output");
  return phase_word_impl(theta_rad, out_word);
}

int awg_grid_word(double f_hz, double fs_hz, int32_t log2_len, uint64_t* out_word, int64_t* out_j) {
  if (!out_word) return fail(AWG_EINVAL, "null output");
  if (!(is_fin(fs_hz) && fs_hz > 0)) return fail(AWG_EINVAL, "sample rate must be finite and > 0");
  if (log2_len < 1 || log2_len > 40) return fail(AWG_EINVAL, "log2_len must be 1..40");
  if (!is_fin(f_hz) || f_hz < 0 || f_hz >= fs_hz) return fail(AWG_EINVAL, "tone frequency must lie in [0, fs)");
  double j = std::rint(std::ldexp(f_hz / fs_hz, log2_len));
  int64_t ji = (int64_t)j;
  *out_word = ((uint64_t)ji) << (64 - log2_len);
  if (out_j) *out_j = ji;
  return AWG_OK;
}

int awg_chirp_length(double duration_s, double fs_hz, int64_t* out_L) {
  if (!out_L) return fail(AWG_EINVAL, "null output");
  return chirp_length_impl(duration_s, fs_hz, out_L);
}

int awg_chirp_render_flags(uint64_t F_start, uint64_t F_end, int64_t L, int32_t profile, int32_t* out_flags) {
  if (!out_flags) return fail(AWG_EINVAL, "null output");
  if (L < 1) return fail(AWG_EINVAL, "chirp length must be >= 1");
  if (profile != AWG_PROFILE_LINEAR && profile != AWG_PROFILE_MINJERK && profile != AWG_PROFILE_EXPONENTIAL)
    return fail(AWG_EINVAL, "unknown chirp profile");
  if (profile == AWG_PROFILE_EXPONENTIAL && (F_start == 0 || F_end == 0))
    return fail(AWG_EINVAL, "an exponential chirp needs f_start, f_end > 0");
  if (profile == AWG_PROFILE_EXPONENTIAL && F_start == F_end) profile = AWG_PROFILE_LINEAR;
  *out_flags = chirp_render_flags(F_start, F_end, L, profile);
  return AWG_OK;
}

int awg_chirp_coeffs(uint64_t F_start, uint64_t F_end, int64_t L, int32_t profile, uint64_t* out21) {
  if (!out21) return fail(AWG_EINVAL, "null output");
  W192 d[7];
  int st = chirp_coeffs_impl(F_start, F_end, L, profile, d);
  if (st) return st;
  for (int k = 0; k < 7; ++k)
    for (int j = 0; j < 3; ++j) out21[3 * k + j] = d[k].w[j];
  return AWG_OK;
}

awg_t* awg_create(double sample_rate_hz) {
  if (!(is_fin(sample_rate_hz) && sample_rate_hz > 0)) {
    fail(AWG_EINVAL, "sample rate must be finite and > 0");
    return nullptr;
  }
  awg_t* h = new awg();
  h->fs = sample_rate_hz;
  fill_constants(h);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = awgk::render_setup_attributes();
  if (e == cudaSuccess) {
    // the allocation-free render's fixed scratch: its device address is looked up (and its module
    // loaded) here, at set-up, so that no awg_render_noalloc call pays for it
    awgk::TileRec* recs = nullptr;
    int32_t* act = nullptr;
    e = awgk::noalloc_scratch(h->device, &recs, &act);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->priv, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_upload, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cuda_fail(e, "awg_create");
    awg_destroy(h);
    return nullptr;
  }
  if (upload_tones(h) || upload_chirps(h)) {
    awg_destroy(h);
    return nullptr;
  }
  return h;
}

void awg_destroy(awg_t* h) {
  if (!h) return;
  if (h->have_done) cudaEventSynchronize(h->ev_done);
  if (h->priv) cudaStreamSynchronize(h->priv);
  cudaFree(h->d_tones);
  cudaFree(h->d_chirps);
  cudaFree(h->d_act);
  cudaFree(h->d_recs);
  cudaFree(h->d_periodic);
  cudaFree(h->d_base);
  cudaFree(h->d_list);
  cudaFree(h->d_part);
  cudaFree(h->d_tctr);
  cudaFree(h->d_seq_recs);
  cudaFree(h->d_seq_act);
  cudaFree(h->d_seq_exit);
  cudaFree(h->d_status);
  cudaFree(h->d_words);
  cudaFree(h->d_trace);
  cudaFree(h->d_tab);
  cudaFree(h->d_gemm);
  for (cudaEvent_t ev : h->prof_ev) cudaEventDestroy(ev);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_upload) cudaEventDestroy(h->ev_upload);
  if (h->priv) cudaStreamDestroy(h->priv);
  if (h->stage) cudaFreeHost(h->stage);
  delete h;
}

int awg_set_tones(awg_t* h, const double* freq_hz, const double* amp, const double* phase_rad, int32_t n) {
  return set_tones_common(h, freq_hz, amp, phase_rad, n, 0);
}

int awg_set_tones_grid(awg_t* h, const double* freq_hz, int32_t log2_len, const double* amp,
                       const double* phase_rad, int32_t n) {
  if (log2_len < 1 || log2_len > 40) return fail(AWG_EINVAL, "log2_len must be 1..40");
  return set_tones_common(h, freq_hz, amp, phase_rad, n, log2_len);
}

int awg_set_chirps(awg_t* h, const int32_t* tone, const double* f_start_hz, const double* f_end_hz,
                   const double* duration_s, const int32_t* profile, const int64_t* start_sample, int32_t n) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0) return fail(AWG_EINVAL, "chirp count must be >= 0");
  if (n == 0) return AWG_OK;
  if (!tone || !f_start_hz || !f_end_hz || !duration_s || !profile || !start_sample)
    return fail(AWG_EINVAL, "null chirp array");
  struct Pending {
    int32_t tone;
    uint64_t F0, F1;
    int64_t L, ns;
    int32_t profile;
  };
  std::vector<Pending> pend((size_t)n);
  std::vector<char> seen((size_t)h->K, 0);
  for (int32_t i = 0; i < n; ++i) {
    Pending& p = pend[(size_t)i];
    p.tone = tone[i];
    if (p.tone < 0 || p.tone >= h->K) return fail(AWG_EINVAL, "chirp tone index out of range");
    if (seen[(size_t)p.tone]) return fail(AWG_EINVAL, "two chirps for one tone in one call");
    seen[(size_t)p.tone] = 1;
    int st = freq_word_impl(f_start_hz[i], h->fs, &p.F0);
    if (st) return st;
    st = freq_word_impl(f_end_hz[i], h->fs, &p.F1);
    if (st) return st;
    st = chirp_length_impl(duration_s[i], h->fs, &p.L);
    if (st) return st;
    p.profile = profile[i];
    if (p.profile != AWG_PROFILE_LINEAR && p.profile != AWG_PROFILE_MINJERK && p.profile != AWG_PROFILE_EXPONENTIAL)
      return fail(AWG_EINVAL, "unknown chirp profile");
    if (p.profile == AWG_PROFILE_EXPONENTIAL && (p.F0 == 0 || p.F1 == 0))
      return fail(AWG_EINVAL, "an exponential chirp needs f_start, f_end > 0");
    if (p.profile == AWG_PROFILE_EXPONENTIAL && p.F0 == p.F1) p.profile = AWG_PROFILE_LINEAR;   // the same phase
    p.ns = start_sample[i];
    if (p.ns < h->cursor) return fail(AWG_EINVAL, "chirp starts before the render cursor");
    if (p.ns > INT64_MAX / 2) return fail(AWG_EINVAL, "chirp start too large");
    const ToneRec& t = h->tones[(size_t)p.tone];
    if (t.slot >= 0 && t.n_e >= h->cursor) return fail(AWG_EINVAL, "tone already has a chirp that has not finished rendering");
  }
  int st;
  h->periodic_start = -1;
  // the coefficient words, end offsets and exact-table flags of every chirp: pure functions of
  // the chirp, computed on several host threads for large batches
  struct Coeffs {
    W192 d[7];
    uint64_t end_offset;
    int32_t flags;   // chirp_render_flags
    float rot_c, rot_s;   // rotator constants of F_end
  };
  std::vector<Coeffs> co(pend.size());
  auto work = [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i) {
      const Pending& p = pend[i];
      (void)chirp_coeffs_impl(p.F0, p.F1, p.L, p.profile, co[i].d);   // validated above
      co[i].end_offset = p.profile == AWG_PROFILE_EXPONENTIAL ? exp_end_offset(p.F0, p.F1, p.L)
                                                               : chirp_offset_word(co[i].d, p.L);
      co[i].flags = chirp_render_flags(p.F0, p.F1, p.L, p.profile);
      rotation_of(p.F1, &co[i].rot_c, &co[i].rot_s);
    }
  };
  HostPool::get().parallel_for(pend.size(), pend.size() / 32 + 1, work);
  std::vector<int32_t> changed_tones, changed_slots;
  for (size_t pi = 0; pi < pend.size(); ++pi) {
    const Pending& p = pend[pi];
    ToneRec& t = h->tones[(size_t)p.tone];
    changed_tones.push_back(p.tone);
    if (t.slot >= 0) {   // fold the finished chirp into the static state
      t.phi_ref = t.phi_post_ref;
      t.F = t.F_end;
      t.rot_c = t.rot_c_end;
      t.rot_s = t.rot_s_end;
      h->chirps[(size_t)t.slot].tone = -1;
      h->free_slots.push_back(t.slot);
      t.slot = -1;
    }
    const W192* d = co[pi].d;
    int32_t slot;
    if (!h->free_slots.empty()) {
      slot = h->free_slots.back();
      h->free_slots.pop_back();
    } else {
      slot = (int32_t)h->chirps.size();
      h->chirps.push_back(ChirpRec{});
    }
    changed_slots.push_back(slot);
    ChirpRec& c = h->chirps[(size_t)slot];
    std::memset(&c, 0, sizeof(c));
    for (int k = 0; k < 7; ++k)
      for (int j = 0; j < 3; ++j) c.d[3 * k + j] = d[k].w[j];
    c.phi_start = t.phi_ref + (uint64_t)p.ns * t.F;
    c.n_s = p.ns;
    c.L = p.L;
    c.tone = p.tone;
    c.flags = co[pi].flags;
    const uint64_t phi_end = c.phi_start + co[pi].end_offset;
    t.slot = slot;
    t.n_s = p.ns;
    t.n_e = p.ns + p.L;
    t.F_end = p.F1;
    t.rot_c_end = co[pi].rot_c;
    t.rot_s_end = co[pi].rot_s;
    t.phi_post_ref = phi_end - (uint64_t)t.n_e * p.F1;
    t.flags = (t.flags & (awgk::TONE_AMP_RAMP | awgk::TONE_AMP_MINJERK)) | c.flags;
  }
  h->flagged_ok = false;
  // only the records that changed go to the device (the whole chirp array if it had to grow)
  std::sort(changed_tones.begin(), changed_tones.end());
  std::sort(changed_slots.begin(), changed_slots.end());
  changed_slots.erase(std::unique(changed_slots.begin(), changed_slots.end()), changed_slots.end());
  bool any_exact = false;
  for (const ChirpRec& c : h->chirps) any_exact |= (c.tone >= 0 && (c.flags & awgk::TONE_EXACT));
  if (h->chirps.size() > h->cap_chirps) {
    // a larger slot pool: synchronous (reallocation waits for the device anyway)
    if ((st = wait_idle(h))) return st;
    if ((st = upload_chirps(h))) return st;
    if ((st = build_exact_tables(h))) return st;
    if (any_exact) return upload_tones(h);   // table offsets may have moved for any exact tone
    return upload_runs(h->d_tones, h->tones, changed_tones, "upload tones");
  }
  // steady state: the copies (and the exact tables' kernels) run on the private stream after the
  // renders issued so far, and later renders wait for them, so this call does not wait for the
  // device.  Staged: chirp records, then the tone records (all of them when an exact table's
  // offset may have moved).
  const size_t tone_bytes = (any_exact ? h->tones.size() : changed_tones.size()) * sizeof(ToneRec);
  if ((st = stage_begin(h, changed_slots.size() * sizeof(ChirpRec) + tone_bytes))) return st;
  size_t off = 0;
  if ((st = stage_runs(h, h->d_chirps, h->chirps, changed_slots, &off))) return st;
  if ((st = build_exact_tables(h, false))) return st;
  if (any_exact) {
    std::vector<int32_t> all(h->tones.size());
    for (size_t k = 0; k < all.size(); ++k) all[k] = (int32_t)k;
    if ((st = stage_runs(h, h->d_tones, h->tones, all, &off))) return st;
  } else if ((st = stage_runs(h, h->d_tones, h->tones, changed_tones, &off))) {
    return st;
  }
  return stage_end(h);
}

int awg_set_amp_ramps(awg_t* h, const int32_t* tone, const double* amp_end, const double* duration_s,
                      const int32_t* profile, const int64_t* start_sample, int32_t n) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0) return fail(AWG_EINVAL, "ramp count must be >= 0");
  if (n == 0) return AWG_OK;
  if (!tone || !amp_end || !duration_s || !profile || !start_sample) return fail(AWG_EINVAL, "null ramp array");
  std::vector<char> seen((size_t)h->K, 0);
  std::vector<int64_t> L((size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    const int32_t k = tone[i];
    if (k < 0 || k >= h->K) return fail(AWG_EINVAL, "ramp tone index out of range");
    if (seen[(size_t)k]) return fail(AWG_EINVAL, "two ramps for one tone in one call");
    seen[(size_t)k] = 1;
    if (!is_fin(amp_end[i]) || std::fabs(amp_end[i]) > 3.0e38) return fail(AWG_EINVAL, "ramp amplitude must be finite");
    int st = chirp_length_impl(duration_s[i], h->fs, &L[(size_t)i]);
    if (st) return st;
    if (profile[i] != AWG_PROFILE_LINEAR && profile[i] != AWG_PROFILE_MINJERK) return fail(AWG_EINVAL, "unknown ramp profile");
    if (start_sample[i] < h->cursor) return fail(AWG_EINVAL, "ramp starts before the render cursor");
    if (start_sample[i] > INT64_MAX / 2) return fail(AWG_EINVAL, "ramp start too large");
    const ToneRec& t = h->tones[(size_t)k];
    if ((t.flags & awgk::TONE_AMP_RAMP) && t.a_ns + t.a_L >= h->cursor)
      return fail(AWG_EINVAL, "tone already has a ramp that has not finished rendering");
  }
  int st = wait_idle(h);
  if (st) return st;
  h->periodic_start = -1;
  std::vector<int32_t> changed;
  for (int32_t i = 0; i < n; ++i) {
    ToneRec& t = h->tones[(size_t)tone[i]];
    if (t.flags & awgk::TONE_AMP_RAMP) t.A = t.A_end;   // fold the finished ramp
    h->flagged_ok = false;
    t.a_ns = start_sample[i];
    t.a_L = (int32_t)L[(size_t)i];
    t.A_end = (float)amp_end[i];
    t.flags = (t.flags & ~(awgk::TONE_AMP_RAMP | awgk::TONE_AMP_MINJERK)) | awgk::TONE_AMP_RAMP |
              (profile[i] == AWG_PROFILE_MINJERK ? awgk::TONE_AMP_MINJERK : 0);
    changed.push_back(tone[i]);
  }
  std::sort(changed.begin(), changed.end());
  return upload_runs(h->d_tones, h->tones, changed, "upload tones");
}

int awg_set_full_scale(awg_t* h, double v) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (!is_fin(v)) return fail(AWG_EINVAL, "full scale must be finite");
  if (v <= 0) {
    h->fs_explicit = false;
    h->full_scale = default_full_scale(h);
  } else {
    h->fs_explicit = true;
    h->full_scale = v;
  }
  return AWG_OK;
}

double awg_full_scale(const awg_t* h) { return h ? h->full_scale : 0.0; }

double awg_sample_rate(const awg_t* h) { return h ? h->fs : 0.0; }

int awg_seek(awg_t* h, int64_t sample) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (sample < 0) return fail(AWG_EINVAL, "sample must be >= 0");
  h->cursor = sample;
  return AWG_OK;
}

int64_t awg_cursor(const awg_t* h) { return h ? h->cursor : -1; }

int awg_set_sine_mode(awg_t* h, int32_t mode) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (mode != AWG_SINE_SFU && mode != AWG_SINE_ROTATOR) return fail(AWG_EINVAL, "unknown sine mode");
  h->sine_mode = mode;
  return AWG_OK;
}

int32_t awg_sine_mode(const awg_t* h) { return h ? h->sine_mode : -1; }

int awg_set_static_engine(awg_t* h, int32_t engine) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (engine != AWG_STATIC_DIRECT && engine != AWG_STATIC_GEMM_BF16 && engine != AWG_STATIC_GEMM_FP16)
    return fail(AWG_EINVAL, "unknown static engine");
  h->static_engine = engine;
  return AWG_OK;
}

int32_t awg_static_engine(const awg_t* h) { return h ? h->static_engine : -1; }

int awg_set_periodic(awg_t* h, int32_t log2_len, int32_t method, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (log2_len < 12 || log2_len > 30) return fail(AWG_EINVAL, "log2_len must be 12..30");
  if (method != AWG_PERIODIC_DIRECT && method != AWG_PERIODIC_GEMM_BF16 && method != AWG_PERIODIC_GEMM_FP16)
    return fail(AWG_EINVAL, "unknown periodic method");
  if (method != AWG_PERIODIC_DIRECT && log2_len < 15) return fail(AWG_EINVAL, "the GEMM table needs log2_len >= 15");
  // the static state that follows every chirp, and where it starts
  const uint64_t grid_mask = (1ull << (64 - log2_len)) - 1;
  int64_t start = h->cursor;
  std::vector<ToneRec> view(h->tones.size());
  for (size_t k = 0; k < h->tones.size(); ++k) {
    const ToneRec& t = h->tones[k];
    ToneRec v;
    std::memset(&v, 0, sizeof(v));
    const bool chirped = t.slot >= 0;
    v.phi_ref = chirped ? t.phi_post_ref : t.phi_ref;
    v.F = chirped ? t.F_end : t.F;
    v.rot_c = chirped ? t.rot_c_end : t.rot_c;
    v.rot_s = chirped ? t.rot_s_end : t.rot_s;
    v.n_s = awgk::NO_CHIRP;
    v.n_e = awgk::NO_CHIRP;
    const bool ramped = (t.flags & awgk::TONE_AMP_RAMP) != 0;
    v.A = ramped ? t.A_end : t.A;
    v.slot = -1;
    if (ramped) start = std::max(start, ((t.a_ns + t.a_L) / awgk::TILE + 1) * awgk::TILE);
    if (v.F & grid_mask) return fail(AWG_EINVAL, "a tone's final frequency is not on the f_s / 2^log2_len grid");
    // from the first whole tile after the chirp the render takes the static path, so replayed
    // samples equal rendered ones bit for bit in either sine mode
    if (chirped) start = std::max(start, (t.n_e / awgk::TILE + 1) * awgk::TILE);
    view[k] = v;
  }
  const int64_t N = (int64_t)1 << log2_len;
  int st = ensure(&h->d_periodic, &h->cap_periodic, (size_t)N, h, "periodic table");
  if (st) return st;
  awg_t* tmp = awg_create(h->fs);
  if (!tmp) return AWG_ENOMEM;
  tmp->tones = view;
  tmp->amp = h->amp;
  tmp->K = h->K;
  tmp->split = h->split;
  tmp->sine_mode = h->sine_mode;
  tmp->static_engine = h->static_engine;
  tmp->full_scale = h->full_scale;
  tmp->fs_explicit = true;
  st = upload_tones(tmp);
  if (!st) st = upload_chirps(tmp);
  if (!st) {
    if (method == AWG_PERIODIC_DIRECT)
      st = render_impl(tmp, N, nullptr, h->d_periodic, stream);
    else
      st = awg_table_gemm(tmp, log2_len, method == AWG_PERIODIC_GEMM_FP16 ? AWG_PREC_FP16 : AWG_PREC_BF16,
                          h->d_periodic, nullptr, stream);
  }
  if (!st) {
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(e, "periodic table");
  }
  awg_destroy(tmp);
  if (st) return st;
  h->periodic_log2 = log2_len;
  h->periodic_start = start;
  return AWG_OK;
}

int64_t awg_periodic_start(const awg_t* h) { return h ? h->periodic_start : -1; }

int awg_clear_periodic(awg_t* h) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  h->periodic_start = -1;
  return AWG_OK;
}

int awg_render(awg_t* h, int64_t n, int16_t* out, void* stream) {
  if (n > 0 && !out) return fail(AWG_EINVAL, "null output");
  return render_impl(h, n, nullptr, out, stream);
}

int awg_render_multiplexed(awg_t* const* handles, int32_t n_channels, int64_t n, int16_t* out, void* stream) {
  if (!handles || n_channels < 1 || n_channels > 8) return fail(AWG_EINVAL, "need 1..8 channel handles");
  if (n < 0) return fail(AWG_EINVAL, "sample count must be >= 0");
  if (n == 0) return AWG_OK;
  if (!out) return fail(AWG_EINVAL, "null output");
  int64_t cursors[8];
  for (int32_t c = 0; c < n_channels; ++c) {
    const awg_t* h = handles[c];
    if (!h) return fail(AWG_EINVAL, "null channel handle");
    for (int32_t d = 0; d < c; ++d)
      if (handles[d] == h) return fail(AWG_EINVAL, "a handle appears in two channels");
    if (h->fs != handles[0]->fs) return fail(AWG_EINVAL, "channels must share one sample rate");
    if (h->device != handles[0]->device) return fail(AWG_EINVAL, "channels must be on one device");
    if (h->cursor > INT64_MAX - n) return fail(AWG_EINVAL, "sample index overflow");
    cursors[c] = h->cursor;
  }
  for (int32_t c = 0; c < n_channels; ++c) {
    const int st = render_impl(handles[c], n, nullptr, out + c, stream, n_channels);
    if (st) {
      for (int32_t d = 0; d < c; ++d) handles[d]->cursor = cursors[d];
      return st;
    }
  }
  return AWG_OK;
}

int awg_render_f32(awg_t* h, int64_t n, float* out_f32, int16_t* out_q, void* stream) {
  if (n > 0 && !out_f32) return fail(AWG_EINVAL, "null output");
  return render_impl(h, n, out_f32, out_q, stream);
}

int awg_render_chunks(awg_t* h, int64_t chunk, int32_t n_chunks, int16_t* out, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (chunk < 1 || n_chunks < 0) return fail(AWG_EINVAL, "chunk must be >= 1 and n_chunks >= 0");
  if (n_chunks == 0) return AWG_OK;
  if (!out) return fail(AWG_EINVAL, "null output");
  if (chunk > (INT64_MAX - h->cursor) / n_chunks) return fail(AWG_EINVAL, "sample index overflow");
  if (chunk / awgk::TILE + 2 > (int64_t)(INT32_MAX / awgk::MAX_SPLIT)) return fail(AWG_EINVAL, "chunk too long");
  if (n_chunks == 1 || h->periodic_start >= 0 || h->static_engine != AWG_STATIC_DIRECT ||
      (h->split > 1 && chunk / awgk::TILE + 2 > SPLIT_LAUNCH_TILES)) {
    // a periodic tail is replayed per chunk; chunks above SPLIT_LAUNCH_TILES tiles go out in
    // several launches each (a pipelined sequence records its profiling events itself)
    for (int32_t c = 0; c < n_chunks; ++c) {
      const int st = render_impl(h, chunk, nullptr, out + (size_t)c * (size_t)chunk, stream);
      if (st) return st;
    }
    return AWG_OK;
  }
  return render_chunks_impl(h, chunk, n_chunks, out, (cudaStream_t)stream);
}

int64_t awg_launch_count(const awg_t* h) { return h ? h->n_launches : -1; }

int awg_render_stream(awg_t* h, int64_t n, int64_t chunk, int16_t* out, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (chunk < 1 || n < 0) return fail(AWG_EINVAL, "chunk must be >= 1 and n >= 0");
  if (n == 0) return AWG_OK;
  if (!out) return fail(AWG_EINVAL, "null output");
  if (h->cursor > INT64_MAX - n) return fail(AWG_EINVAL, "sample index overflow");
  if (chunk / awgk::TILE + 2 > (int64_t)(INT32_MAX / awgk::MAX_SPLIT)) return fail(AWG_EINVAL, "chunk too long");
  if (n / chunk > (int64_t)INT32_MAX - 1) return fail(AWG_EINVAL, "too many chunks");
  const int32_t full = (int32_t)(n / chunk);
  const int64_t tail = n - (int64_t)full * chunk;
  if (full + (tail > 0 ? 1 : 0) <= 1 || h->periodic_start >= 0 || h->static_engine != AWG_STATIC_DIRECT ||
      (h->split > 1 && chunk / awgk::TILE + 2 > SPLIT_LAUNCH_TILES)) {
    for (int64_t c = 0; c < n; c += chunk) {
      const int st = render_impl(h, std::min(chunk, n - c), nullptr, out + c, stream);
      if (st) return st;
    }
    return AWG_OK;
  }
  return render_chunks_impl(h, chunk, full, out, (cudaStream_t)stream, tail);
}

int awg_phase_words(awg_t* h, int64_t sample, uint64_t* out_host, int32_t n) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0 || n > h->K) return fail(AWG_EINVAL, "tone count out of range");
  if (sample < 0) return fail(AWG_EINVAL, "sample must be >= 0");
  if (n == 0) return AWG_OK;
  if (!out_host) return fail(AWG_EINVAL, "null output");
  int st = ensure(&h->d_words, &h->cap_words, (size_t)n, h, "phase words");
  if (st) return st;
  awgk::PhaseArgs pa;
  pa.tones = h->d_tones;
  pa.chirps = h->d_chirps;
  pa.n = n;
  pa.sample = sample;
  pa.out = h->d_words;
  std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
  cudaError_t e = counted(h, awgk::launch_phase_words(pa, h->priv));
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, h->d_words, (size_t)n * 8, cudaMemcpyDeviceToHost, h->priv);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->priv);
  if (e != cudaSuccess) return cuda_fail(e, "phase words");
  return AWG_OK;
}

int awg_render_phases(awg_t* h, int32_t tone, int64_t n0, int32_t count, uint32_t* out_host) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (tone < 0 || tone >= h->K) return fail(AWG_EINVAL, "tone index out of range");
  if (n0 < 0 || count < 0 || count > (1 << 20)) return fail(AWG_EINVAL, "bad sample range");
  if (count == 0) return AWG_OK;
  if (!out_host) return fail(AWG_EINVAL, "null output");
  int st = wait_idle(h);
  if (st) return st;
  const int64_t tile0 = n0 / awgk::TILE, tile_last = (n0 + count - 1) / awgk::TILE;
  const int32_t n_tiles = (int32_t)(tile_last - tile0 + 1);
  const ToneRec& t = h->tones[(size_t)tone];
  st = ensure(&h->d_recs, &h->cap_recs, (size_t)n_tiles, h, "tile records");
  if (st) return st;
  st = ensure(&h->d_trace, &h->cap_trace, (size_t)count, h, "trace");
  if (st) return st;
  cudaError_t e = cudaSuccess;
  if (t.slot >= 0 && !(t.flags & awgk::TONE_EXACT)) {
    awgk::PrepArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.chirps = h->d_chirps;
    pa.recs = h->d_recs;
    pa.act_of_slot = h->d_act;
    pa.tile0 = tile0;
    pa.n_tiles = n_tiles;
    pa.n_active = 1;
    pa.act_base = 0;
    std::memcpy(pa.W, h->W, sizeof(pa.W));
    std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
    pa.slots[0] = t.slot;
    e = counted(h, awgk::launch_prep(pa, h->priv));
  }
  awgk::TraceArgs ta;
  ta.tones = h->d_tones;
  ta.chirps = h->d_chirps;
  ta.recs = h->d_recs;
  ta.act_of_slot = h->d_act;
  ta.tone = tone;
  ta.n0 = n0;
  ta.count = count;
  ta.tile0 = tile0;
  ta.n_tiles = n_tiles;
  ta.K = h->K;
  ta.split = h->split;
  ta.listed = h->static_engine != AWG_STATIC_DIRECT;
  ta.out = h->d_trace;
  std::memcpy(ta.inv_odd, h->inv_odd, sizeof(ta.inv_odd));
  if (e == cudaSuccess) e = counted(h, awgk::launch_trace(ta, h->priv));
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, h->d_trace, (size_t)count * 4, cudaMemcpyDeviceToHost, h->priv);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->priv);
  if (e != cudaSuccess) return cuda_fail(e, "render phases");
  return AWG_OK;
}

int32_t awg_tone_split(const awg_t* h) { return h ? h->split : 0; }

float awg_last_render_ms(awg_t* h) {
  if (!h || !h->timed) return -1.f;
  float ms = -1.f;
  if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess) return -1.f;
  return ms;
}

int awg_table_gemm(awg_t* h, int32_t log2_len, int32_t precision, int16_t* out_q, float* out_f, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (log2_len < 15 || log2_len > 30) return fail(AWG_EINVAL, "log2_len must be 15..30");
  if (precision != AWG_PREC_BF16 && precision != AWG_PREC_FP16) return fail(AWG_EINVAL, "unknown precision");
  if (!out_q && !out_f) return fail(AWG_EINVAL, "no output buffer");
  const uint64_t grid_mask = (log2_len >= 64) ? 0 : ((1ull << (64 - log2_len)) - 1);
  for (const ToneRec& t : h->tones) {
    if (t.slot >= 0) return fail(AWG_EINVAL, "table GEMM needs static tones (a tone holds a chirp)");
    if (t.flags & awgk::TONE_AMP_RAMP) return fail(AWG_EINVAL, "table GEMM needs constant amplitudes (a tone holds a ramp)");
    if (t.F & grid_mask) return fail(AWG_EINVAL, "table GEMM needs every tone on the f_s / 2^log2_len grid");
  }
  const int64_t M = (int64_t)1 << (log2_len - 8);
  const size_t Kp = awgk::table_kp(std::max(h->K, 1));
  const size_t b_elems = (size_t)256 * Kp;
  int st = ensure(&h->d_gemm, &h->cap_gemm, 2 * b_elems, h, "table GEMM operands");
  if (st) return st;
  awgk::TableArgs2 t;
  std::memset(&t, 0, sizeof(t));   // every field not set below is 0 (a periodic table's K split is free)
  t.tones = h->d_tones;
  t.K = h->K;
  t.M = M;
  t.nb_log2 = 8;
  t.precision = precision;
  t.b_hi = h->d_gemm;
  t.b_lo = h->d_gemm + b_elems;
  t.row_base = 0;
  t.win_start = 0;
  t.win_end = (int64_t)M * 256;
  t.window_mode = 0;
  t.out_q = out_q;
  t.out_f = out_f;
  t.scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
  t.a_scale = awgk::table_amp_scale(max_amplitude(h));
  t.status = h->d_status;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t pe[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  if (h->profiling) {   // operand preparation and GEMM timed like a render's set-up and render
    while (e == cudaSuccess && h->prof_ev.size() < 4 * (h->prof_calls + 1)) {
      cudaEvent_t ev;
      e = cudaEventCreate(&ev);
      if (e == cudaSuccess) h->prof_ev.push_back(ev);
    }
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) pe[i] = h->prof_ev[4 * h->prof_calls + (size_t)i];
  }
  if (e == cudaSuccess) e = order_after_uploads(h, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess && pe[0]) e = cudaEventRecord(pe[0], s);
  if (e == cudaSuccess) e = counted(h, awgk::launch_table_prep(t, s));
  if (e == cudaSuccess && pe[1]) e = cudaEventRecord(pe[1], s);
  if (e == cudaSuccess && pe[2]) e = cudaEventRecord(pe[2], s);
  if (e == cudaSuccess) e = counted(h, awgk::launch_table_gemm(t, s));
  if (e == cudaSuccess && pe[3]) e = cudaEventRecord(pe[3], s);
  if (e == cudaSuccess && pe[3]) {
    ++h->prof_calls;
    h->prof_launches += 3;
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_done, s);
  if (e != cudaSuccess) return cuda_fail(e, "table GEMM");
  h->timed = true;
  h->have_done = true;
  return AWG_OK;
}

int awg_render_noalloc(awg_t* h, int64_t n, int16_t* out, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (n < 0) return fail(AWG_EINVAL, "sample count must be >= 0");
  if (n == 0) return AWG_OK;
  if (!out) return fail(AWG_EINVAL, "null output");
  if (h->cursor > INT64_MAX - n) return fail(AWG_EINVAL, "sample index overflow");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != h->device) return fail(AWG_EINVAL, "call on the device the handle was created on");
  TileRec* recs = nullptr;
  int32_t* act = nullptr;
  if ((e = awgk::noalloc_scratch(cur, &recs, &act)) != cudaSuccess) return cuda_fail(e, "fixed scratch lookup");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t c = h->cursor;
  const int64_t tile0 = c / awgk::TILE;
  const int64_t tile_last = (c + n - 1) / awgk::TILE;
  const int64_t n_tiles = tile_last - tile0 + 1;
  if (n_tiles > (int64_t)(INT32_MAX / awgk::MAX_SPLIT)) return fail(AWG_EINVAL, "render window too long");
  const int64_t span0 = tile0 * awgk::TILE, span1 = (tile_last + 1) * awgk::TILE - 1;
  auto is_active = [&](const ChirpRec& cr) {
    return cr.tone >= 0 && !(cr.flags & awgk::TONE_EXACT) && cr.n_s <= span1 && cr.n_s + cr.L >= span0;
  };
  int64_t n_active = 0;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    if (!is_active(h->chirps[sl])) continue;
    if ((int64_t)sl >= awgk::NOALLOC_MAX_SLOTS)
      return fail(AWG_ENOMEM, "chirp slot index beyond the fixed scratch's slot map (AWG_NOALLOC_MAX_SLOTS)");
    ++n_active;
  }
  if (n_active * n_tiles > (int64_t)awgk::NOALLOC_MAX_RECORDS)
    return fail(AWG_ENOMEM, "window needs " + std::to_string(n_active * n_tiles) +
                                " chirp tile records; the fixed scratch holds " +
                                std::to_string(awgk::NOALLOC_MAX_RECORDS) + " (AWG_NOALLOC_MAX_RECORDS)");
  if ((e = order_after_uploads(h, s)) != cudaSuccess) return cuda_fail(e, "upload ordering");
  if ((e = cudaEventRecord(h->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
  awgk::PrepArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.chirps = h->d_chirps;
  pa.recs = recs;
  pa.act_of_slot = act;
  pa.tile0 = tile0;
  pa.n_tiles = (int32_t)n_tiles;
  std::memcpy(pa.W, h->W, sizeof(pa.W));
  std::memcpy(pa.inv_odd, h->inv_odd, sizeof(pa.inv_odd));
  int32_t batch_base = 0;
  for (size_t sl = 0; sl < h->chirps.size(); ++sl) {
    if (!is_active(h->chirps[sl])) continue;
    pa.slots[pa.n_active++] = (int32_t)sl;
    if (pa.n_active == awgk::MAX_ACTIVE_PER_LAUNCH) {
      pa.act_base = batch_base;
      if ((e = counted(h, awgk::launch_prep(pa, s))) != cudaSuccess) return cuda_fail(e, "prep launch");
      batch_base += pa.n_active;
      pa.n_active = 0;
    }
  }
  if (pa.n_active > 0) {
    pa.act_base = batch_base;
    if ((e = counted(h, awgk::launch_prep(pa, s))) != cudaSuccess) return cuda_fail(e, "prep launch");
  }
  awgk::RenderArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.tones = h->d_tones;
  ra.exact_tab = h->d_tab;
  ra.chirps = h->d_chirps;
  ra.recs = recs;
  ra.act_of_slot = act;
  ra.K = h->K;
  ra.split = h->split;
  ra.sine_mode = h->sine_mode;
  ra.tile0 = tile0;
  ra.n_tiles = (int32_t)n_tiles;
  ra.win_start = c;
  ra.win_end = c + n;
  ra.out_q = out;
  ra.out_f = nullptr;
  ra.scale = h->full_scale > 0 ? (float)(32767.0 / h->full_scale) : 0.f;
  ra.status = h->d_status;
  std::memcpy(ra.inv_odd, h->inv_odd, sizeof(ra.inv_odd));
  if ((e = counted(h, awgk::launch_render(ra, s))) != cudaSuccess) return cuda_fail(e, "render launch");
  if ((e = cudaEventRecord(h->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
  if ((e = cudaEventRecord(h->ev_done, s)) != cudaSuccess) return cuda_fail(e, "event");
  h->timed = true;
  h->have_done = true;
  h->cursor = c + n;
  return AWG_OK;
}

int awg_profile_begin(awg_t* h) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  h->profiling = true;
  h->prof_calls = 0;
  h->prof_launches = 0;
  return AWG_OK;
}

int awg_profile_end(awg_t* h, float* prep_ms, float* render_ms, int32_t cap, int64_t* launches) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (!h->profiling) return fail(AWG_ESTATE, "profiling was not started");
  h->profiling = false;
  if (launches) *launches = h->prof_launches;
  const size_t n = h->prof_calls;
  if (n == 0) return 0;
  cudaError_t e = cudaEventSynchronize(h->prof_ev[4 * (n - 1) + 3]);
  if (e != cudaSuccess) return cuda_fail(e, "profiling sync");
  for (size_t i = 0; i < n && (int64_t)i < (int64_t)cap; ++i) {
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, h->prof_ev[4 * i], h->prof_ev[4 * i + 1]);
    cudaEventElapsedTime(&b, h->prof_ev[4 * i + 2], h->prof_ev[4 * i + 3]);
    if (prep_ms) prep_ms[i] = a;
    if (render_ms) render_ms[i] = b;
  }
  return (int)std::min<size_t>(n, (size_t)INT32_MAX);
}

int awg_test_wait_timeout(awg_t* h, int64_t limit_us, void* stream) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  if (limit_us < 1 || limit_us > 10000000) return fail(AWG_EINVAL, "limit_us must be in 1 .. 10^7");
  int st = ensure_seq_counter(h);
  if (st) return st;
  // one above the running total of every sequence issued so far: no render CTA brings the counter
  // there, so the wait runs out
  cudaError_t e = counted(h, awgk::launch_join(h->d_seq_exit, h->seq_exit_target + 1, h->d_status,
                                               (uint64_t)limit_us * 1000ull, (cudaStream_t)stream));
  if (e != cudaSuccess) return cuda_fail(e, "join launch");
  return AWG_OK;
}

int awg_sfu_rate_probe(float* out, int32_t blocks, int32_t runs, void* stream) {
  if (!out) return fail(AWG_EINVAL, "null output");
  if (blocks < 1 || blocks > (1 << 20)) return fail(AWG_EINVAL, "blocks must be in 1 .. 2^20");
  if (runs < 1 || runs > (1 << 20)) return fail(AWG_EINVAL, "runs must be in 1 .. 2^20");
  cudaError_t e = awgk::launch_sfu_rate(out, blocks, runs, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "probe launch");
  return AWG_OK;
}

int awg_chirp_rate_probe(float* out, int32_t blocks, int32_t runs, void* stream) {
  if (!out) return fail(AWG_EINVAL, "null output");
  if (blocks < 1 || blocks > (1 << 20)) return fail(AWG_EINVAL, "blocks must be in 1 .. 2^20");
  if (runs < 1 || runs > (1 << 20)) return fail(AWG_EINVAL, "runs must be in 1 .. 2^20");
  cudaError_t e = awgk::launch_chirp_rate(out, blocks, runs, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "probe launch");
  return AWG_OK;
}

int awg_device_status(awg_t* h) {
  if (!h) return fail(AWG_EINVAL, "null handle");
  int32_t v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "device status");
  return v;
}

}  // extern "C"
