/*
 * awg_oracle.c -- CPU oracle for multi-tone additive synthesis (TEST INFRASTRUCTURE ONLY).
 *
 * This file is the plain, slow reference that the CUDA library is checked against.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, includes or calls it, and it shares no code with the library.
 *
 * What it computes (paper: Tu & Subhankar, "Fast real-time arbitrary waveform generation using
 * graphic processing units"):
 *   x[n] = sum_k A_k sin(phi_k(n))                       (Sec. II, Eq. main / Eq. static1 and the
 *                                                          dynamic form Eq. dynamicandstatic)
 * with phi_k(n) = 2*pi * Phi_k(n) / 2^64, where Phi_k(n) is an integer phase word:
 *   static tone:  Phi(n) = Phi_ref + n*F  (mod 2^64), stepped one sample at a time
 *                 (the modf() range reduction of the Appendix is implicit: the word wraps).
 *   chirp:        Phi(n_s + m) = Phi_start + top64( sum_k d_k C(m,k) )   for 0 <= m <= L,
 *                 produced by a cascade of seven 192-bit accumulators (a polynomial
 *                 direct-digital synthesiser).  d_k are the exact forward differences of the
 *                 chirp phase polynomial (Eq. freqchirp, case 1, and its linear analogue), scaled
 *                 by 2^128 and rounded; they are derived with exact rationals in oracle/__init__.py.
 *                 d_0 carries the rounding offset 2^127, so top64() rounds to nearest.
 *   exponential:  (has_chirp == 2) Phi(n_s + m) = Phi_start + R(m), R the integral of a frequency
 *                 that moves geometrically from F_start to F_end (see exp_offset).
 *   after chirp:  Phi(n) = Phi_end + (n - n_s - L) * F_end   (Eq. freqchirp, case 2),
 *                 Phi_end = Phi(n_s + L) from the cascade (or from R(L)).
 *   amplitude:    A_k, or a ramp a_k(n) from A_k to A_end (see amp_at) for a_j[i] of
 *                 Eq. dynamicandstatic.
 * Sine is libm sin() in FP64 of the signed turn u = (int64)Phi * 2^-64, the sum runs over
 * tones in ascending order in FP64, and quantisation is round-half-even with a symmetric clamp
 * at +-32767.
 *
 * The sequential cascade is the definition; the closed form sum_k d_k C(m,k) (mod 2^192) is
 * its exact skip, used to start a thread or a sampled evaluation in the middle of a chirp.
 * Both give the same integers; tests check that by brute force.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef struct { uint64_t w[3]; } u192; /* little-endian limbs, arithmetic mod 2^192 */

static u192 add192(u192 a, u192 b) {
  u192 r;
  u128 s = (u128)a.w[0] + b.w[0];
  r.w[0] = (uint64_t)s;
  s = (u128)a.w[1] + b.w[1] + (uint64_t)(s >> 64);
  r.w[1] = (uint64_t)s;
  r.w[2] = a.w[2] + b.w[2] + (uint64_t)(s >> 64);
  return r;
}

/* a*b mod 2^192, schoolbook on 64-bit limbs */
static u192 mul192(u192 a, u192 b) {
  u192 r = {{0, 0, 0}};
  for (int i = 0; i < 3; i++) {
    uint64_t carry = 0;
    for (int j = 0; i + j < 3; j++) {
      u128 t = (u128)a.w[i] * b.w[j] + r.w[i + j] + carry;
      r.w[i + j] = (uint64_t)t;
      carry = (uint64_t)(t >> 64);
    }
  }
  return r;
}

static u192 from_u64(uint64_t v) { u192 r = {{v, 0, 0}}; return r; }

/* exact division of a non-negative 192-bit value by a small positive integer */
static u192 div192_small(u192 a, uint64_t d) {
  u192 q;
  u128 rem = 0;
  for (int i = 2; i >= 0; i--) {
    u128 cur = (rem << 64) | a.w[i];
    q.w[i] = (uint64_t)(cur / d);
    rem = cur % d;
  }
  return q;
}

/* binomial C(m,k) for 0 <= m < 2^28, 0 <= k <= 6: the product of k consecutive integers is
 * below 2^168, so it is exact in 192 bits, and division by k! is exact. */
static u192 binom192(int64_t m, int k) {
  if (k == 0) return from_u64(1);
  if (m < k) return from_u64(0);
  u192 p = from_u64(1);
  uint64_t fact = 1;
  for (int i = 0; i < k; i++) {
    p = mul192(p, from_u64((uint64_t)(m - i)));
    fact *= (uint64_t)(i + 1);
  }
  return div192_small(p, fact);
}

/* Closed-form cascade state at chirp sample m: acc_k(m) = sum_{i>=k} d_i C(m, i-k). */
static void cascade_at(const uint64_t* d /*7x3*/, int64_t m, u192 acc[7]) {
  u192 c[7];
  for (int j = 0; j < 7; j++) c[j] = binom192(m, j);
  for (int k = 0; k < 7; k++) {
    u192 s = from_u64(0);
    for (int i = k; i < 7; i++) {
      u192 di = {{d[3 * i], d[3 * i + 1], d[3 * i + 2]}};
      s = add192(s, mul192(di, c[i - k]));
    }
    acc[k] = s;
  }
}

/* one sample step of the cascade: acc_k <- acc_k + acc_{k+1}, lowest order first */
static void cascade_step(u192 acc[7]) {
  for (int k = 0; k < 6; k++) acc[k] = add192(acc[k], acc[k + 1]);
}

/*
 * Exponential chirp (Sec. II names exponential chirps beside the minimum-jerk one but prints no
 * formula).  Reading: the instantaneous frequency moves geometrically, F(t) = F_start r^(t/L)
 * words per sample with r = F_end / F_start (both > 0), and the phase offset is its integral
 *     R(m) = F_start L (r^(m/L) - 1) / ln r          (F_start m when r = 1),
 * rounded to the nearest word, mod 2^64.  Evaluated in long double (expm1l, logl): unlike the
 * polynomial chirps this is not an exact-integer definition; its error is a few 1e-10 turn at the
 * largest phases, far below any rendering tolerance.
 */
static uint64_t ld_to_word(long double R) {
  const long double two64 = 18446744073709551616.0L;
  long double r = fmodl(R, two64); /* exact; the sign of R */
  if (r < 0) r += two64;
  r = floorl(r + 0.5L);
  if (r >= two64) r -= two64;
  return (uint64_t)r;
}

/* Planted-mistake switch for the pin tests only (0: the definition above).  1: F_start and F_end
 * swapped; 2: m off by one; 3: exp instead of expm1 (a constant offset); 4: log2 instead of ln;
 * 5: L + 1 instead of L. */
int oracle_exp_plant = 0;

static uint64_t exp_offset(uint64_t F0, uint64_t F1, int64_t L, int64_t m) {
  if (F0 == F1) return (uint64_t)m * F0;
  if (oracle_exp_plant == 1) { uint64_t t = F0; F0 = F1; F1 = t; }
  if (oracle_exp_plant == 2) m += 1;
  if (oracle_exp_plant == 5) L += 1;
  long double lam = oracle_exp_plant == 4 ? log2l((long double)F1 / (long double)F0)
                                          : logl((long double)F1 / (long double)F0);
  long double e = oracle_exp_plant == 3 ? expl(lam * (long double)m / (long double)L)
                                        : expm1l(lam * (long double)m / (long double)L);
  long double R = (long double)F0 * (long double)L * e / lam;
  return ld_to_word(R);
}

typedef struct {
  uint64_t F, phi_ref;          /* static segment: Phi(n) = phi_ref + n F */
  double A;
  int32_t has_chirp;            /* 0 none, 1 polynomial (cascade), 2 exponential */
  int64_t n_s, L;               /* chirp covers samples n_s .. n_s+L (m = 0..L) */
  const uint64_t* d;            /* 7 x 3 limbs (exponential: d_0 = F_start, d_1 = F_end) */
  uint64_t phi_start, phi_end, F_end;
  int32_t has_ramp, ramp_prof;  /* amplitude ramp a_j[i] of Eq. dynamicandstatic (0: none) */
  int64_t a_ns, a_L;            /* the amplitude moves from A to A_end over samples a_ns .. a_ns+a_L */
  double A_end;
} tone_t;

/*
 * Amplitude a(n) of Eq. dynamicandstatic.  The paper leaves a_j[i] open; the ramp used here moves
 * from A to A_end along the same profiles as the frequency ramps: with tau = (n - a_ns)/a_L,
 * linear s(tau) = tau, minimum-jerk s(tau) = 10 tau^3 - 15 tau^4 + 6 tau^5 (the minimum-jerk
 * frequency trajectory whose integral is the phase of Eq. freqchirp); a = A + (A_end - A) s.
 * Before the ramp a = A, after it a = A_end.
 */
static double amp_at(const tone_t* t, int64_t n) {
  if (!t->has_ramp || n <= t->a_ns) return t->A;
  int64_t m = n - t->a_ns;
  if (m >= t->a_L) return t->A_end;
  double tau = (double)m / (double)t->a_L;
  double s = t->ramp_prof == 0 ? tau : tau * tau * tau * (10.0 - 15.0 * tau + 6.0 * tau * tau);
  return t->A + (t->A_end - t->A) * s;
}

/* Phase word at absolute sample n by the closed form (used to seed sequential runs). */
static uint64_t phase_closed(const tone_t* t, int64_t n) {
  if (!t->has_chirp || n < t->n_s) return t->phi_ref + (uint64_t)n * t->F;
  int64_t m = n - t->n_s;
  if (m > t->L) return t->phi_end + (uint64_t)(m - t->L) * t->F_end;
  if (t->has_chirp == 2) return t->phi_start + exp_offset(t->d[0], t->d[3], t->L, m);
  u192 acc[7];
  cascade_at(t->d, m, acc);
  return t->phi_start + acc[0].w[2];
}

/* Sequential generator over a contiguous sample range. */
typedef struct {
  const tone_t* t;
  int64_t n;        /* next absolute sample */
  uint64_t phi;     /* static / post phase word at n */
  u192 acc[7];      /* chirp cascade at n (valid when in chirp segment) */
  int seg;          /* 0 = before chirp / static, 1 = chirp, 2 = after chirp */
} gen_t;

static void gen_init(gen_t* g, const tone_t* t, int64_t n) {
  g->t = t;
  g->n = n;
  if (!t->has_chirp || n < t->n_s) {
    g->seg = 0;
    g->phi = t->phi_ref + (uint64_t)n * t->F;
  } else if (n - t->n_s > t->L) {
    g->seg = 2;
    g->phi = t->phi_end + (uint64_t)(n - t->n_s - t->L) * t->F_end;
  } else {
    g->seg = 1;
    if (t->has_chirp == 1) cascade_at(t->d, n - t->n_s, g->acc);
  }
}

static uint64_t gen_phase(const gen_t* g) {
  if (g->seg == 1 && g->t->has_chirp == 2) return phase_closed(g->t, g->n);   /* no recurrence */
  return g->seg == 1 ? g->t->phi_start + g->acc[0].w[2] : g->phi;
}

static void gen_advance(gen_t* g) {
  const tone_t* t = g->t;
  int64_t next = g->n + 1;
  if (g->seg == 0) {
    if (t->has_chirp && next == t->n_s) {
      g->seg = 1;
      if (t->has_chirp == 1) cascade_at(t->d, 0, g->acc);
    } else {
      g->phi += t->F;
    }
  } else if (g->seg == 1) {
    if (next - t->n_s > t->L) {
      g->seg = 2;
      g->phi = t->phi_end + t->F_end; /* one sample past the chirp end */
    } else if (t->has_chirp == 1) {
      cascade_step(g->acc);
    }
  } else {
    g->phi += t->F_end;
  }
  g->n = next;
}

static double word_sin(uint64_t phi) {
  /* signed turn in [-1/2, 1/2) */
  double u = ldexp((double)(int64_t)phi, -64);
  return sin(2.0 * M_PI * u);
}

static void build_tones(int K, const uint64_t* F, const uint64_t* phi_ref, const double* A,
                        const int32_t* has_chirp, const int64_t* n_s, const int64_t* L,
                        const uint64_t* d, const uint64_t* F_end, tone_t* tones) {
  for (int k = 0; k < K; k++) {
    tone_t* t = &tones[k];
    t->has_ramp = 0;
    t->ramp_prof = 0;
    t->a_ns = t->a_L = 0;
    t->A_end = A[k];
    t->F = F[k];
    t->phi_ref = phi_ref[k];
    t->A = A[k];
    t->has_chirp = has_chirp[k];
    t->n_s = n_s[k];
    t->L = L[k];
    t->d = d + 21 * (size_t)k;
    t->F_end = F_end[k];
    t->phi_start = t->phi_ref + (uint64_t)t->n_s * t->F;
    if (t->has_chirp == 2) {
      t->phi_end = t->phi_start + exp_offset(t->d[0], t->d[3], t->L, t->L);
    } else if (t->has_chirp) {
      u192 acc[7];
      cascade_at(t->d, t->L, acc);
      t->phi_end = t->phi_start + acc[0].w[2];
    } else {
      t->phi_end = 0;
    }
  }
}

/* Amplitude ramps (ramp: K x {has_ramp, profile} int32 pairs; a_ns, a_L: int64; A_end: FP64). */
static void apply_ramps(int K, const int32_t* ramp, const int64_t* a_ns, const int64_t* a_L, const double* A_end,
                        tone_t* tones) {
  if (!ramp) return;
  for (int k = 0; k < K; k++) {
    tones[k].has_ramp = ramp[2 * k];
    tones[k].ramp_prof = ramp[2 * k + 1];
    tones[k].a_ns = a_ns[k];
    tones[k].a_L = a_L[k];
    tones[k].A_end = A_end[k];
  }
}

/* Amplitudes a(n) of one tone at samples n[0..N) (for tests). */
void oracle_amp_at(double A, int32_t profile, int64_t a_ns, int64_t a_L, double A_end, const int64_t* n,
                   int64_t N, double* out) {
  tone_t t;
  memset(&t, 0, sizeof(t));
  t.A = A;
  t.has_ramp = 1;
  t.ramp_prof = profile;
  t.a_ns = a_ns;
  t.a_L = a_L;
  t.A_end = A_end;
  for (int64_t i = 0; i < N; i++) out[i] = amp_at(&t, n[i]);
}

/* Post-chirp anchor Phi_end = Phi(n_s + L), for tests and for the host bookkeeping of tests. */
uint64_t oracle_chirp_end_word(uint64_t F, uint64_t phi_ref, int32_t has_chirp, int64_t n_s, int64_t L,
                               const uint64_t* d) {
  if (has_chirp == 2) return phi_ref + (uint64_t)n_s * F + exp_offset(d[0], d[3], L, L);
  u192 acc[7];
  cascade_at(d, L, acc);
  return phi_ref + (uint64_t)n_s * F + acc[0].w[2];
}

/* Phase words of one tone, sequentially, for samples n0 .. n0+N-1. */
void oracle_phase_words_seq(uint64_t F, uint64_t phi_ref, int32_t has_chirp, int64_t n_s,
                            int64_t L, const uint64_t* d, uint64_t F_end, int64_t n0, int64_t N,
                            uint64_t* out) {
  double A = 0.0;
  tone_t t;
  build_tones(1, &F, &phi_ref, &A, &has_chirp, &n_s, &L, d, &F_end, &t);
  gen_t g;
  gen_init(&g, &t, n0);
  for (int64_t i = 0; i < N; i++) {
    out[i] = gen_phase(&g);
    gen_advance(&g);
  }
}

/* Phase words of one tone at arbitrary samples, by the closed form. */
void oracle_phase_words_at(uint64_t F, uint64_t phi_ref, int32_t has_chirp, int64_t n_s,
                           int64_t L, const uint64_t* d, uint64_t F_end, const int64_t* n,
                           int64_t N, uint64_t* out) {
  double A = 0.0;
  tone_t t;
  build_tones(1, &F, &phi_ref, &A, &has_chirp, &n_s, &L, d, &F_end, &t);
  for (int64_t i = 0; i < N; i++) out[i] = phase_closed(&t, n[i]);
}

/* Closed-form cascade state of one chirp at sample m (7 x 3 limbs), for tests. */
void oracle_cascade_at(const uint64_t* d, int64_t m, uint64_t* out) {
  u192 acc[7];
  cascade_at(d, m, acc);
  for (int k = 0; k < 7; k++) memcpy(out + 3 * k, acc[k].w, 24);
}

/*
 * x[n] for n = n0 .. n0+N-1, FP64, tones summed in ascending order.  With nthreads > 1 the
 * sample range is cut into contiguous pieces; each piece seeds its generators by the closed
 * form and then steps sequentially.  Returns the number of threads used.
 */
int oracle_render(int K, const uint64_t* F, const uint64_t* phi_ref, const double* A,
                  const int32_t* has_chirp, const int64_t* n_s, const int64_t* L,
                  const uint64_t* d, const uint64_t* F_end, int64_t n0, int64_t N, double* out,
                  int nthreads, void* work /* K * sizeof(tone_t) + nthreads*K*sizeof(gen_t) */,
                  const int32_t* ramp, const int64_t* a_ns, const int64_t* a_L, const double* A_end) {
  tone_t* tones = (tone_t*)work;
  gen_t* gens = (gen_t*)((char*)work + (size_t)K * sizeof(tone_t));
  build_tones(K, F, phi_ref, A, has_chirp, n_s, L, d, F_end, tones);
  apply_ramps(K, ramp, a_ns, a_L, A_end, tones);
  if (nthreads < 1) nthreads = 1;
  int used = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
  {
    int tid = omp_get_thread_num();
    int nt = omp_get_num_threads();
#pragma omp single
    used = nt;
#else
  {
    int tid = 0, nt = 1;
#endif
    int64_t lo = N * tid / nt, hi = N * (tid + 1) / nt;
    gen_t* g = gens + (size_t)tid * K;
    if (hi > lo) {
      for (int k = 0; k < K; k++) gen_init(&g[k], &tones[k], n0 + lo);
      for (int64_t i = lo; i < hi; i++) {
        double x = 0.0;
        for (int k = 0; k < K; k++) {
          x += amp_at(&tones[k], n0 + i) * word_sin(gen_phase(&g[k]));
          gen_advance(&g[k]);
        }
        out[i] = x;
      }
    }
  }
  return used;
}

size_t oracle_render_work_bytes(int K, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  return (size_t)K * sizeof(tone_t) + (size_t)nthreads * K * sizeof(gen_t);
}

/* x[n] at arbitrary absolute samples, each by the closed form (for sampled parity at full size). */
void oracle_render_at(int K, const uint64_t* F, const uint64_t* phi_ref, const double* A,
                      const int32_t* has_chirp, const int64_t* n_s, const int64_t* L,
                      const uint64_t* d, const uint64_t* F_end, const int64_t* n, int64_t N,
                      double* out, int nthreads, void* work /* K * sizeof(tone_t) */,
                      const int32_t* ramp, const int64_t* a_ns, const int64_t* a_L, const double* A_end) {
  tone_t* tones = (tone_t*)work;
  build_tones(K, F, phi_ref, A, has_chirp, n_s, L, d, F_end, tones);
  apply_ramps(K, ramp, a_ns, a_L, A_end, tones);
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 4)
#endif
  for (int64_t i = 0; i < N; i++) {
    double x = 0.0;
    for (int k = 0; k < K; k++) x += amp_at(&tones[k], n[i]) * word_sin(phase_closed(&tones[k], n[i]));
    out[i] = x;
  }
}

/* q = clamp(rint(x * (32767 / FS)), -32767, 32767), round half to even (default FP mode). */
void oracle_quantize(const double* x, int64_t N, double FS, int16_t* out) {
  double scale = 32767.0 / FS;
  for (int64_t i = 0; i < N; i++) {
    double q = rint(x[i] * scale);
    if (q > 32767.0) q = 32767.0;
    if (q < -32767.0) q = -32767.0;
    out[i] = (int16_t)q;
  }
}
