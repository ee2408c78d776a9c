// Render kernels for multi-tone additive synthesis on sm_103a.
//
//   x[n] = sum_k A_k sin(2 pi Phi_k(n) / 2^64)       (Eq. main / Eq. dynamicandstatic)
//
// Phase words.  Static tones: Phi(n) = phi_ref + n F.  Chirps (Eq. freqchirp, linear or
// minimum-jerk): Phi(n_s + m) = Phi(n_s) + top64(sum_k d_k C(m,k)) with the 192-bit forward
// differences d_k set up on the host; evaluated here exactly by the closed form
// (exact_chirp_word), which is what a sequential 192-bit cascade would produce.  Exponential
// chirps: Phi(n_s) + C (e^(alpha m) - 1) in FP64.
//
// Work decomposition (see awg_internal.h): a CTA renders one tile of TILE = 4096 absolute-aligned
// samples; thread j owns the run of RUN = 32 samples starting at T0 + 32 j and keeps its 32 partial
// sums in registers; the tones are split over `split` CTAs, whose partial tiles are added in rank
// order (through L2 scratch by the last CTA of the tile to finish, or through distributed shared
// memory in a thread-block cluster), then scaled, rounded and stored by the same kernel.
//
// Per (tone, run) the phase is set up once and then stepped per sample in 32-bit fixed point
// (units of 2^-32 turn):
//   static runs   p_r = p_0 + r f                                  (p_0 from the exact word)
//   chirp runs    p_r = p_0 + r f + C(r,2) g + C(r,3) h            (32-bit difference cascade)
// where (p_0, f, g, h) come from a per-(chirp, tile) record of stride-32 forward differences
// (prep_kernel) evaluated at the run index j.  The sine takes the top 23 bits of p_r as a
// signed fraction of a turn (round to nearest) and runs on the SFU (__sinf in [-pi, pi)).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "awg_internal.h"

namespace cg = cooperative_groups;

namespace awgk {

namespace {

constexpr int STATUS_TIMEOUT = -4;   // AWG_ETIMEOUT

// ------------------------------------------------------------------------------------------
// 192-bit integers, arithmetic mod 2^192 (two's complement for signed values)
// ------------------------------------------------------------------------------------------
struct U192 {
  uint64_t w0, w1, w2;
};

__device__ __forceinline__ U192 from_s64(int64_t a) {
  uint64_t s = (uint64_t)(a >> 63);
  return {(uint64_t)a, s, s};
}

__device__ __forceinline__ U192 add192(U192 a, U192 b) {
  U192 r;
  unsigned __int128 t = (unsigned __int128)a.w0 + b.w0;
  r.w0 = (uint64_t)t;
  t = (unsigned __int128)a.w1 + b.w1 + (uint64_t)(t >> 64);
  r.w1 = (uint64_t)t;
  r.w2 = a.w2 + b.w2 + (uint64_t)(t >> 64);
  return r;
}

__device__ __forceinline__ U192 mul192(U192 a, U192 b) {
  unsigned __int128 p00 = (unsigned __int128)a.w0 * b.w0;
  unsigned __int128 p01 = (unsigned __int128)a.w0 * b.w1;
  unsigned __int128 p10 = (unsigned __int128)a.w1 * b.w0;
  unsigned __int128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  U192 r;
  r.w0 = (uint64_t)p00;
  r.w1 = (uint64_t)mid;
  r.w2 = (uint64_t)(mid >> 64) + (uint64_t)(p01 >> 64) + (uint64_t)(p10 >> 64) + a.w0 * b.w2 +
         a.w1 * b.w1 + a.w2 * b.w0;
  return r;
}

__device__ __forceinline__ U192 sar192(U192 a, int v) {
  if (v == 0) return a;
  U192 r;
  r.w0 = (a.w0 >> v) | (a.w1 << (64 - v));
  r.w1 = (a.w1 >> v) | (a.w2 << (64 - v));
  r.w2 = (uint64_t)((int64_t)a.w2 >> v);
  return r;
}


// C(m, j) for j = 0..6 and signed m (|m| < 2^30): the product of j consecutive integers is
// below 2^180 in magnitude, so it is exact mod 2^192; dividing by j! = 2^v * odd is a
// multiplication by the inverse of the odd part mod 2^192 and an arithmetic shift.
__device__ __forceinline__ void binomials(int64_t m, const uint64_t (*inv)[3], U192 c[7]) {
  U192 p = {1, 0, 0};
  c[0] = p;
#pragma unroll
  for (int j = 1; j <= 6; ++j) {
    p = mul192(p, from_s64(m - (j - 1)));
    U192 q = p;
    if (j == 3 || j == 4) q = mul192(q, U192{inv[0][0], inv[0][1], inv[0][2]});   // 1/3
    if (j == 5) q = mul192(q, U192{inv[1][0], inv[1][1], inv[1][2]});              // 1/15
    if (j == 6) q = mul192(q, U192{inv[2][0], inv[2][1], inv[2][2]});              // 1/45
    const int v = (j == 2 || j == 3) ? 1 : (j == 4 || j == 5) ? 3 : (j == 6) ? 4 : 0;
    c[j] = sar192(q, v);
  }
}

__device__ __forceinline__ U192 dword(const ChirpRec& c, int i) {
  return U192{c.d[3 * i], c.d[3 * i + 1], c.d[3 * i + 2]};
}

// x 2^64 rounded to an integer, mod 2^128 (two's complement): the double's exact value M 2^e
// (M its 53-bit integer mantissa) shifted into Q64.64.  Zero for |x| < 2^-65.
__device__ __forceinline__ unsigned __int128 q64_of(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1075 + 64;
  unsigned __int128 v;
  if (sh >= 128) v = 0;
  else if (sh >= 0) v = (unsigned __int128)M << sh;
  else if (sh > -54) v = ((unsigned __int128)M + ((unsigned __int128)1 << (-sh - 1))) >> (-sh);
  else v = 0;
  return (b >> 63) ? (unsigned __int128)0 - v : v;
}

// Exponential chirp (TONE_EXP): the phase offset R(m) = C (e^(alpha m) - 1) words (the integral of
// the frequency F_start e^(alpha t)), FP64, rounded to the word.
__device__ __forceinline__ uint64_t exp_chirp_offset(const ChirpRec& c, int64_t m) {
  const double alpha = __longlong_as_double((long long)c.d[2]);
  const double C = __longlong_as_double((long long)c.d[3]);
  return (uint64_t)((q64_of(C * expm1(alpha * (double)m)) + ((unsigned __int128)1 << 63)) >> 64);
}

// Exact phase word of a chirp at offset m from its start: Phi(n_s) + top64(sum_i d_i C(m, i)).
// d_0 carries the 2^127 rounding offset.  (Exponential chirps: Phi(n_s) + R(m).)
__device__ uint64_t exact_chirp_word(const ChirpRec& c, int64_t m, const uint64_t (*inv)[3]) {
  if (c.flags & TONE_EXP) return c.phi_start + exp_chirp_offset(c, m);
  U192 b[7];
  binomials(m, inv, b);
  U192 s = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < 7; ++i) s = add192(s, mul192(dword(c, i), b[i]));
  return c.phi_start + s.w2;
}

__device__ __forceinline__ uint64_t exact_word(const ToneRec& t, const ChirpRec* chirps, int64_t n,
                                               const uint64_t (*inv)[3]) {
  if (t.slot < 0 || n < t.n_s) return t.phi_ref + (uint64_t)n * t.F;
  if (n > t.n_e) return t.phi_post_ref + (uint64_t)n * t.F_end;
  return exact_chirp_word(chirps[t.slot], n - t.n_s, inv);
}

// ------------------------------------------------------------------------------------------
// 32-bit run phases
// ------------------------------------------------------------------------------------------
constexpr uint64_t P_OFFSET = 1ull << 40;   // makes the 23-bit truncation of p round to nearest
constexpr uint64_t HALF32 = 1ull << 31;
// P_OFFSET plus half a turn: folded into the records' B_0 (stride_records)
constexpr uint64_t B0_OFFSET = P_OFFSET + (1ull << 63);

// A run's 32-bit cascade state: p is the run-start phase plus half a turn (the centred form that
// sin_centred takes), f, g, h its first three differences.
struct RunPoly {
  uint32_t p, f, g, h;
};

// C(j, q) for the run index j (0 <= j < RUNS = 128): q <= 5 fit in 32 bits, C(j, 6) needs 33.
struct RunBin {
  uint32_t c1, c2, c3, c4, c5;
  uint64_t c6;
};

__device__ __forceinline__ RunBin run_binomials(int j) {
  RunBin b;
  const uint64_t u = (uint64_t)j;
  const uint64_t c2 = u * (u - 1) / 2, c3 = c2 * (u - 2) / 3, c4 = c3 * (u - 3) / 4, c5 = c4 * (u - 4) / 5;
  b.c1 = (uint32_t)j;
  b.c2 = (uint32_t)c2;
  b.c3 = (uint32_t)c3;
  b.c4 = (uint32_t)c4;
  b.c5 = (uint32_t)c5;
  b.c6 = c5 * (u - 5) / 6;
  // a factor (u - i) is zero for j = i, so every product with q > j vanishes; j < q wraps (u - i)
  // but the zero factor comes first, so the products above are already 0 for those j.
  return b;
}

// acc + x * c (mod 2^64) for a 32-bit c: one wide and one narrow integer multiply-add
__device__ __forceinline__ uint64_t mac_u32(uint64_t acc, uint64_t x, uint32_t c) {
  const uint64_t lo = (uint64_t)(uint32_t)x * c;
  const uint32_t hi = (uint32_t)(x >> 32) * c;
  return acc + lo + ((uint64_t)hi << 32);
}

// The top 32 bits of a sum of 64-bit words times small integers, (sum_q x_q c_q mod 2^64) >> 32,
// accumulated as a 64-bit sum of the low halves' products plus a 32-bit sum of the high halves'
// products: S = 2^32 sum hi32(x_q) c_q + sum lo32(x_q) c_q, so bits 32..63 of S are the high sum
// plus bits 32..63 of the low sum, whatever wraps above bit 63.  Two integer multiply-adds per
// term; the same integers as the full 64-bit sum.
struct Top32 {
  uint64_t lo;
  uint32_t hi;
};
// start from word x (the records carry the rounding offsets in their order-0 words)
__device__ __forceinline__ Top32 top_init(uint64_t x) {
  return Top32{(uint64_t)(uint32_t)x, (uint32_t)(x >> 32)};
}
__device__ __forceinline__ void top_mac(Top32& t, uint64_t x, uint32_t c) {
  t.lo += (uint64_t)(uint32_t)x * c;
  t.hi += (uint32_t)(x >> 32) * c;
}
// x c mod 2^64 for a 64-bit c: lo32(x) lo32(c) + 2^32 (hi32(x) lo32(c) + lo32(x) hi32(c))
__device__ __forceinline__ void top_mac64(Top32& t, uint64_t x, uint64_t c) {
  t.lo += (uint64_t)(uint32_t)x * (uint32_t)c;
  t.hi += (uint32_t)(x >> 32) * (uint32_t)c + (uint32_t)x * (uint32_t)(c >> 32);
}
__device__ __forceinline__ uint32_t top_get(const Top32& t) { return t.hi + (uint32_t)(t.lo >> 32); }

constexpr uint64_t HALF32_OFF = 1ull << 31;

// (p, f, g, h) at run j from the stride-RUN records: p = sum_q B_q C(j,q), f = sum_q E_q C(j,q),
// g = sum_q G_q C(j,q), h = sum_q H_q C(j,q), all mod 2^64, then the top 32 bits.  The records'
// order-0 words carry the offsets (stride_records): B_0 the 2^8 offset of the sine argument and
// half a turn, so p is floor((phase + 2^40) / 2^32) + 2^31; E_0, G_0, H_0 half a unit, so f, g, h
// round to nearest.
__device__ __forceinline__ RunPoly poly_state(const TileRec& rc, const RunBin& b, bool linear) {
  RunPoly r;
  if (linear) {   // B_q (q >= 3), E_q (q >= 2), G_q (q >= 1) and H are exactly zero
    Top32 p = top_init(rc.B[0]);
    top_mac(p, rc.B[1], b.c1);
    top_mac(p, rc.B[2], b.c2);
    Top32 f = top_init(rc.E[0]);
    top_mac(f, rc.E[1], b.c1);
    r.p = top_get(p);
    r.f = top_get(f);
    r.g = (uint32_t)(rc.G[0] >> 32);
    r.h = 0;
    return r;
  }
  Top32 p = top_init(rc.B[0]);
  top_mac(p, rc.B[1], b.c1);
  top_mac(p, rc.B[2], b.c2);
  top_mac(p, rc.B[3], b.c3);
  top_mac(p, rc.B[4], b.c4);
  top_mac(p, rc.B[5], b.c5);
  top_mac64(p, rc.B[6], b.c6);
  Top32 f = top_init(rc.E[0]);
  top_mac(f, rc.E[1], b.c1);
  top_mac(f, rc.E[2], b.c2);
  top_mac(f, rc.E[3], b.c3);
  top_mac(f, rc.E[4], b.c4);
  top_mac(f, rc.E[5], b.c5);
  Top32 g = top_init(rc.G[0]);
  top_mac(g, rc.G[1], b.c1);
  top_mac(g, rc.G[2], b.c2);
  top_mac(g, rc.G[3], b.c3);
  top_mac(g, rc.G[4], b.c4);
  Top32 h = top_init(rc.H[0]);
  top_mac(h, rc.H[1], b.c1);
  top_mac(h, rc.H[2], b.c2);
  top_mac(h, rc.H[3], b.c3);
  r.p = top_get(p);
  r.f = top_get(f);
  r.g = top_get(g);
  r.h = top_get(h);
  return r;
}

// poly_state for a degree-6 chirp whose h is known to round to 0 (TONE_FLAT3): no H polynomial.
__device__ __forceinline__ RunPoly poly_state_flat3(const TileRec& rc, const RunBin& b) {
  Top32 p = top_init(rc.B[0]);
  top_mac(p, rc.B[1], b.c1);
  top_mac(p, rc.B[2], b.c2);
  top_mac(p, rc.B[3], b.c3);
  top_mac(p, rc.B[4], b.c4);
  top_mac(p, rc.B[5], b.c5);
  top_mac64(p, rc.B[6], b.c6);
  Top32 f = top_init(rc.E[0]);
  top_mac(f, rc.E[1], b.c1);
  top_mac(f, rc.E[2], b.c2);
  top_mac(f, rc.E[3], b.c3);
  top_mac(f, rc.E[4], b.c4);
  top_mac(f, rc.E[5], b.c5);
  Top32 g = top_init(rc.G[0]);
  top_mac(g, rc.G[1], b.c1);
  top_mac(g, rc.G[2], b.c2);
  top_mac(g, rc.G[3], b.c3);
  top_mac(g, rc.G[4], b.c4);
  return RunPoly{top_get(p), top_get(f), top_get(g), 0u};
}

// poly_state for a TONE_LOW6 chirp: FLAT3, and the set-up bounds B_6, E_5 and G_2..G_4 below 64
// units of 2^-32 turn of phase over a run, so they are left out.
__device__ __forceinline__ RunPoly poly_state_low6(const TileRec& rc, const RunBin& b) {
  Top32 p = top_init(rc.B[0]);
  top_mac(p, rc.B[1], b.c1);
  top_mac(p, rc.B[2], b.c2);
  top_mac(p, rc.B[3], b.c3);
  top_mac(p, rc.B[4], b.c4);
  top_mac(p, rc.B[5], b.c5);
  Top32 f = top_init(rc.E[0]);
  top_mac(f, rc.E[1], b.c1);
  top_mac(f, rc.E[2], b.c2);
  top_mac(f, rc.E[3], b.c3);
  top_mac(f, rc.E[4], b.c4);
  Top32 g = top_init(rc.G[0]);
  top_mac(g, rc.G[1], b.c1);
  return RunPoly{top_get(p), top_get(f), top_get(g), 0u};
}

// poly_state for a TONE_LOW3 chirp: LOW6, and B_5, E_3, E_4 left out as well (the set-up bounds all
// left-out terms below 256 units of 2^-32 turn over a two-run cascade).
__device__ __forceinline__ RunPoly poly_state_low3(const TileRec& rc, const RunBin& b) {
  Top32 p = top_init(rc.B[0]);
  top_mac(p, rc.B[1], b.c1);
  top_mac(p, rc.B[2], b.c2);
  top_mac(p, rc.B[3], b.c3);
  top_mac(p, rc.B[4], b.c4);
  Top32 f = top_init(rc.E[0]);
  top_mac(f, rc.E[1], b.c1);
  top_mac(f, rc.E[2], b.c2);
  Top32 g = top_init(rc.G[0]);
  top_mac(g, rc.G[1], b.c1);
  return RunPoly{top_get(p), top_get(f), top_get(g), 0u};
}


__device__ __forceinline__ uint32_t static_p0(uint64_t phi_ref, uint64_t F, int64_t n0) {
  return (uint32_t)((phi_ref + (uint64_t)n0 * F + P_OFFSET) >> 32);
}
__device__ __forceinline__ uint32_t static_f(uint64_t F) { return (uint32_t)((F + HALF32) >> 32); }

// Tile classification of a tone against a tile [T0, T0 + TILE).
enum { TILE_PRE = 0, TILE_POST = 1, TILE_CHIRP = 2 };
__device__ __forceinline__ int classify_tile(const ToneRec& t, int64_t T0) {
  if (t.slot < 0 || T0 + TILE - 1 < t.n_s) return TILE_PRE;
  if (T0 > t.n_e) return TILE_POST;
  return TILE_CHIRP;
}

// sin(2 pi p / 2^32) for a phase already offset by half a turn (pc = p + 2^31): the top 23 bits
// of pc become the mantissa of a float v in [1, 2); 2 pi (v - 3/2) lies in [-pi, pi) and is
// congruent to the phase.  The half-turn offset is added once per run, not per sample.
constexpr uint32_t HALF_TURN = 1u << 31;
// The float 1.m with the 23-bit fraction m = pc >> 9 (exponent field of [1, 2)).
__device__ __forceinline__ float mantissa_float(uint32_t pc) { return __uint_as_float((pc >> 9) + 0x3F800000u); }
__device__ __forceinline__ float sin_centred(uint32_t pc) {
  const float v = mantissa_float(pc);
  return __sinf(fmaf(v, 6.28318530717958647692f, -9.42477796076937971538f));
}

// ------------------------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after ~2 s of wall time.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------------------------------------
// prep: per (active chirp, tile) stride-RUN forward differences at the tile start
// ------------------------------------------------------------------------------------------
// a * b mod 2^192 for a signed 64-bit b: a (b mod 2^64) - [b < 0] a 2^64
__device__ __forceinline__ U192 mul192_s64(U192 a, int64_t bs) {
  const uint64_t b = (uint64_t)bs;
  unsigned __int128 p0 = (unsigned __int128)a.w0 * b;
  unsigned __int128 p1 = (unsigned __int128)a.w1 * b + (uint64_t)(p0 >> 64);
  U192 r;
  r.w0 = (uint64_t)p0;
  r.w1 = (uint64_t)p1;
  r.w2 = a.w2 * b + (uint64_t)(p1 >> 64);
  if (bs < 0) {
    unsigned __int128 t = (unsigned __int128)r.w1 - a.w0;
    r.w1 = (uint64_t)t;
    r.w2 = r.w2 - a.w1 - (uint64_t)((t >> 64) & 1);
  }
  return r;
}

// C(m, j), j = 0..DEG, signed m, exact (see binomials())
template <int DEG>
__device__ __forceinline__ void binomials_deg(int64_t m, const uint64_t (*inv)[3], U192 c[DEG + 1]) {
  U192 p = {1, 0, 0};
  c[0] = p;
#pragma unroll
  for (int j = 1; j <= DEG; ++j) {
    p = mul192_s64(p, m - (j - 1));
    U192 q = p;
    if (j == 3 || j == 4) q = mul192(q, U192{inv[0][0], inv[0][1], inv[0][2]});
    if (j == 5) q = mul192(q, U192{inv[1][0], inv[1][1], inv[1][2]});
    if (j == 6) q = mul192(q, U192{inv[2][0], inv[2][1], inv[2][2]});
    const int v = (j == 2 || j == 3) ? 1 : (j == 4 || j == 5) ? 3 : (j == 6) ? 4 : 0;
    c[j] = sar192(q, v);
  }
}

// Upper 128 bits of a 192-bit value (units of 2^64 of the Q64.128 word, i.e. Q64.64).
__device__ __forceinline__ unsigned __int128 hi128(U192 a) {
  return ((unsigned __int128)a.w2 << 64) | a.w1;
}
// Q64.64 -> word, rounded to nearest (mod 2^64)
__device__ __forceinline__ uint64_t round_q64(unsigned __int128 v) {
  return (uint64_t)((v + ((unsigned __int128)1 << 63)) >> 64);
}

// The stride-RUN records of a tile from the unit-stride forward differences h[1..DEG] of the
// chirp phase at the tile start (Q64.64 words, mod 2^128) and its phase word B0.  The order-0
// words take the run set-up's rounding offsets (poly_state): B_0 + 2^40 + 2^63, E_0, G_0 and
// H_0 + 2^31.
template <int DEG, class Args>
__device__ __forceinline__ void stride_records(const unsigned __int128* h, uint64_t B0, const Args& a,
                                               TileRec& out) {
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    unsigned __int128 s = 0;
#pragma unroll
    for (int i = q; i <= DEG; ++i) s += h[i] * (unsigned __int128)a.W[q][i];
    out.B[q] = (q == 0) ? B0 + B0_OFFSET : (q <= DEG ? round_q64(s) : 0);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    unsigned __int128 s = 0;
#pragma unroll
    for (int i = q; i + 1 <= DEG; ++i) s += h[i + 1] * (unsigned __int128)a.W[q][i];
    out.E[q] = (q + 1 <= DEG) ? round_q64(s) : 0;
    if (q == 0) out.E[0] += HALF32_OFF;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    unsigned __int128 s = 0;
#pragma unroll
    for (int i = q; i + 2 <= DEG; ++i) s += h[i + 2] * (unsigned __int128)a.W[q][i];
    out.G[q] = (q + 2 <= DEG) ? round_q64(s) : 0;
    if (q == 0) out.G[0] += HALF32_OFF;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned __int128 s = 0;
#pragma unroll
    for (int i = q; i + 3 <= DEG; ++i) s += h[i + 3] * (unsigned __int128)a.W[q][i];
    out.H[q] = (q + 3 <= DEG) ? round_q64(s) : 0;
    if (q == 0) out.H[0] += HALF32_OFF;
  }
}

// d c mod 2^192 for a multiplier c whose 64-bit limbs above the first L are zero: the partial
// products of those limbs are left out (the same value as mul192).
template <int L>
__device__ __forceinline__ U192 mul192_limbs(U192 d, U192 c) {
  const unsigned __int128 p00 = (unsigned __int128)d.w0 * c.w0;
  const unsigned __int128 p10 = (unsigned __int128)d.w1 * c.w0;
  unsigned __int128 mid = (p00 >> 64) + (uint64_t)p10;
  uint64_t top = (uint64_t)(p10 >> 64) + d.w2 * c.w0;
  if (L >= 2) {
    const unsigned __int128 p01 = (unsigned __int128)d.w0 * c.w1;
    mid += (uint64_t)p01;
    top += (uint64_t)(p01 >> 64) + d.w1 * c.w1;
  }
  if (L >= 3) top += d.w0 * c.w2;
  return U192{(uint64_t)p00, (uint64_t)mid, top + (uint64_t)(mid >> 64)};
}

// Inverses of 3 and 5 modulo 2^128 / 2^192 (3 * 0xA..AB = 1 and 5 * 0xC..CD = 1 modulo the power of
// two): an exact quotient by 3 or 5 is a product with the inverse.
constexpr uint64_t INV3_W = 0xAAAAAAAAAAAAAAAAull, INV3_W0 = 0xAAAAAAAAAAAAAAABull;
constexpr uint64_t INV5_W = 0xCCCCCCCCCCCCCCCCull, INV5_W0 = 0xCCCCCCCCCCCCCCCDull;

// C(m, j), j = 0..DEG, for 0 <= m < 2^29 (every tile a chirp covers), each from the one before:
// C(m, j) = C(m, j-1) (m - j + 1) / j.  C(m, 1), C(m, 2) < 2^57 fit one 64-bit limb, C(m, 3) and
// C(m, 4) < 2^112 two, C(m, 5), C(m, 6) < 2^165 three; the quotients are exact, so a division by 3
// or 5 is a product with the inverse modulo 2^128 or 2^192 and a division by 2 or 4 a shift.
template <int DEG>
__device__ __forceinline__ void binomials_pos(uint64_t m, U192 c[DEG + 1]) {
  c[0] = U192{1, 0, 0};
  c[1] = U192{m, 0, 0};
  const uint64_t c2 = (m * (m - 1)) >> 1;
  c[2] = U192{c2, 0, 0};
  if (DEG >= 3) {
    unsigned __int128 t = (unsigned __int128)c2 * (m - 2);                 // 3 C(m, 3) < 2^86
    t *= ((unsigned __int128)INV3_W << 64) | INV3_W0;
    c[3] = U192{(uint64_t)t, (uint64_t)(t >> 64), 0};
    t = (t * (unsigned __int128)(m - 3)) >> 2;                              // C(m, 4) < 2^112
    c[4] = U192{(uint64_t)t, (uint64_t)(t >> 64), 0};
    U192 u = mul192_limbs<1>(c[4], U192{m - 4, 0, 0});                      // 5 C(m, 5)
    c[5] = mul192(u, U192{INV5_W0, INV5_W, INV5_W});
    u = mul192_limbs<1>(c[5], U192{m - 5, 0, 0});                           // 6 C(m, 6)
    u = mul192(u, U192{INV3_W0, INV3_W, INV3_W});                           // 2 C(m, 6)
    c[6] = U192{(u.w0 >> 1) | (u.w1 << 63), (u.w1 >> 1) | (u.w2 << 63), u.w2 >> 1};
  }
}

// acc[k] = sum over i >= k of d_i C(m, i - k), k = 0..DEG, the products by C(m, j) taking its limb
// count.  Each d_i is loaded once and added into every acc[k] it contributes to (the sums are
// exact mod 2^192, so their order does not matter).
template <int DEG>
__device__ __forceinline__ void newton_shift_pos(const ChirpRec& c, const U192* bin, U192* acc) {
#pragma unroll
  for (int i = 0; i <= DEG; ++i) {
    const U192 d = dword(c, i);
    acc[i] = d;
#pragma unroll
    for (int k = 0; k < i; ++k) {
      const int j = i - k;
      if (j <= 2) acc[k] = add192(acc[k], mul192_limbs<1>(d, bin[j]));
      else if (j <= 4) acc[k] = add192(acc[k], mul192_limbs<2>(d, bin[j]));
      else acc[k] = add192(acc[k], mul192_limbs<3>(d, bin[j]));
    }
  }
}

// DEG = 2 (linear chirps) or 6 (minimum-jerk).  The unit-stride differences at the tile start
// are exact (192-bit); the stride-RUN transform that follows only needs the word-level result,
// so it runs on the upper 128 bits (error < W 2^-64 word per term, below 2^-20 word).  Tiles
// from the chirp's start on (0 <= m < 2^29) take the binomials' limb counts into account; a tile
// that begins before the chirp (m < 0) takes signed binomials (both the same integers).
// the unit-stride differences at a tile that begins before the chirp (signed binomials)
template <int DEG>
__device__ __forceinline__ void newton_shift_signed(const ChirpRec& c, int64_t m, const uint64_t (*inv)[3], U192* acc) {
  U192 bin[DEG + 1];
  binomials_deg<DEG>(m, inv, bin);
#pragma unroll
  for (int k = 0; k <= DEG; ++k) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = k; i <= DEG; ++i) s = add192(s, mul192(dword(c, i), bin[i - k]));
    acc[k] = s;
  }
}

template <int DEG, class Args>
__device__ __forceinline__ void prep_one(const ChirpRec& c, int64_t m, const Args& a, TileRec& out) {
  U192 acc[DEG + 1];
  if (m >= 0 && m < ((int64_t)1 << 29)) {
    U192 bin[DEG + 1];
    binomials_pos<DEG>((uint64_t)m, bin);
    newton_shift_pos<DEG>(c, bin, acc);
  } else {
    newton_shift_signed<DEG>(c, m, a.inv_odd, acc);
  }
  unsigned __int128 h[DEG + 1];
#pragma unroll
  for (int k = 0; k <= DEG; ++k) h[k] = hi128(acc[k]);
  stride_records<DEG>(h, c.phi_start + acc[0].w2, a, out);   // acc_0 holds 2^127
}

// Exponential chirps: the unit forward differences of R(m) = C (e^(alpha m) - 1) at the tile
// start are C e^(alpha m) q^k (k >= 1, q = e^alpha - 1), in FP64 (a few 1e-10 turn), cut after
// order 6: the set-up gives a chirp a per-sample table instead when the dropped orders could
// reach 2^-26 turn over a tile.
template <class Args>
__device__ __forceinline__ void prep_exp(const ChirpRec& c, int64_t m, const Args& a, TileRec& out) {
  const double alpha = __longlong_as_double((long long)c.d[2]);
  const double C = __longlong_as_double((long long)c.d[3]);
  const double q = __longlong_as_double((long long)c.d[4]);
  const double e1 = expm1(alpha * (double)m);
  unsigned __int128 h[7];
  h[0] = q64_of(C * e1);
  double g = C * (e1 + 1.0) * q;
#pragma unroll
  for (int k = 1; k <= 6; ++k) {
    h[k] = q64_of(g);
    g *= q;
  }
  stride_records<6>(h, c.phi_start + (uint64_t)((h[0] + ((unsigned __int128)1 << 63)) >> 64), a, out);
}

// Programmatic dependent launch (pipelined chunk sequences): the next kernel in the stream may
// start once every CTA of this one has passed launch_dependents; wait blocks until the preceding
// kernel has completed and its memory is visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bounded wait (limit_ns of wall time) until a device counter reaches target; false on timeout.
__device__ bool wait_counter(const unsigned long long* ctr, unsigned long long target, uint64_t limit_ns) {
  const volatile unsigned long long* v = ctr;
  if (*v >= target) return true;
  const uint64_t t0 = global_ns();
  while (*v < target) {
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(256);
  }
  return true;
}

template <class Args>
__global__ void __launch_bounds__(128, 5) prep_kernel(const __grid_constant__ Args a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)a.n_active * a.n_tiles;
  if (idx >= total) return;
  const int ai = (int)(idx / a.n_tiles);
  const int t = (int)(idx - (int64_t)ai * a.n_tiles);
  const int slot = a.slots[ai];
  const ChirpRec& c = a.chirps[slot];
  if (t == 0) a.act_of_slot[slot] = a.act_base + ai;
  const int64_t T0 = (a.tile0 + t) * (int64_t)TILE;
  TileRec out;
  if (c.flags & TONE_LINEAR) prep_one<2>(c, T0 - c.n_s, a, out);
  else if (c.flags & TONE_EXP) prep_exp(c, T0 - c.n_s, a, out);
  else prep_one<6>(c, T0 - c.n_s, a, out);
  a.recs[(int64_t)(a.act_base + ai) * a.n_tiles + t] = out;
}

// ------------------------------------------------------------------------------------------
// render
// ------------------------------------------------------------------------------------------
// Accumulators: a thread's RUN partial sums as RUN / 2 pairs of consecutive samples (float2).
// The static and chirp loops compute the sine arguments and the multiply-adds of two samples as
// packed FP32 pairs (each component rounds as fmaf, so the sums are the same bits as with scalar
// fmaf): one instruction per tone-sample fewer (8.5 -> 7.5 on the 1000-chirp record).
typedef float2 Acc[RUN / 2];

constexpr float TWO_PI_F = 6.28318530717958647692f;
constexpr float THREE_PI_F = 9.42477796076937971538f;

// acc += (A0 sin(p0), A1 sin(p1)) for two phases already offset by half a turn (see sin_centred)
__device__ __forceinline__ void acc_pair(float2& acc, float A0, float A1, uint32_t p0, uint32_t p1) {
  acc.x = fmaf(A0, sin_centred(p0), acc.x);
  acc.y = fmaf(A1, sin_centred(p1), acc.y);
}
// the same for one amplitude, as packed FP32 pairs
__device__ __forceinline__ void acc_pair_packed(float2& acc, float A, uint32_t p0, uint32_t p1) {
  const float2 v = make_float2(mantissa_float(p0), mantissa_float(p1));
  const float2 x = __ffma2_rn(v, make_float2(TWO_PI_F, TWO_PI_F), make_float2(-THREE_PI_F, -THREE_PI_F));
  acc = __ffma2_rn(make_float2(A, A), make_float2(__sinf(x.x), __sinf(x.y)), acc);
}
// acc += (A0 s0, A1 s1) for sines already computed
__device__ __forceinline__ void acc_pair_s(float2& acc, float A0, float A1, float s0, float s1) {
  acc.x = fmaf(A0, s0, acc.x);
  acc.y = fmaf(A1, s1, acc.y);
}

// Static segment over N samples from acc pair B: p += f per sample.
template <int B, int N>
__device__ __forceinline__ void static_loop(uint32_t p, uint32_t f, float A, Acc& acc) {
#pragma unroll
  for (int r = 0; r < N; r += 2) {
    const uint32_t p1 = p + f;
    acc_pair_packed(acc[B + r / 2], A, p, p1);
    p = p1 + f;
  }
}

// Chirp cascade over N samples from acc pair B: p += f, f += g (and g += h with WITH_H).
template <int B, int N, bool WITH_H>
__device__ __forceinline__ void cascade(const RunPoly& q, float A, Acc& acc) {
  uint32_t p = q.p, f = q.f, g = q.g;
  const uint32_t h = q.h;
#pragma unroll
  for (int r = 0; r < N; r += 2) {
    const uint32_t p1 = p + f;
    uint32_t f1 = f + g;
    if (WITH_H) g += h;
    acc_pair_packed(acc[B + r / 2], A, p, p1);
    p = p1 + f1;
    f = f1 + g;
    if (WITH_H) g += h;
  }
}

// Per (tone, run) contribution of one staged tone, added into the thread's partial sums.
// Amplitude a(n) of a ramping tone (TONE_AMP_RAMP): A before a_ns, A_end from a_ns + a_L on, and
// A + (A_end - A) s(tau) between, tau = (n - a_ns) / a_L, s linear or minimum-jerk
// (10 tau^3 - 15 tau^4 + 6 tau^5).  FP32 (tau as m times the rounded 1 / a_L); error
// <= 6e-7 |A_end - A|.
// Per run: the offset of the run start into the ramp and 1 / a_L; ramp_amp_at(rr, r) is a(n0 + r),
// with tau = m (1 / a_L) in FP32 (a function of the absolute sample only, whatever the window).
struct RampRun {
  int64_t m0;       // n0 - a_ns
  int64_t L;
  float inv_L, A, A_end, dA;
  bool minjerk;
};
__device__ __forceinline__ RampRun ramp_run_setup(const ToneRec& t, int64_t n0) {
  RampRun rr;
  rr.m0 = n0 - t.a_ns;
  rr.L = t.a_L;
  rr.inv_L = 1.0f / (float)t.a_L;
  rr.A = t.A;
  rr.A_end = t.A_end;
  rr.dA = t.A_end - t.A;
  rr.minjerk = (t.flags & TONE_AMP_MINJERK) != 0;
  return rr;
}
__device__ __forceinline__ float ramp_amp_at(const RampRun& rr, int r) {
  const int64_t m = rr.m0 + r;
  if (m <= 0) return rr.A;
  if (m >= rr.L) return rr.A_end;
  const float tau = (float)m * rr.inv_L;
  const float s = rr.minjerk ? tau * tau * tau * fmaf(tau, fmaf(6.f, tau, -15.f), 10.f) : tau;
  return fmaf(rr.dA, s, rr.A);
}

// The general paths for the thread's run (samples n0 .. n0 + RUN - 1), used where a tile holds a
// chirp boundary, an amplitude ramp or a per-sample phase table; col holds the run's RUN sines,
// sample r at col[r * cs] (a column of the cluster render's shared tile buffer, stride RUNS, or a
// local array, stride 1).
__device__ __forceinline__ void tone_run(const ToneRec& tr, const TileRec* rec, const RunBin& rb, float* col,
                                         Acc& acc, int64_t T0, int64_t n0, const uint32_t* exact_tab, int cs) {
  constexpr int B = 0;
  const bool ramp = (tr.flags & TONE_AMP_RAMP) != 0;
  const bool ramp_run = ramp && n0 + RUN - 1 > tr.a_ns && n0 < tr.a_ns + tr.a_L;   // a(n) varies in the run
  const float A = (ramp && n0 >= tr.a_ns + tr.a_L) ? tr.A_end : tr.A;
  const int tcls = classify_tile(tr, T0);
  int mode;   // 0 static before the chirp, 1 static after, 2 chirp polynomial, 3 general
  if (tcls == TILE_PRE) {
    mode = 0;
  } else if (tcls == TILE_POST) {
    mode = 1;
  } else {
    const int64_t last = n0 + RUN - 1;
    if (last < tr.n_s) mode = 0;
    else if (n0 > tr.n_e) mode = 1;
    else if (n0 >= tr.n_s && last <= tr.n_e && !(tr.flags & TONE_EXACT)) mode = 2;
    else mode = 3;
  }
  if (!ramp && !(tr.flags & TONE_EXACT)) {
    // no ramp and no table (tile TILE_CHIRP, record present): one loop per warp.  The same
    // integers as the per-thread paths below, without running three of them one after another
    // in the warp that holds a chirp boundary.
    if (__all_sync(0xffffffffu, mode <= 1)) {
      const uint64_t phi = mode == 0 ? tr.phi_ref : tr.phi_post_ref;
      const uint64_t F = mode == 0 ? tr.F : tr.F_end;
      static_loop<B, RUN>(static_p0(phi, F, n0) + HALF_TURN, static_f(F), A, acc);
      return;
    }
    const RunPoly st = poly_state(*rec, rb, (tr.flags & TONE_LINEAR) != 0);
    if (__all_sync(0xffffffffu, mode == 2)) {
      if (__all_sync(0xffffffffu, st.h == 0)) cascade<B, RUN, false>(st, A, acc);
      else cascade<B, RUN, true>(st, A, acc);
      return;
    }
    // a boundary in the warp: sample r takes the static phase before the chirp (r < i1), the
    // one after it (r > i2), else the chirp cascade; i1, i2 clamped to [-1, RUN]
    const int i1 = (int)max((int64_t)-1, min((int64_t)RUN, tr.n_s - n0));
    const int i2 = (int)max((int64_t)-1, min((int64_t)RUN, tr.n_e - n0));
    uint32_t qa = static_p0(tr.phi_ref, tr.F, n0) + HALF_TURN, qb = static_p0(tr.phi_post_ref, tr.F_end, n0) + HALF_TURN;
    const uint32_t fa = static_f(tr.F), fb = static_f(tr.F_end);
    uint32_t pp = st.p, ff = st.f, gg = st.g;
    const uint32_t hh = st.h;
#pragma unroll
    for (int r = 0; r < RUN; r += 2) {
      const uint32_t ph0 = r < i1 ? qa : (r > i2 ? qb : pp);
      qa += fa;
      qb += fb;
      pp += ff;
      ff += gg;
      gg += hh;
      const uint32_t ph1 = r + 1 < i1 ? qa : (r + 1 > i2 ? qb : pp);
      qa += fa;
      qb += fb;
      pp += ff;
      ff += gg;
      gg += hh;
      acc_pair(acc[B + r / 2], A, A, ph0, ph1);
    }
    return;
  }
  if (ramp_run && mode <= 1) {
    // a ramp on a static segment: stepped phase, the amplitude of ramp_amp per sample
    const uint64_t phi = mode == 0 ? tr.phi_ref : tr.phi_post_ref;
    const uint64_t F = mode == 0 ? tr.F : tr.F_end;
    uint32_t p = static_p0(phi, F, n0) + HALF_TURN;
    const uint32_t f = static_f(F);
    const RampRun rr = ramp_run_setup(tr, n0);
#pragma unroll
    for (int r = 0; r < RUN; r += 2) {
      acc_pair(acc[B + r / 2], ramp_amp_at(rr, r), ramp_amp_at(rr, r + 1), p, p + f);
      p += 2 * f;
    }
  } else if (ramp_run) {
    mode = 3;
  }
  if (ramp_run) {
    if (mode <= 1) return;
  } else if (mode <= 1) {
    const uint64_t phi = mode == 0 ? tr.phi_ref : tr.phi_post_ref;
    const uint64_t F = mode == 0 ? tr.F : tr.F_end;
    static_loop<B, RUN>(static_p0(phi, F, n0) + HALF_TURN, static_f(F), A, acc);
    return;
  }
  if (mode == 2) {
    cascade<B, RUN, true>(poly_state(*rec, rb, (tr.flags & TONE_LINEAR) != 0), A, acc);
  } else {
    // a segment boundary inside this run, or a table chirp: choose the segment per sample; the
    // sines go to col, then into the accumulators
    const uint32_t p_pre = static_p0(tr.phi_ref, tr.F, n0) + HALF_TURN, f_pre = static_f(tr.F);
    const uint32_t p_post = static_p0(tr.phi_post_ref, tr.F_end, n0) + HALF_TURN, f_post = static_f(tr.F_end);
    const bool exact = (tr.flags & TONE_EXACT) != 0;
    RunPoly st = {0, 0, 0, 0};
    if (!exact && tcls == TILE_CHIRP) st = poly_state(*rec, rb, (tr.flags & TONE_LINEAR) != 0);
    const int64_t r1 = tr.n_s - n0, r2 = tr.n_e - n0;
    uint32_t pp = st.p, ff = st.f, gg = st.g;
    for (int r = 0; r < RUN; ++r) {
      uint32_t ph;
      if (r < r1) ph = p_pre + (uint32_t)r * f_pre;
      else if (r > r2) ph = p_post + (uint32_t)r * f_post;
      else ph = exact ? exact_tab[tr.tab_off + (int32_t)(r - r1)] + HALF_TURN : pp;
      col[r * cs] = sin_centred(ph);
      pp += ff;
      ff += gg;
      gg += st.h;
    }
    if (ramp_run) {
      const RampRun rr = ramp_run_setup(tr, n0);
#pragma unroll
      for (int r = 0; r < RUN; r += 2)
        acc_pair_s(acc[B + r / 2], ramp_amp_at(rr, r), ramp_amp_at(rr, r + 1), col[r * cs], col[(r + 1) * cs]);
    } else {
#pragma unroll
      for (int r = 0; r < RUN; r += 2) acc_pair_s(acc[B + r / 2], A, A, col[r * cs], col[(r + 1) * cs]);
    }
  }
}

// Per-stage tone descriptor, built by warp 0 once per (tone, tile) so that the other threads
// skip the classification and the 64-bit phase set-up of static segments.
struct alignas(16) Desc {
  uint64_t p0;    // static: phase word at the tile start of the segment covering the tile
  uint64_t F;     // static: its frequency word
  float A;
  int32_t kind;
  float c, s;     // DESC_STATIC_ROT: cos and sin of the per-sample phase step
};
enum { DESC_STATIC = 0, DESC_LINEAR = 1, DESC_MINJERK = 2, DESC_MIXED = 3, DESC_STATIC_ROT = 4, DESC_SKIP = 5,
       DESC_FLAT3 = 6,     // FLAT3: a degree-6 chirp whose h is 0 in every run (TONE_FLAT3)
       DESC_LOW6 = 7,      // LOW6: FLAT3 without the negligible high orders (TONE_LOW6)
       DESC_LOW3 = 8 };    // LOW3: LOW6 without B_5, E_3, E_4 (TONE_LOW3)

// Kind of a chirp tile that the chirp covers from start to end (no table, no ramp in the tile).
__device__ __forceinline__ int chirp_inside_kind(int32_t flags) {
  return (flags & TONE_LINEAR) ? DESC_LINEAR : (flags & TONE_LOW3) ? DESC_LOW3 : (flags & TONE_LOW6) ? DESC_LOW6
         : (flags & TONE_FLAT3) ? DESC_FLAT3 : DESC_MINJERK;
}

// Descriptor kind of a tone in the tile [T0, T0 + TILE): DESC_STATIC for a static segment (the
// stage turns it into DESC_STATIC_ROT under the rotator sine), a chirp kind for a chirp that covers
// the tile without a table, DESC_MIXED for a chirp boundary, a table or an amplitude ramp in the
// tile, DESC_SKIP for a static segment the tensor-core engine sums.
__device__ __forceinline__ int tile_kind(const ToneRec& tr, int64_t T0, bool skip_static) {
  const int tcls = classify_tile(tr, T0);
  int kind;
  if (tcls == TILE_PRE || tcls == TILE_POST) {
    kind = DESC_STATIC;
  } else {
    const bool inside = T0 >= tr.n_s && T0 + TILE - 1 <= tr.n_e;
    kind = (inside && !(tr.flags & TONE_EXACT)) ? chirp_inside_kind(tr.flags) : DESC_MIXED;
  }
  if ((tr.flags & TONE_AMP_RAMP) && T0 + TILE - 1 > tr.a_ns && T0 < tr.a_ns + tr.a_L) kind = DESC_MIXED;
  if (skip_static && tile_static(tr, T0)) kind = DESC_SKIP;
  return kind;
}

// Visit group of a stage's tone: chirps in linear form that may share their run set-up (TONE_PAIR),
// the other linear ones, chirps in LOW3 form that may share it, the same two for LOW6 form, static
// segments, then the rest (every tone of a listed render; LOW3 chirps that may not share).  Shared
// set-ups only in renders without the tensor-core engine (pair false).
enum { GRP_LIN_PAIR = 0, GRP_LIN = 1, GRP_LOW3_PAIR = 2, GRP_LOW6_PAIR = 3, GRP_LOW6 = 4, GRP_STATIC = 5, GRP_REST = 6,
       N_GRP = 7 };
__device__ __forceinline__ int visit_group(int kind, bool listed, bool pair) {
  if (listed) return GRP_REST;
  if (kind == DESC_LINEAR) return pair ? GRP_LIN_PAIR : GRP_LIN;
  if (kind == DESC_LOW3) return pair ? GRP_LOW3_PAIR : GRP_REST;
  if (kind == DESC_LOW6) return pair ? GRP_LOW6_PAIR : GRP_LOW6;
  return (kind == DESC_STATIC || kind == DESC_STATIC_ROT) ? GRP_STATIC : GRP_REST;
}

// Run set-up shared by a lane pair.  Lanes 2m and 2m + 1 (runs j and j + 1) take two tones of a
// group: each evaluates one tone's set-up exactly (the even lane the first tone's, the odd lane the
// second's) and takes the other tone's from its partner, moved by one run with the cascade's own
// integer steps (h = 0): forward from run j - 1, p + 32 f + 496 g and f + 32 g (the state the
// partner's cascade reaches after 32 samples); backward from run j + 1, p - 32 f + 528 g and
// f - 32 g (C(-32, 2) = 528).  The moved state's error is the cascade's over up to 63 steps
// (pair_setup_ok on the host bounds it).  Every lane of the warp takes part.
__device__ __forceinline__ RunPoly partner_state(const RunPoly& own, bool odd) {
  const uint32_t p = __shfl_xor_sync(0xffffffffu, own.p, 1);
  const uint32_t f = __shfl_xor_sync(0xffffffffu, own.f, 1);
  const uint32_t g = __shfl_xor_sync(0xffffffffu, own.g, 1);
  RunPoly q;
  if (odd) {
    q.p = p + 32u * f + 496u * g;
    q.f = f + 32u * g;
  } else {
    q.p = p - 32u * f + 528u * g;
    q.f = f - 32u * g;
  }
  q.g = g;
  q.h = 0;
  return q;
}

// Scale, round half to even, clamp and store sample n (inside the window), after adding the
// tensor-core engine's static sum when there is one.
__device__ __forceinline__ void store_sample(const RenderArgs& a, int64_t n, float x) {
  if (n < a.win_start || n >= a.win_end) return;
  if (a.base) x += a.base[n - a.win_start];
  float q = rintf(x * a.scale);
  q = fminf(fmaxf(q, -32767.f), 32767.f);
  if (a.out_q) a.out_q[(n - a.win_start) * (a.q_stride ? a.q_stride : 1)] = (int16_t)q;
  if (a.out_f) a.out_f[n - a.win_start] = x;
}

// Whether 8-sample groups (first sample a multiple of 8) of the int16 and FP32 outputs start on
// 16-byte boundaries: sample n sits at out + (n - win_start), so this holds for every group at
// once when out - win_start is 16-byte aligned.
__device__ __forceinline__ bool q_vec_ok(const RenderArgs& a) {
  return a.out_q && a.q_stride <= 1 && (((uintptr_t)a.out_q - 2u * (uint64_t)a.win_start) & 15u) == 0;
}
__device__ __forceinline__ bool f_vec_ok(const RenderArgs& a) {
  return !a.out_f || (((uintptr_t)a.out_f - 4u * (uint64_t)a.win_start) & 15u) == 0;
}

// Store the 8 samples n .. n + 7 (n a multiple of 8): one 16-byte vector of int16 codes (and two
// of FP32 sums) when the group lies inside the window and the outputs are aligned, else sample
// by sample.
__device__ __forceinline__ void store_group(const RenderArgs& a, int64_t n, const float (&xv)[8], bool vec) {
  if (vec && n >= a.win_start && n + 8 <= a.win_end) {
    const int64_t o = n - a.win_start;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = a.base ? xv[u] + a.base[o + u] : xv[u];
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float q0 = fminf(fmaxf(rintf(x[2 * u] * a.scale), -32767.f), 32767.f);
      const float q1 = fminf(fmaxf(rintf(x[2 * u + 1] * a.scale), -32767.f), 32767.f);
      w[u] = (uint32_t)(uint16_t)(int16_t)q0 | ((uint32_t)(uint16_t)(int16_t)q1 << 16);
    }
    if (a.out_q) *reinterpret_cast<uint4*>(a.out_q + o) = make_uint4(w[0], w[1], w[2], w[3]);
    if (a.out_f) {
      float4* f4 = reinterpret_cast<float4*>(a.out_f + o);
      f4[0] = make_float4(x[0], x[1], x[2], x[3]);
      f4[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) store_sample(a, n + u, xv[u]);
}

// Sum over the split without clusters.  Thread t holds samples RUN t .. RUN t + RUN - 1 of the
// tile in acc.  With split 1 it stores them; otherwise the CTA writes them to its partial tile
// a.part[(tile split + crank) TILE ...] and counts itself in on a.tile_ctr[tile]; the CTA that
// brings the count to split - 1 (mod split) is the last of the tile: it sums the split's partials
// in rank order (as the cluster reduction does: the same FP32 sums) and stores all 4096 samples,
// thread t taking the 8-sample groups t, t + RT, ... (coalesced 16-byte stores).
// In a pipelined sequence (pdl 2) the scratch of this launch was used two launches back: waiting
// for the preceding launch to complete (which waited for the one before) makes it free.
__device__ __forceinline__ void tile_epilogue_split(const RenderArgs& a, int tile, int crank, int split, int64_t T0,
                                                    const Acc& acc) {
  const int tid = threadIdx.x;
  __shared__ int s_last;
  const bool vec = q_vec_ok(a) && f_vec_ok(a);
  if (split == 1) {
#pragma unroll
    for (int g = 0; g < RUN / 8; ++g) {
      float xv[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xv[2 * u] = 0.f + acc[4 * g + u].x;
        xv[2 * u + 1] = 0.f + acc[4 * g + u].y;
      }
      store_group(a, T0 + (int64_t)tid * RUN + 8 * g, xv, vec);
    }
  } else {
    if (a.pdl == 2) pdl_wait();
    float4* dst = reinterpret_cast<float4*>(a.part + ((int64_t)tile * split + crank) * TILE + tid * RUN);
#pragma unroll
    for (int j = 0; j < RUN / 4; ++j)
      __stcg(dst + j, make_float4(acc[2 * j].x, acc[2 * j].y, acc[2 * j + 1].x, acc[2 * j + 1].y));
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.tile_ctr[tile], 1ull) % (unsigned long long)split == (unsigned long long)(split - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      // rank by rank, the thread's 8-sample groups tid + RT v, 16-byte loads in flight
      constexpr int G = TILE / 8 / RT;   // 8-sample groups per thread
      const float4* src = reinterpret_cast<const float4*>(a.part + (int64_t)tile * split * TILE) + 2 * tid;
      float xs[G][8];
#pragma unroll
      for (int v = 0; v < G; ++v)
#pragma unroll
        for (int u = 0; u < 8; ++u) xs[v][u] = 0.f;
      for (int c = 0; c < split; ++c) {
#pragma unroll
        for (int v = 0; v < G; ++v) {
          const float4 lo = __ldcg(src + (int64_t)c * (TILE / 4) + 2 * RT * v);
          const float4 hi = __ldcg(src + (int64_t)c * (TILE / 4) + 2 * RT * v + 1);
          xs[v][0] += lo.x;
          xs[v][1] += lo.y;
          xs[v][2] += lo.z;
          xs[v][3] += lo.w;
          xs[v][4] += hi.x;
          xs[v][5] += hi.y;
          xs[v][6] += hi.z;
          xs[v][7] += hi.w;
        }
      }
#pragma unroll
      for (int v = 0; v < G; ++v) store_group(a, T0 + 8 * ((int64_t)tid + RT * v), xs[v], vec);
    }
  }
  if (a.exit_ctr) {   // this CTA's samples (if any) are stored and visible
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(a.exit_ctr, 1ull);
  }
}

// One CTA's share of one tile: tones [K crank / split, K (crank+1) / split) of window tile `tile`
// of the render described by `a` (or the listed tones of its bounds), then the sum over the split
// and the store.  CLUSTER: the split's CTAs form a thread-block cluster, sum through distributed
// shared memory in rank order and each stores a slice.  Otherwise each CTA writes its partial
// tile to a.part and the last of the split to finish (a counter per tile) sums the partials in
// rank order and stores the whole tile: the same sums, and no CTA waits for the others.
template <bool CLUSTER>
__device__ __forceinline__ void render_tile(const RenderArgs& a, const int tile, const int crank, const int split) {
  __shared__ alignas(16) ToneRec s_tone[2][STAGE];
  __shared__ alignas(16) TileRec s_rec[2][STAGE];
  __shared__ alignas(16) Desc s_desc[2][STAGE];
  __shared__ uint8_t s_order[2][STAGE];          // visit order: linear chirps, LOW6 chirps, the rest
  __shared__ int s_ngrp[2][N_GRP - 1];            // ends of the visit groups before the last
  // cluster sums through distributed shared memory: [i][thread]; without clusters the general
  // per-sample path keeps its run's sines in a local array (lcol) instead, so that the CTA's
  // shared memory (20 KB) leaves room for AWG_RENDER_SPLIT_MIN_BLOCKS CTAs per SM
  __shared__ alignas(16) float s_red[CLUSTER ? TILE : 4];
  float lcol[RUN];
  __shared__ alignas(8) uint64_t s_bar[4];        // tones[0], tones[1], records[0], records[1]

  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const int64_t T0 = (a.tile0 + tile) * (int64_t)TILE;
  const int64_t n0 = T0 + (int64_t)tid * RUN;       // the thread's run
  const uint32_t run_off = (uint32_t)(tid * RUN);
  // positions [l_begin, l_end) of the visit: the CTA's range of tones, or of the tone list
  int l_begin = (int)((int64_t)a.K * crank / split);
  int l_end = (int)((int64_t)a.K * (crank + 1) / split);
  if (a.tone_list) {
    const int k_begin = a.bounds[crank], k_end = a.bounds[crank + 1];
    auto lower = [&](int key) {
      int lo = 0, hi = a.n_list;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a.tone_list[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    l_begin = lower(k_begin);
    l_end = lower(k_end);
  }
  const int n_stages = (l_end - l_begin + STAGE - 1) / STAGE;

  Acc acc;
#pragma unroll
  for (int r = 0; r < RUN / 2; ++r) acc[r] = make_float2(0.f, 0.f);

  if (a.pdl == 1) {   // pipelined sequence: the records' set-up (the preceding kernel) is complete
    pdl_wait();         // before the next render may start (it relies on the same set-up)
    pdl_launch_dependents();
  } else if (a.pdl == 2) {
    pdl_launch_dependents();
  }
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < 4; ++b) mbar_init(&s_bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // thread 0 issues the tone copies and counts the issues per barrier (for a bounded drain)
  uint32_t issued = 0;   // 8-bit issue count per barrier
  // warp 0: one bulk copy of the stage's contiguous tone records, or one per listed tone
  auto issue_tones = [&](int st) {
    const int lb = l_begin + st * STAGE;
    const int cnt = min(STAGE, l_end - lb);
    fence_proxy_async();
    if (tid == 0) {
      mbar_arrive_expect_tx(&s_bar[st & 1], (uint32_t)cnt * (uint32_t)sizeof(ToneRec));
      issued += 1u << (8 * (st & 1));
    }
    __syncwarp();
    if (!a.tone_list) {
      if (tid == 0) bulk_g2s(&s_tone[st & 1][0], a.tones + lb, (uint32_t)cnt * (uint32_t)sizeof(ToneRec), &s_bar[st & 1]);
    } else if (tid < cnt) {
      bulk_g2s(&s_tone[st & 1][tid], a.tones + a.tone_list[lb + tid], (uint32_t)sizeof(ToneRec), &s_bar[st & 1]);
    }
  };
  // warp 0, once the stage's tones have landed: descriptors, and the records of tones that
  // chirp inside this tile
  auto prepare_stage = [&](int st) {
    const int b = st & 1;
    const int cnt = min(STAGE, l_end - (l_begin + st * STAGE));
    bool need = false, pairable = false;
    const TileRec* src = nullptr;
    int kind = -1;
    if (tid < cnt) {
      const ToneRec& tr = s_tone[b][tid];
      Desc d;
      const bool ramp = (tr.flags & TONE_AMP_RAMP) != 0;
      d.A = (ramp && T0 >= tr.a_ns + tr.a_L) ? tr.A_end : tr.A;
      d.c = d.s = 0.f;
      const int tcls = classify_tile(tr, T0);
      const bool exact = (tr.flags & TONE_EXACT) != 0;
      if (tcls == TILE_PRE || tcls == TILE_POST) {
        const bool pre = tcls == TILE_PRE;
        d.F = pre ? tr.F : tr.F_end;
        d.p0 = (pre ? tr.phi_ref : tr.phi_post_ref) + (uint64_t)T0 * d.F;
        if (a.sine_mode == SINE_ROTATOR) {
          d.c = pre ? tr.rot_c : tr.rot_c_end;
          d.s = pre ? tr.rot_s : tr.rot_s_end;
        }
      } else {
        d.F = 0;
        d.p0 = 0;
        if (!exact) {
          need = true;
          src = a.recs + (int64_t)a.act_of_slot[tr.slot] * (a.rec_stride ? a.rec_stride : a.n_tiles) + a.rec_tile0 + tile;
        }
      }
      // a ramp inside the tile takes the general per-sample path; static segments the engine sums
      // are skipped
      d.kind = tile_kind(tr, T0, a.skip_static != 0);
      if (d.kind == DESC_STATIC && a.sine_mode == SINE_ROTATOR) d.kind = DESC_STATIC_ROT;
      s_desc[b][tid] = d;
      kind = d.kind;
      pairable = (tr.flags & TONE_PAIR) && !a.skip_static;
    }
    // visit order: the chirps that cover the tile in linear form, those in LOW6 form, the static
    // tones (SFU or rotator), then the rest; tone order within each group.  The first three
    // groups run in loops without a per-tone dispatch.  The order of the FP32 sums then depends
    // on which tones share a stage; with a tone list (the window's listed tones) that changes with
    // the window, so listed renders keep plain tone order, and every window cut gives the same bits.
    const int grp = visit_group(kind, a.tone_list != nullptr, pairable);
    const unsigned below = (1u << tid) - 1u;
    int pos = 0, end = 0;
#pragma unroll
    for (int g = 0; g < N_GRP; ++g) {
      const unsigned m = __ballot_sync(0xffffffffu, tid < cnt && grp == g);
      if (grp == g) pos = end + __popc(m & below);
      end += __popc(m);
      if (tid == 0 && g < N_GRP - 1) s_ngrp[b][g] = end;
    }
    if (tid < cnt) s_order[b][pos] = (uint8_t)tid;
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&s_bar[2 + b], (uint32_t)__popc(mask) * (uint32_t)sizeof(TileRec));
      issued += 1u << (8 * (2 + b));
    }
    __syncwarp();
    if (need) bulk_g2s(&s_rec[b][tid], src, (uint32_t)sizeof(TileRec), &s_bar[2 + b]);
  };

  bool ok = true;
  if (n_stages > 0) {
    if (tid < 32) {
      issue_tones(0);
      if (n_stages > 1) issue_tones(1);
    }
    if (tid < 32) {
      ok &= mbar_wait(&s_bar[0], 0);
      prepare_stage(0);
    }
    __syncthreads();   // stage-0 descriptors visible
  }
  int fail_stage = -1;
  const RunBin rb0 = run_binomials(tid);
  for (int st = 0; st < n_stages; ++st) {
    const int b = st & 1;
    const uint32_t par = (uint32_t)((st >> 1) & 1);
    if (tid < 32 && st + 1 < n_stages) {
      ok &= mbar_wait(&s_bar[(st + 1) & 1], (uint32_t)(((st + 1) >> 1) & 1));
      prepare_stage(st + 1);
    }
    ok &= mbar_wait(&s_bar[b], par);
    ok &= mbar_wait(&s_bar[2 + b], par);
    // the same decision in every lane of the warp: the loops below exchange values between lanes
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      const int cnt = min(STAGE, l_end - (l_begin + st * STAGE));
      const int e_lp = s_ngrp[b][GRP_LIN_PAIR], e_lin = s_ngrp[b][GRP_LIN], e_l3p = s_ngrp[b][GRP_LOW3_PAIR],
                e_l6p = s_ngrp[b][GRP_LOW6_PAIR], e_low6 = s_ngrp[b][GRP_LOW6], e_static = s_ngrp[b][GRP_STATIC];
      auto linear = [&](int i) { cascade<0, RUN, false>(poly_state(s_rec[b][i], rb0, true), s_desc[b][i].A, acc); };
      // LOW6, FLAT3: the third difference rounds to 0 everywhere (set-up bound), g is constant
      auto low6 = [&](int i) { cascade<0, RUN, false>(poly_state_low6(s_rec[b][i], rb0), s_desc[b][i].A, acc); };
      auto low3 = [&](int i) { cascade<0, RUN, false>(poly_state_low3(s_rec[b][i], rb0), s_desc[b][i].A, acc); };
      auto flat3 = [&](int i) { cascade<0, RUN, false>(poly_state_flat3(s_rec[b][i], rb0), s_desc[b][i].A, acc); };
      auto static_sfu = [&](int i) {
        const Desc& d = s_desc[b][i];
        static_loop<0, RUN>((uint32_t)((mac_u32(d.p0 + P_OFFSET, d.F, run_off)) >> 32) + HALF_TURN, static_f(d.F), d.A, acc);
      };
      auto static_rot = [&](int i) {
        // the exact phase word at the run start, SFU sine and cosine once, then 31 rotations by
        // the per-sample step on the FP32 pipe (amplitude folded into the phasor)
        const Desc& d = s_desc[b][i];
        const float c = d.c, s = d.s;
        const uint64_t w = d.p0 + (uint64_t)run_off * d.F;
        float sn, cs;
        __sincosf((float)(int32_t)(w >> 32) * 1.46291807926715968e-9f, &sn, &cs);   // 2 pi / 2^32
        float im = d.A * sn, re = d.A * cs;
#pragma unroll
        for (int r = 0; r < RUN; ++r) {
          if (r & 1) acc[r / 2].y += im;
          else acc[r / 2].x += im;
          const float t = fmaf(re, c, -im * s);
          im = fmaf(re, s, im * c);
          re = t;
        }
      };
      // the sharing groups two tones at a time: one set-up per lane, the other tone's state from the
      // partner lane (partner_state); per sample the first tone's multiply-add, then the second's,
      // as in two single loops; an odd group's last tone alone
      const bool odd = (tid & 1) != 0;
      for (int o = 0; o + 1 < e_lp; o += 2) {
        const int i = s_order[b][o], k = s_order[b][o + 1];
        const RunPoly own = poly_state(s_rec[b][odd ? k : i], rb0, true);
        const RunPoly oth = partner_state(own, odd);
        cascade<0, RUN, false>(odd ? oth : own, s_desc[b][i].A, acc);
        cascade<0, RUN, false>(odd ? own : oth, s_desc[b][k].A, acc);
      }
      for (int o = e_lp & ~1; o < e_lin; ++o) linear(s_order[b][o]);
      for (int o = e_lin; o + 1 < e_l3p; o += 2) {
        const int i = s_order[b][o], k = s_order[b][o + 1];
        const RunPoly own = poly_state_low3(s_rec[b][odd ? k : i], rb0);
        const RunPoly oth = partner_state(own, odd);
        cascade<0, RUN, false>(odd ? oth : own, s_desc[b][i].A, acc);
        cascade<0, RUN, false>(odd ? own : oth, s_desc[b][k].A, acc);
      }
      if ((e_l3p - e_lin) & 1) low3(s_order[b][e_l3p - 1]);
      for (int o = e_l3p; o + 1 < e_l6p; o += 2) {
        const int i = s_order[b][o], k = s_order[b][o + 1];
        const RunPoly own = poly_state_low6(s_rec[b][odd ? k : i], rb0);
        const RunPoly oth = partner_state(own, odd);
        cascade<0, RUN, false>(odd ? oth : own, s_desc[b][i].A, acc);
        cascade<0, RUN, false>(odd ? own : oth, s_desc[b][k].A, acc);
      }
      for (int o = e_l3p + ((e_l6p - e_l3p) & ~1); o < e_low6; ++o) low6(s_order[b][o]);
      if (a.sine_mode == SINE_ROTATOR) {
        for (int o = e_low6; o < e_static; ++o) static_rot(s_order[b][o]);
      } else {
        for (int o = e_low6; o < e_static; ++o) static_sfu(s_order[b][o]);
      }
      for (int o = e_static; o < cnt; ++o) {
        const int i = s_order[b][o];
        const Desc& d = s_desc[b][i];
        const int kind = d.kind;
        const float A = d.A;
        if (kind == DESC_SKIP) continue;
        if (kind == DESC_STATIC) {
          static_sfu(i);
        } else if (kind == DESC_STATIC_ROT) {
          static_rot(i);
        } else if (kind == DESC_LINEAR) {
          linear(i);
        } else if (kind == DESC_LOW6) {
          low6(i);
        } else if (kind == DESC_LOW3) {
          low3(i);
        } else if (kind == DESC_FLAT3) {
          flat3(i);
        } else if (kind == DESC_MINJERK) {
          // third difference below 2^-33 turn (long ramps): g is constant over the run, the same
          // integers as the loop with h
          const RunPoly q0 = poly_state(s_rec[b][i], rb0, false);
          if (__all_sync(0xffffffffu, q0.h == 0)) cascade<0, RUN, false>(q0, A, acc);
          else cascade<0, RUN, true>(q0, A, acc);
        } else {
          if constexpr (CLUSTER) tone_run(s_tone[b][i], &s_rec[b][i], rb0, &s_red[tid], acc, T0, n0, a.exact_tab, RUNS);
          else tone_run(s_tone[b][i], &s_rec[b][i], rb0, lcol, acc, T0, n0, a.exact_tab, 1);
        }
      }
    }
    if (!__syncthreads_and(ok)) {   // stage buffers free, next stage's descriptors visible
      fail_stage = st;
      break;
    }
    if (tid < 32 && st + 2 < n_stages) issue_tones(st + 2);
  }
  if (fail_stage >= 0) {
    // report, then let every copy still in flight land (bounded) before shared memory goes away
    if (tid == 0) {
      atomicExch(a.status, STATUS_TIMEOUT);
      for (int bb = 0; bb < 4; ++bb) {
        const uint32_t cnt_b = (issued >> (8 * bb)) & 0xffu;
        if (cnt_b > 0) (void)mbar_wait(&s_bar[bb], (cnt_b - 1) & 1u);
      }
    }
    __syncthreads();
  }

  if constexpr (!CLUSTER) {
    tile_epilogue_split(a, tile, crank, split, T0, acc);
  } else {
    // partial sums -> shared memory ([i][thread], sample RUN thread + i), then the cluster-wide
    // sum in rank order
#pragma unroll
    for (int r = 0; r < RUN / 2; ++r) {
      s_red[(2 * r) * RT + tid] = acc[r].x;
      s_red[(2 * r + 1) * RT + tid] = acc[r].y;
    }
    cluster.sync();

    // this CTA reduces and stores samples [lo, hi) of the tile; thread t takes `per` consecutive ones
    const int lo = (int)((int64_t)TILE * crank / split), hi = (int)((int64_t)TILE * (crank + 1) / split);
    const int per = (hi - lo + RT - 1) / RT;
    const int s_first = lo + tid * per;
    float xs[RUN];
#pragma unroll
    for (int u = 0; u < RUN; ++u) xs[u] = 0.f;
    for (int c = 0; c < split; ++c) {
      const float* rem = cluster.map_shared_rank(s_red, c);
#pragma unroll
      for (int u = 0; u < RUN; ++u) {
        const int sidx = s_first + u;
        if (u < per && sidx < hi) xs[u] += rem[(sidx % RUN) * RT + sidx / RUN];
      }
    }
    cluster.sync();   // remote reads done before any CTA of the cluster exits

    // scale, round half to even, clamp, store the window part
#pragma unroll
    for (int u = 0; u < RUN; ++u) {
      const int sidx = s_first + u;
      if (u < per && sidx < hi) store_sample(a, T0 + sidx, xs[u]);
    }
    if (a.exit_ctr) {   // this CTA's samples are stored and visible
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.exit_ctr, 1ull);
    }
  }
}

// 96 registers: five CTAs of RT threads per SM (the cluster and batched renders)
#define AWG_RENDER_MIN_BLOCKS 5
// The direct render: seven CTAs per SM (72 registers, some spills, 20 KB of shared memory each) ran
// the 1000-chirp record 1.6 % faster than six and six 1.6 % faster than five; the batched render
// of the served stream, whose spills grow more, stays at five.
#define AWG_RENDER_SPLIT_MIN_BLOCKS 7
__global__ void __launch_bounds__(RT, AWG_RENDER_MIN_BLOCKS) render_kernel(const __grid_constant__ RenderArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  render_tile<true>(a, blockIdx.x / a.split, (int)cluster.block_rank(), a.split);
}

// The same without clusters (a.part set): CTA blockIdx.x takes rank blockIdx.x % split.
__global__ void __launch_bounds__(RT, AWG_RENDER_SPLIT_MIN_BLOCKS) render_split_kernel(const __grid_constant__ RenderArgs a) {
  render_tile<false>(a, blockIdx.x / a.split, blockIdx.x % a.split, a.split);
}

// Several renders in one grid (continuous batching): CTA group i (split CTAs) renders window tile
// items[i].y of request items[i].x; every request of the launch has the same tone split.  The
// split sums through each request's scratch (reqs[i].part and .tile_ctr, counters zero at
// launch); CTA blockIdx.x takes rank blockIdx.x % split.
__global__ void __launch_bounds__(RT, AWG_RENDER_MIN_BLOCKS) render_batch_split_kernel(const RenderArgs* __restrict__ reqs,
                                                                                       const int2* __restrict__ items,
                                                                                       int split) {
  const int2 it = items[blockIdx.x / split];
  render_tile<false>(reqs[it.x], it.y, (int)(blockIdx.x % split), split);
}

// The 32-bit phase the render feeds to the sine for sample s of the tile [T0, T0 + TILE) (any
// segment), by the same integer steps as the render's loops: run j = s / RUN, sample r = s % RUN.
// role: 0 the tone's own run set-up, 1 / 2 the first / second tone of a lane pair sharing its
// set-up (the first tone's state is the odd lanes' partner state, the second's the even lanes').
__device__ __noinline__ uint32_t phase32_at(const ToneRec& t, const TileRec* rec, const ChirpRec* chirps, int64_t T0,
                                            int s, const uint64_t (*inv)[3], int role = 0) {
  const int j = s / RUN, r = s % RUN;
  const int64_t n0 = T0 + (int64_t)j * RUN, n = T0 + s;
  const uint32_t ur = (uint32_t)r;
  const uint32_t c2 = ur * (ur - 1) / 2, c3 = (r >= 3) ? ur * (ur - 1) * (ur - 2) / 6 : 0u;
  if (t.slot < 0 || n < t.n_s) return static_p0(t.phi_ref, t.F, n0) + ur * static_f(t.F);
  if (n > t.n_e) return static_p0(t.phi_post_ref, t.F_end, n0) + ur * static_f(t.F_end);
  if (t.flags & TONE_EXACT) return (uint32_t)((exact_chirp_word(chirps[t.slot], n - t.n_s, inv) + P_OFFSET) >> 32);
  const bool ramp_in_tile = (t.flags & TONE_AMP_RAMP) && T0 + TILE - 1 > t.a_ns && T0 < t.a_ns + t.a_L;
  const bool inside = T0 >= t.n_s && T0 + TILE - 1 <= t.n_e;
  RunPoly q;
  if (!ramp_in_tile && inside) {   // the tile's kind decides the set-up (LOW6 leaves terms out)
    const int kind = chirp_inside_kind(t.flags);
    const bool odd = (j & 1) != 0;
    // a shared set-up: the lane of the other parity evaluated it one run away
    const bool moved = (role == 1 && odd) || (role == 2 && !odd);
    const int js = moved ? (odd ? j - 1 : j + 1) : j;
    const RunBin b = run_binomials(js);
    q = kind == DESC_LOW3 ? poly_state_low3(*rec, b)
        : kind == DESC_LOW6 ? poly_state_low6(*rec, b)
        : kind == DESC_FLAT3 ? poly_state_flat3(*rec, b) : poly_state(*rec, b, kind == DESC_LINEAR);
    if (moved) {
      if (odd) {
        q.p = q.p + 32u * q.f + 496u * q.g;
        q.f = q.f + 32u * q.g;
      } else {
        q.p = q.p - 32u * q.f + 528u * q.g;
        q.f = q.f - 32u * q.g;
      }
    }
  } else {
    const RunBin b = run_binomials(j);
    q = poly_state(*rec, b, (t.flags & TONE_LINEAR) != 0);
  }
  return q.p - HALF_TURN + ur * q.f + c2 * q.g + c3 * q.h;
}

// Exact phase words of the first n tones at one sample (test hook).
__global__ void phase_words_kernel(const __grid_constant__ PhaseArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  a.out[k] = exact_word(a.tones[k], a.chirps, a.sample, a.inv_odd);
}

// Exact per-sample 32-bit phases of a short chirp (TONE_EXACT), m = 0..L.
__global__ void exact_table_kernel(const __grid_constant__ TableArgs a, int64_t L) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m > L) return;
  a.out[m] = (uint32_t)((exact_chirp_word(a.chirps[a.slot], m, a.inv_odd) + P_OFFSET) >> 32);
}

// Whether tone k shares its run set-up in tile T0 of a render without a tone list or the tensor-
// core engine, by the render's own visit: the CTA whose tone range [K c / split, K (c + 1) / split)
// holds k, its stage of STAGE tones, and k's place among the stage's tones of its sharing group
// (in tone order, taken two at a time).  0: own set-up, 1 / 2: first / second tone of a pair.
__device__ __noinline__ int pair_role(const TraceArgs& a, int k, int64_t T0) {
  if (a.listed || !(a.tones[k].flags & TONE_PAIR)) return 0;
  const int g = visit_group(tile_kind(a.tones[k], T0, false), false, true);
  if (g != GRP_LIN_PAIR && g != GRP_LOW3_PAIR && g != GRP_LOW6_PAIR) return 0;
  const int64_t K = a.K, S = a.split;
  int c = (int)((int64_t)k * S / K);
  while (c + 1 < S && K * (c + 1) / S <= k) ++c;
  while (c > 0 && K * c / S > k) --c;
  const int lb = (int)(K * c / S), le = (int)(K * (c + 1) / S);
  const int s0 = lb + (k - lb) / STAGE * STAGE, s1 = min(s0 + STAGE, le);
  int pos = 0, n = 0;
  for (int u = s0; u < s1; ++u) {
    const ToneRec& t = a.tones[u];
    if (visit_group(tile_kind(t, T0, false), false, (t.flags & TONE_PAIR) != 0) != g) continue;
    if (u == k) pos = n;
    ++n;
  }
  if (pos & 1) return 2;
  return pos + 1 < n ? 1 : 0;
}

// The render's per-sample 32-bit phases of one tone (test hook).
__global__ void trace_kernel(const __grid_constant__ TraceArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int64_t n = a.n0 + i;
  const int64_t tile_abs = n / TILE;
  const int64_t T0 = tile_abs * TILE;
  const ToneRec t = a.tones[a.tone];
  const TileRec* rec = nullptr;
  if (classify_tile(t, T0) == TILE_CHIRP && !(t.flags & TONE_EXACT))
    rec = a.recs + (int64_t)a.act_of_slot[t.slot] * a.n_tiles + (tile_abs - a.tile0);
  a.out[i] = phase32_at(t, rec, a.chirps, T0, (int)(n - T0), a.inv_odd, pair_role(a, a.tone, T0));
}

}  // namespace

int device_sm_count() {
  constexpr int MAX_DEV = 64;
  static std::atomic<int> cache[MAX_DEV];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return 1;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

cudaError_t render_setup_attributes() {
  cudaError_t e = cudaFuncSetAttribute(render_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  // shared memory before L1 for AWG_RENDER_SPLIT_MIN_BLOCKS CTAs
  if (e == cudaSuccess) e = cudaFuncSetAttribute(render_split_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

cudaError_t launch_render_batch_split(const RenderArgs* reqs, const int2* items, int n_items, int split,
                                      cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  render_batch_split_kernel<<<(unsigned)(n_items * split), RT, 0, s>>>(reqs, items, split);
  return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
  const int64_t total = (int64_t)a.n_active * a.n_tiles;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 127) / 128);
  if (a.n_active <= SMALL_PREP) {   // the small parameter form: fewer bytes copied with the launch
    PrepArgsT<SMALL_PREP> b;
    b.chirps = a.chirps;
    b.recs = a.recs;
    b.act_of_slot = a.act_of_slot;
    b.tile0 = a.tile0;
    b.n_tiles = a.n_tiles;
    b.n_active = a.n_active;
    b.act_base = a.act_base;
    for (int q = 0; q < 7; ++q)
      for (int i = 0; i < 7; ++i) b.W[q][i] = a.W[q][i];
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < 3; ++i) b.inv_odd[q][i] = a.inv_odd[q][i];
    for (int i = 0; i < a.n_active; ++i) b.slots[i] = a.slots[i];
    prep_kernel<PrepArgsT<SMALL_PREP>><<<blocks, 128, 0, s>>>(b);
  } else {
    prep_kernel<PrepArgs><<<blocks, 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Replay of a periodic record (period mask + 1 = 2^log2 samples): out[i * stride] =
// table[(c + i) mod period].  16-byte vectors when the stride is 1 and both sides are aligned
// to 8 samples (a vector never wraps: the period is a multiple of 8).
__global__ void replay_kernel(const int16_t* __restrict__ tab, uint64_t mask, int64_t c, int64_t n,
                              int16_t* __restrict__ out, int32_t stride, int vec) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (vec) {
    // four 16-byte vectors in flight per thread; streaming stores keep the table resident in L2
    const int64_t nv = n / 8;
    for (int64_t v0 = t0; v0 < nv; v0 += 4 * step) {
      uint4 x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t v = v0 + j * step;
        if (v < nv) x[j] = __ldg(reinterpret_cast<const uint4*>(tab + (((uint64_t)c + (uint64_t)v * 8u) & mask)));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t v = v0 + j * step;
        if (v < nv) __stcs(reinterpret_cast<uint4*>(out) + v, x[j]);
      }
    }
    done = nv * 8;
  }
  for (int64_t i = done + t0; i < n; i += step) out[i * stride] = tab[((uint64_t)c + (uint64_t)i) & mask];
}

cudaError_t launch_replay(const int16_t* tab, int32_t log2_len, int64_t c, int64_t n, int16_t* out, int32_t stride,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const uint64_t mask = ((uint64_t)1 << log2_len) - 1;
  const int vec = stride == 1 && (c & 7) == 0 && ((uintptr_t)out & 15) == 0 && log2_len >= 3;
  const int64_t work = vec ? n / 8 + 1 : n;
  const int64_t blocks = std::min<int64_t>((work + 255) / 256, (int64_t)device_sm_count() * 16);
  replay_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(tab, mask, c, n, out, stride, vec);
  return cudaGetLastError();
}

// End of a pipelined sequence: returns once every render CTA of the sequence has stored its
// samples (*exit_ctr >= target), so that later work in the stream sees all of them.  Gives up after
// limit_ns, sets the status word to AWG_ETIMEOUT and returns.
__global__ void join_kernel(const unsigned long long* exit_ctr, unsigned long long target, int32_t* status,
                            uint64_t limit_ns) {
  if (!wait_counter(exit_ctr, target, limit_ns)) atomicExch(status, STATUS_TIMEOUT);
  __threadfence();
}

cudaError_t launch_join(const unsigned long long* exit_ctr, unsigned long long target, int32_t* status,
                        uint64_t limit_ns, cudaStream_t s) {
  join_kernel<<<1, 1, 0, s>>>(exit_ctr, target, status, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t s) {
  if (a.n_tiles == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_tiles * a.split), 1, 1);
  cfg.blockDim = dim3(RT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  if (a.part) {   // no cluster: the split sums through the scratch partials
    cfg.attrs = attr + 1;
    cfg.numAttrs = a.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, render_split_kernel, a);
  }
  cfg.attrs = attr;
  cfg.numAttrs = a.pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, render_kernel, a);
}

cudaError_t launch_exact_table(const TableArgs& a, int64_t L, cudaStream_t s) {
  const int64_t n = L + 1;
  exact_table_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a, L);
  return cudaGetLastError();
}

cudaError_t launch_phase_words(const PhaseArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  phase_words_kernel<<<(a.n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  trace_kernel<<<(a.count + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// The rate the SFU sustains in the render's own static loop (a measured ceiling for the sine
// roofline): every thread runs `runs` runs of RUN samples of one static tone through static_loop,
// with no staging, set-up or split sum, and writes the sum of its partial sums (so that nothing
// is optimised away).  One sine per sample: blocks x RT x runs x RUN sines per launch.
__global__ void __launch_bounds__(RT, AWG_RENDER_MIN_BLOCKS) sfu_rate_kernel(float* __restrict__ out, int runs) {
  const uint32_t id = blockIdx.x * RT + threadIdx.x;
  uint32_t p = id * 0x9E3779B9u;
  const uint32_t f = (id * 0x85EBCA6Bu) | 1u;
  const float A = 1e-3f;
  Acc acc;
#pragma unroll
  for (int r = 0; r < RUN / 2; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int k = 0; k < runs; ++k) {
    static_loop<0, RUN>(p, f, A, acc);
    p += (uint32_t)RUN * f;
  }
  float t = 0.f;
#pragma unroll
  for (int r = 0; r < RUN / 2; ++r) t += acc[r].x + acc[r].y;
  out[id] = t;
}

cudaError_t launch_sfu_rate(float* out, int blocks, int runs, cudaStream_t s) {
  sfu_rate_kernel<<<blocks, RT, 0, s>>>(out, runs);
  return cudaGetLastError();
}

// The same for the render's chirp loop (cascade without h, the loop of linear and LOW6 chirps):
// each run takes a chirp state (p, f, g) from the thread's id, one sine per sample.
__global__ void __launch_bounds__(RT, AWG_RENDER_MIN_BLOCKS) chirp_rate_kernel(float* __restrict__ out, int runs) {
  const uint32_t id = blockIdx.x * RT + threadIdx.x;
  RunPoly q;
  q.p = id * 0x9E3779B9u;
  q.f = (id * 0x85EBCA6Bu) | 1u;
  q.g = (id * 0xC2B2AE35u) >> 8;
  q.h = 0;
  const float A = 1e-3f;
  Acc acc;
#pragma unroll
  for (int r = 0; r < RUN / 2; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int k = 0; k < runs; ++k) {
    cascade<0, RUN, false>(q, A, acc);
    q.p += 32u * q.f + 496u * q.g;   // the state after the run
    q.f += 32u * q.g;
  }
  float t = 0.f;
#pragma unroll
  for (int r = 0; r < RUN / 2; ++r) t += acc[r].x + acc[r].y;
  out[id] = t;
}

cudaError_t launch_chirp_rate(float* out, int blocks, int runs, cudaStream_t s) {
  chirp_rate_kernel<<<blocks, RT, 0, s>>>(out, runs);
  return cudaGetLastError();
}

}  // namespace awgk
