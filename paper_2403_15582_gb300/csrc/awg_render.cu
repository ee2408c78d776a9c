// Render kernels for multi-tone additive synthesis on sm_103a.
//
//   x[n] = sum_k A_k sin(2 pi Phi_k(n) / 2^64)       (Eq. main / Eq. dynamicandstatic)
//
// Phase words.  Static tones: Phi(n) = phi_ref + n F.  Chirps (Eq. freqchirp, linear or
// minimum-jerk): Phi(n_s + m) = Phi(n_s) + top64(sum_k d_k C(m,k)) with the 192-bit forward
// differences d_k set up on the host; evaluated here exactly by the closed form
// (exact_chirp_word), which is what a sequential 192-bit cascade would produce.
//
// Work decomposition (see awg_internal.h): a CTA renders one tile of TILE = 4096 absolute-aligned
// samples; thread j owns the run of RUN = 32 samples starting at T0 + 32 j and keeps its 32 partial
// sums in registers; the tones are split over the CTAs of a thread-block cluster and the partial
// sums are added through distributed shared memory in a fixed order, then scaled, rounded and
// stored by the same kernel.
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

// top 64 bits of a Q64.128 value, rounded to nearest
__device__ __forceinline__ uint64_t round_top64(U192 a) {
  return add192(a, U192{0, 1ull << 63, 0}).w2;
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

// Exact phase word of a chirp at offset m from its start: Phi(n_s) + top64(sum_i d_i C(m, i)).
// d_0 carries the 2^127 rounding offset.
__device__ uint64_t exact_chirp_word(const ChirpRec& c, int64_t m, const uint64_t (*inv)[3]) {
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

struct RunPoly {
  uint32_t p, f, g, h;
};

// C(j, q) for the run index j (0 <= j < NT), q = 0..6
__device__ __forceinline__ void run_binomials(int j, uint64_t cj[7]) {
  uint64_t u = (uint64_t)j;
  cj[0] = 1;
  cj[1] = u;
  cj[2] = u * (u - 1) / 2;
  cj[3] = cj[2] * (u - 2) / 3;
  cj[4] = cj[3] * (u - 3) / 4;
  cj[5] = cj[4] * (u - 4) / 5;
  cj[6] = cj[5] * (u - 5) / 6;
  // for j < q the product has a zero factor; the unsigned wrap of (u - i) is multiplied by it
  if (j < 2) cj[2] = 0;
  if (j < 3) cj[3] = 0;
  if (j < 4) cj[4] = 0;
  if (j < 5) cj[5] = 0;
  if (j < 6) cj[6] = 0;
}

__device__ __forceinline__ RunPoly poly_state(const TileRec& rc, const uint64_t cj[7]) {
  uint64_t p = rc.B[0], f = 0, g = 0, h = 0;
#pragma unroll
  for (int q = 1; q <= 6; ++q) p += rc.B[q] * cj[q];
#pragma unroll
  for (int q = 0; q <= 5; ++q) f += rc.E[q] * cj[q];
#pragma unroll
  for (int q = 0; q <= 4; ++q) g += rc.G[q] * cj[q];
#pragma unroll
  for (int q = 0; q <= 3; ++q) h += rc.H[q] * cj[q];
  RunPoly r;
  r.p = (uint32_t)((p + P_OFFSET) >> 32);
  r.f = (uint32_t)((f + HALF32) >> 32);
  r.g = (uint32_t)((g + HALF32) >> 32);
  r.h = (uint32_t)((h + HALF32) >> 32);
  return r;
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

// The 32-bit phase the render feeds to the sine for sample r of run j (any segment).  The fast
// loops below produce the same integers by stepping.
__device__ uint32_t phase32_at(const ToneRec& t, const TileRec* rec, const ChirpRec* chirps, int64_t T0,
                               int j, int r, const uint64_t (*inv)[3]) {
  const int64_t n0 = T0 + (int64_t)j * RUN;
  const int64_t n = n0 + r;
  const uint32_t ur = (uint32_t)r;
  if (t.slot < 0 || n < t.n_s) return static_p0(t.phi_ref, t.F, n0) + ur * static_f(t.F);
  if (n > t.n_e) return static_p0(t.phi_post_ref, t.F_end, n0) + ur * static_f(t.F_end);
  if (t.flags & TONE_EXACT) return (uint32_t)((exact_chirp_word(chirps[t.slot], n - t.n_s, inv) + P_OFFSET) >> 32);
  uint64_t cj[7];
  run_binomials(j, cj);
  RunPoly s = poly_state(*rec, cj);
  const uint32_t c2 = ur * (ur - 1) / 2, c3 = (r >= 3) ? ur * (ur - 1) * (ur - 2) / 6 : 0u;
  return s.p + ur * s.f + c2 * s.g + c3 * s.h;
}

// sin(2 pi p / 2^32): the top 23 bits of p, offset by half a turn, become the mantissa of a float
// v in [1, 2); 2 pi (v - 3/2) lies in [-pi, pi) and is congruent to the phase.
__device__ __forceinline__ float sin_turn(uint32_t p) {
  const float v = __uint_as_float((p >> 9) ^ 0x3FC00000u);
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
__global__ void __launch_bounds__(128) prep_kernel(const __grid_constant__ PrepArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)a.n_active * a.n_tiles;
  if (idx >= total) return;
  const int ai = (int)(idx / a.n_tiles);
  const int t = (int)(idx - (int64_t)ai * a.n_tiles);
  const int slot = a.slots[ai];
  const ChirpRec& c = a.chirps[slot];
  if (t == 0) a.act_of_slot[slot] = a.act_base + ai;
  const int64_t T0 = (a.tile0 + t) * (int64_t)TILE;
  const int64_t m = T0 - c.n_s;

  U192 bin[7];
  binomials(m, a.inv_odd, bin);
  // unit-stride forward differences of the phase (Q64.128) at the tile start
  U192 acc[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = k; i < 7; ++i) s = add192(s, mul192(dword(c, i), bin[i - k]));
    acc[k] = s;
  }
  TileRec out;
  // B_q = sum_{i>=q} acc_i W[q][i]; E, G, H: the same for the first, second and third unit
  // differences (acc shifted by 1, 2, 3).
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = q; i < 7; ++i) s = add192(s, mul192(acc[i], from_s64(a.W[q][i])));
    out.B[q] = (q == 0) ? c.phi_start + s.w2 : round_top64(s);   // acc_0 already holds 2^127
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = q; i < 6; ++i) s = add192(s, mul192(acc[i + 1], from_s64(a.W[q][i])));
    out.E[q] = round_top64(s);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = q; i < 5; ++i) s = add192(s, mul192(acc[i + 2], from_s64(a.W[q][i])));
    out.G[q] = round_top64(s);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    U192 s = {0, 0, 0};
#pragma unroll
    for (int i = q; i < 4; ++i) s = add192(s, mul192(acc[i + 3], from_s64(a.W[q][i])));
    out.H[q] = round_top64(s);
  }
  a.recs[(int64_t)(a.act_base + ai) * a.n_tiles + t] = out;
}

// ------------------------------------------------------------------------------------------
// render
// ------------------------------------------------------------------------------------------
constexpr int RED_STRIDE = RUN + 1;   // conflict-free row stride of the per-thread partial sums

__global__ void __launch_bounds__(NT) render_kernel(const __grid_constant__ RenderArgs a) {
  __shared__ alignas(16) ToneRec s_tone[2][STAGE];
  __shared__ alignas(16) TileRec s_rec[STAGE];
  __shared__ alignas(16) float s_red[NT * RED_STRIDE];
  __shared__ alignas(16) int16_t s_q[TILE];
  __shared__ alignas(8) uint64_t s_bar[3];

  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const int split = a.split;
  const int crank = (int)cluster.block_rank();
  const int tile = blockIdx.x / split;
  const int64_t T0 = (a.tile0 + tile) * (int64_t)TILE;
  const int64_t n0 = T0 + (int64_t)tid * RUN;
  const int k_begin = (int)((int64_t)a.K * crank / split);
  const int k_end = (int)((int64_t)a.K * (crank + 1) / split);
  const int n_tones = k_end - k_begin;
  const int n_stages = (n_tones + STAGE - 1) / STAGE;

  uint64_t cj[7];
  run_binomials(tid, cj);

  float acc[RUN];
#pragma unroll
  for (int r = 0; r < RUN; ++r) acc[r] = 0.f;

  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init(&s_bar[2], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue_tones = [&](int st) {
    const int kb = k_begin + st * STAGE;
    const int cnt = min(STAGE, k_end - kb);
    const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(ToneRec);
    fence_proxy_async();
    mbar_arrive_expect_tx(&s_bar[st & 1], bytes);
    bulk_g2s(&s_tone[st & 1][0], a.tones + kb, bytes, &s_bar[st & 1]);
  };
  if (tid == 0 && n_stages > 0) issue_tones(0);

  int fail_stage = -1, fail_kind = 0;   // kind 1: tone copy wait gave up, 2: record wait gave up
  for (int st = 0; st < n_stages; ++st) {
    const int buf = st & 1;
    const int cnt = min(STAGE, k_end - (k_begin + st * STAGE));
    if (tid == 0 && st + 1 < n_stages) issue_tones(st + 1);
    bool w = mbar_wait(&s_bar[buf], (uint32_t)((st >> 1) & 1));
    if (!__syncthreads_and(w)) {
      fail_stage = st;
      fail_kind = 1;
      break;
    }
    // chirp tile records for the tones of this stage that chirp inside this tile
    if (tid < 32) {
      bool need = false;
      const TileRec* src = nullptr;
      if (tid < cnt) {
        const ToneRec& tr = s_tone[buf][tid];
        if (classify_tile(tr, T0) == TILE_CHIRP && !(tr.flags & TONE_EXACT)) {
          need = true;
          src = a.recs + (int64_t)a.act_of_slot[tr.slot] * a.n_tiles + tile;
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, need);
      if (tid == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&s_bar[2], (uint32_t)__popc(mask) * (uint32_t)sizeof(TileRec));
      }
      __syncwarp();
      if (need) bulk_g2s(&s_rec[tid], src, (uint32_t)sizeof(TileRec), &s_bar[2]);
    }
    w = mbar_wait(&s_bar[2], (uint32_t)(st & 1));
    if (!__syncthreads_and(w)) {
      fail_stage = st;
      fail_kind = 2;
      break;
    }

    for (int i = 0; i < cnt; ++i) {
      const ToneRec& tr = s_tone[buf][i];
      const float A = tr.A;
      const int tcls = classify_tile(tr, T0);
      int mode;   // 0 static pre, 1 static post, 2 poly, 3 general
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
      if (mode <= 1) {
        const uint64_t phi = mode == 0 ? tr.phi_ref : tr.phi_post_ref;
        const uint64_t F = mode == 0 ? tr.F : tr.F_end;
        uint32_t p = static_p0(phi, F, n0);
        const uint32_t f = static_f(F);
#pragma unroll
        for (int r = 0; r < RUN; ++r) {
          acc[r] = fmaf(A, sin_turn(p), acc[r]);
          p += f;
        }
      } else if (mode == 2) {
        RunPoly s = poly_state(s_rec[i], cj);
        uint32_t p = s.p, f = s.f, g = s.g;
        const uint32_t h = s.h;
#pragma unroll
        for (int r = 0; r < RUN; ++r) {
          acc[r] = fmaf(A, sin_turn(p), acc[r]);
          p += f;
          f += g;
          g += h;
        }
      } else {
        float* row = &s_red[tid * RED_STRIDE];
        for (int r = 0; r < RUN; ++r)
          row[r] = sin_turn(phase32_at(tr, &s_rec[i], a.chirps, T0, tid, r, a.inv_odd));
#pragma unroll
        for (int r = 0; r < RUN; ++r) acc[r] = fmaf(A, row[r], acc[r]);
      }
    }
    __syncthreads();   // stage buffers and records are reused by the next stage
  }
  if (fail_stage >= 0) {
    // report, then let the copies still in flight land (bounded) before shared memory goes away
    if (tid == 0) {
      atomicExch(a.status, STATUS_TIMEOUT);
      const int st = fail_stage;
      if (fail_kind == 1) (void)mbar_wait(&s_bar[st & 1], (uint32_t)((st >> 1) & 1));
      if (st + 1 < n_stages) (void)mbar_wait(&s_bar[(st + 1) & 1], (uint32_t)(((st + 1) >> 1) & 1));
      if (fail_kind == 2) (void)mbar_wait(&s_bar[2], (uint32_t)(st & 1));
    }
    __syncthreads();
  }

  // partial sums -> shared memory, then cluster-wide reduction in rank order
  {
    float* row = &s_red[tid * RED_STRIDE];
#pragma unroll
    for (int r = 0; r < RUN; ++r) row[r] = acc[r];
  }
  cluster.sync();

  const int slice = TILE / split;          // samples reduced and stored by this CTA
  const int per = slice / NT;              // per thread (32 / split, >= 2)
  const int s_first = crank * slice + tid * per;
  float xs[RUN];
#pragma unroll
  for (int u = 0; u < RUN; ++u) xs[u] = 0.f;
  for (int c = 0; c < split; ++c) {
    const float* rem = cluster.map_shared_rank(s_red, c);
#pragma unroll
    for (int u = 0; u < RUN; ++u) {
      if (u < per) {
        const int s = s_first + u;
        xs[u] += rem[(s / RUN) * RED_STRIDE + (s % RUN)];
      }
    }
  }
  cluster.sync();   // remote reads done; shared memory may be reused

  // scale, round half to even, clamp, stage, then coalesced stores of the window part
#pragma unroll
  for (int u = 0; u < RUN; ++u) {
    if (u < per) {
      const int s = s_first + u - crank * slice;
      float q = rintf(xs[u] * a.scale);
      q = fminf(fmaxf(q, -32767.f), 32767.f);
      s_q[s] = (int16_t)q;
      if (a.out_f) s_red[s] = xs[u];
    }
  }
  __syncthreads();
  const int64_t base = T0 + (int64_t)crank * slice;
  for (int i = tid; i < slice; i += NT) {
    const int64_t n = base + i;
    if (n >= a.win_start && n < a.win_end) {
      if (a.out_q) a.out_q[n - a.win_start] = s_q[i];
      if (a.out_f) a.out_f[n - a.win_start] = s_red[i];
    }
  }
}

// Exact phase words of the first n tones at one sample (test hook).
__global__ void phase_words_kernel(const __grid_constant__ PhaseArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  a.out[k] = exact_word(a.tones[k], a.chirps, a.sample, a.inv_odd);
}

// The render's per-sample 32-bit phases of one tone (test hook).
__global__ void trace_kernel(const __grid_constant__ TraceArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int64_t n = a.n0 + i;
  const int64_t tile_abs = n / TILE;
  const int64_t T0 = tile_abs * TILE;
  const int j = (int)((n - T0) / RUN);
  const int r = (int)((n - T0) % RUN);
  const ToneRec t = a.tones[a.tone];
  const TileRec* rec = nullptr;
  if (classify_tile(t, T0) == TILE_CHIRP && !(t.flags & TONE_EXACT))
    rec = a.recs + (int64_t)a.act_of_slot[t.slot] * a.n_tiles + (tile_abs - a.tile0);
  a.out[i] = phase32_at(t, rec, a.chirps, T0, j, r, a.inv_odd);
}

}  // namespace

cudaError_t render_setup_attributes() {
  return cudaFuncSetAttribute(render_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
  const int64_t total = (int64_t)a.n_active * a.n_tiles;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 127) / 128);
  prep_kernel<<<blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t s) {
  if (a.n_tiles == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_tiles * a.split), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, render_kernel, a);
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

}  // namespace awgk
