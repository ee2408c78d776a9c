// Periodic multi-tone table as a split-precision tensor-core GEMM (tcgen05, sm_103a).
//
// For tones on the f_s / 2^log2_len grid (Eq. freqapprox) the record of N = 2^log2_len samples is
// periodic.  With n = n1 * NB + n2 (NB = 256) and the angle-addition identity,
//   x[n] = sum_k A_k sin(a_k(n1) + b_k(n2))
//        = sum_k [A_k sin a_k(n1)] cos b_k(n2) + [A_k cos a_k(n1)] sin b_k(n2),
// a_k(n1) = 2 pi (Phi0_k + n1 NB F_k) / 2^64 and b_k(n2) = 2 pi n2 F_k / 2^64 from exact 64-bit
// phase words.  That is a GEMM X[M = N/NB, NB] = Aop[M, 2K] * Bop[2K, NB].  Each operand is split
// into hi + lo in BF16 (or FP16); the kernel accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor
// memory and quantises in the epilogue.
//
// Kernel structure: a cluster of S CTAs per 128-row tile of X splits the K dimension (fewer FP32
// accumulations per chain); each CTA (320 threads) has a 2-stage ring of
// {A_hi, A_lo (128 x 64), B_hi, B_lo (256 x 64)} tiles in the 128-byte-swizzled K-major layout:
//   warp 0   TMA producer of the B tiles (prepared once per call, 256 x 2K, L2-resident),
//            mbarrier transaction counts
//   warp 1   allocates 512 TMEM columns; lane 0 issues tcgen05.mma (M 128, N 256, K 16) x 3 passes
//            x 4 k-steps per stage, commits each stage back to the producers
//   warps 2-9 generate the A tiles in shared memory (one tone per lane, every eighth row per warp:
//            A_k sin a_k(n1), A_k cos a_k(n1) from the exact phase word, SFU sine and cosine, hi + lo
//            split), so the M x 2K A
//            operand never exists in HBM; then the epilogue: tcgen05.ld 32x32b of both
//            accumulators (warp w reads TMEM lane quarter w mod 4, half of the columns) into a
//            padded FP32 partial tile in shared memory; the cluster sums the S
//            partial tiles through distributed shared memory in rank order, and each CTA scales,
//            rounds, clamps and stores its rows.
// Every wait is bounded (about 2 s); on a timeout the CTA records AWG_ETIMEOUT, lets in-flight
// copies and MMAs drain (bounded), frees its TMEM and exits.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "awg_internal.h"

namespace cg = cooperative_groups;

namespace awgk {

namespace {

constexpr int TM = 128;               // rows of X per CTA (UMMA M)
constexpr int TN = 256;               // NB: columns of X (UMMA N)
constexpr int TK = 64;                // K elements per stage (128 bytes of 16-bit values)
constexpr int NSTAGE = 2;
// A-operand generator warps (rows g, g + NGEN, ...): eight keep the tensor pipe fed (four left the
// MMAs waiting for the A tiles: 1.44 -> 1.29 ms on the 10,000-tone 2^24 table; sixteen, no faster)
constexpr int NGEN = 8;
constexpr int GEMM_THREADS = 32 * (2 + NGEN);
static_assert(NGEN % 4 == 0 && TM % NGEN == 0, "generator warps cover every TMEM lane quarter and every row");
constexpr uint32_t A_TILE = TM * TK * 2;   // 16 KB
constexpr uint32_t B_TILE = TN * TK * 2;   // 32 KB
constexpr uint32_t STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;   // 96 KB
constexpr int STATUS_TIMEOUT = -4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (!mbar_try(bar, parity))
    if (now_ns() - t0 > 2000000000ull) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile with 128-byte rows, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

constexpr int PART_STRIDE = TN + 1;   // padded row of a partial tile (conflict-free column writes)

struct TableGemmArgs {
  int32_t n_kb;          // K blocks of TK (all CTAs of a cluster together)
  int16_t* out_q;
  float* out_f;
  float scale;           // 32767 / FS
  int32_t* status;
  uint32_t idesc;
  const ToneRec* tones;  // A operand source: phase word, frequency word, amplitude
  int32_t K;
  int32_t nb_log2;       // row n1 starts at sample n1 << nb_log2
  int64_t row_base;      // absolute row of tile row 0 of tile 0
  int64_t win_start, win_end;
  int32_t window_mode;
  float a_scale, inv_a_scale;   // A operand scaling (a power of two) and its inverse
};

template <typename T>
__device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
template <typename T>
__device__ __forceinline__ float2 unpack2(uint32_t u);
template <>
__device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}
template <>
__device__ __forceinline__ float2 unpack2<__half>(uint32_t u) {
  const __half2 v = *reinterpret_cast<const __half2*>(&u);
  return __half22float2(v);
}

// The A tile of one stage for one generator warp: lane j takes tone kt0 + j (its phase word,
// frequency word and amplitude, loaded once), warp g the rows g, g + 4, ..., g + 124; for each row
// n1 it forms the hi and lo halves of (A_k sin a, A_k cos a), a = 2 pi (Phi0_k + n1 NB F_k) / 2^64,
// stepping the exact phase word by 4 NB F_k from row to row.  The pair is one 32-bit word at byte
// 4 (j mod 4) of 16-byte chunk j / 4 of the row, which the 128-byte swizzle moves to chunk
// (j / 4) ^ (row mod 8).  The sine and cosine take the top 32 bits of the phase word as a signed
// turn on the SFU (|error| < 5e-7).
template <typename T, bool WINDOW>
__device__ __forceinline__ void gen_a_tile(const TableGemmArgs& a, int kt0, uint32_t row0, int g, int lane,
                                           uint32_t tile_hi, uint32_t tile_lo) {
  // table mode: lane j = tone kt0 + j (one (sin, cos) pair per tone); static engine: lane j = tone
  // kt0 / 2 + j / 2, segment j % 2 (two pairs per tone), zero in tiles where it is not static
  const int k = WINDOW ? (kt0 >> 1) + (lane >> 1) : kt0 + lane;
  const int seg = lane & 1;
  uint64_t w = 0, step = 0;
  float amp = 0.f;
  // static engine: the tiles [T0, T0 + TILE) where this (tone, segment) is static are those with
  // seg_lo <= T0 <= seg_hi outside (ramp_lo, ramp_hi); amplitude A before the ramp, A_end after
  int64_t seg_lo = 0, seg_hi = -1, ramp_lo = INT64_MAX, ramp_hi = INT64_MIN;
  float amp_end = 0.f;
  if (k < a.K) {
    uint64_t phi, F;
    float A;
    if (WINDOW) {
      const ToneRec& t = a.tones[k];
      phi = seg ? t.phi_post_ref : t.phi_ref;
      F = seg ? t.F_end : t.F;
      A = t.A;
      amp_end = t.A;
      if (seg == 0) {
        seg_lo = INT64_MIN;
        seg_hi = t.slot >= 0 ? t.n_s - TILE : INT64_MAX;      // T0 + TILE - 1 < n_s
      } else if (t.slot >= 0) {
        seg_lo = t.n_e + 1;                                   // T0 > n_e
        seg_hi = INT64_MAX;
      }
      if (t.flags & TONE_AMP_RAMP) {                          // not static: T0 + TILE - 1 > a_ns and T0 < a_ns + a_L
        ramp_lo = t.a_ns - TILE + 2;
        ramp_hi = t.a_ns + t.a_L - 1;
        amp_end = t.A_end;
      }
    } else {
      const ToneRec* t = a.tones + k;
      phi = __ldg(&t->phi_ref);
      F = __ldg(&t->F);
      A = __ldg(&t->A);
    }
    const uint64_t f8 = F << a.nb_log2;
    w = phi + (uint64_t)(a.row_base + (int64_t)row0 + g) * f8;
    step = f8 * (uint64_t)NGEN;
    amp = A * a.a_scale;
    amp_end *= a.a_scale;
  }
  const uint32_t col = (uint32_t)(lane & 3) * 4u;
  const uint32_t chunk = (uint32_t)(lane >> 2);
#pragma unroll 8
  for (int i = 0; i < TM / NGEN; ++i) {
    const uint32_t r = (uint32_t)(g + NGEN * i);
    float sn, cs;
    __sincosf((float)(int32_t)(w >> 32) * 1.46291807926715968e-9f, &sn, &cs);   // 2 pi / 2^32
    float a_row = amp;
    if (WINDOW) {   // the row's tile decides whether this segment is summed here
      const int64_t T0 = ((a.row_base + (int64_t)row0 + (int64_t)r) << a.nb_log2) & ~(int64_t)(TILE - 1);
      const bool in_seg = T0 >= seg_lo && T0 <= seg_hi;
      const bool ramping = T0 >= ramp_lo && T0 <= ramp_hi;
      a_row = (in_seg && !ramping) ? (T0 > ramp_hi ? amp_end : amp) : 0.f;
    }
    const float sv = a_row * sn, cv = a_row * cs;
    const uint32_t hv = pack2<T>(sv, cv);
    const float2 h = unpack2<T>(hv);
    const uint32_t lv = pack2<T>(sv - h.x, cv - h.y);
    const uint32_t off = r * 128u + ((chunk ^ (r & 7u)) << 4) + col;
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(tile_hi + off), "r"(hv) : "memory");
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(tile_lo + off), "r"(lv) : "memory");
    w += step;
  }
}

// Table mode with the lane's tone words already loaded (phi, F, A; zero amplitude past K): the
// same rows as gen_a_tile<T, false>.
template <typename T>
__device__ __forceinline__ void gen_a_rows(const TableGemmArgs& a, uint64_t phi, uint64_t F, float A, uint32_t row0,
                                           int g, int lane, uint32_t tile_hi, uint32_t tile_lo) {
  const uint64_t f8 = F << a.nb_log2;
  uint64_t w = phi + (uint64_t)(a.row_base + (int64_t)row0 + g) * f8;
  const uint64_t step = f8 * (uint64_t)NGEN;
  const uint32_t col = (uint32_t)(lane & 3) * 4u;
  const uint32_t chunk = (uint32_t)(lane >> 2);
#pragma unroll 8
  for (int i = 0; i < TM / NGEN; ++i) {
    const uint32_t r = (uint32_t)(g + NGEN * i);
    float sn, cs;
    __sincosf((float)(int32_t)(w >> 32) * 1.46291807926715968e-9f, &sn, &cs);   // 2 pi / 2^32
    const float sv = A * sn, cv = A * cs;
    const uint32_t hv = pack2<T>(sv, cv);
    const float2 h = unpack2<T>(hv);
    const uint32_t lv = pack2<T>(sv - h.x, cv - h.y);
    const uint32_t off = r * 128u + ((chunk ^ (r & 7u)) << 4) + col;
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(tile_hi + off), "r"(hv) : "memory");
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(tile_lo + off), "r"(lv) : "memory");
    w += step;
  }
}

template <typename T, bool WINDOW>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    table_gemm_kernel(const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
                      const __grid_constant__ TableGemmArgs a) {
  extern __shared__ uint8_t dyn_smem[];
  __shared__ alignas(8) uint64_t bars[2 * NSTAGE + 1];   // full[2], empty[2], done
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_fail;

  cg::cluster_group cluster = cg::this_cluster();
  const int split = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t base = (smem_u32(dyn_smem) + 1023u) & ~1023u;   // 1024-byte aligned stages
  float* part = reinterpret_cast<float*>(dyn_smem + (base - smem_u32(dyn_smem)));   // reuses the stages
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSTAGE]), done = smem_u32(&bars[2 * NSTAGE]);
  const int row0 = (blockIdx.x / split) * TM;
  const int kb0 = (int)((int64_t)a.n_kb * crank / split), kb1 = (int)((int64_t)a.n_kb * (crank + 1) / split);
  const int n_kb = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(full0 + 8 * s, 1 + NGEN);   // the B copies' transaction arrive + one per generator warp
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // whole warp: 512 TMEM columns, two 128 x 256 FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)), "r"(2 * TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int kb = 0; kb < n_kb; ++kb) {
      const int s = kb % NSTAGE;
      if (kb >= NSTAGE && !mbar_wait(empty0 + 8 * s, (uint32_t)(((kb / NSTAGE) - 1) & 1))) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
      mbar_expect_tx(full0 + 8 * s, 2 * B_TILE);
      const int kx = (kb0 + kb) * TK;
      tma_load_2d(st + 2 * A_TILE, &mB_hi, kx, 0, full0 + 8 * s);
      tma_load_2d(st + 2 * A_TILE + B_TILE, &mB_lo, kx, 0, full0 + 8 * s);
      issued = kb + 1;
    }
    if (s_fail) {   // let the copies already issued land (bounded) before the CTA exits
      for (int kb = (issued > NSTAGE ? issued - NSTAGE : 0); kb < issued; ++kb)
        (void)mbar_wait(full0 + 8 * (kb % NSTAGE), (uint32_t)((kb / NSTAGE) & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool ok = true;
    for (int kb = 0; kb < n_kb && ok; ++kb) {
      const int s = kb % NSTAGE;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)((kb / NSTAGE) & 1)) || s_fail) {
        ok = false;
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
      const uint32_t a_hi = st, a_lo = st + A_TILE, b_hi = st + 2 * A_TILE, b_lo = st + 2 * A_TILE + B_TILE;
#pragma unroll
      for (int j = 0; j < TK / 16; ++j) {   // K = 16 per instruction: +32 bytes inside the swizzle atom
        const uint32_t off = 32u * (uint32_t)j;
        const uint32_t first = (kb == 0 && j == 0) ? 0u : 1u;
        // the large products and the small corrections accumulate separately, so the large
        // accumulator takes one rounding per k-step instead of three
        mma_f16(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), a.idesc, first);
        mma_f16(tmem + TN, sw128_desc(a_hi + off), sw128_desc(b_lo + off), a.idesc, first);
        mma_f16(tmem + TN, sw128_desc(a_lo + off), sw128_desc(b_hi + off), a.idesc, 1u);
      }
      mma_commit(empty0 + 8 * s);   // stage free once these MMAs have read it
    }
    mma_commit(done);               // all MMAs issued so far complete -> epilogue (also on abort)
  } else if (warp >= 2) {
    // ---------------- A operand generation ----------------
    {
      const int g = warp - 2;   // rows g, g + NGEN, ...
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % NSTAGE;
        // table mode: this k-block's tone words are loaded before the wait for the stage, so
        // their latency hides under it
        uint64_t phi = 0, F = 0;
        float A = 0.f;
        if (!WINDOW) {
          const int k = (kb0 + kb) * (TK / 2) + lane;
          if (k < a.K) {
            phi = __ldg(&a.tones[k].phi_ref);
            F = __ldg(&a.tones[k].F);
            A = __ldg(&a.tones[k].A) * a.a_scale;
          }
        }
        if (kb >= NSTAGE && !mbar_wait(empty0 + 8 * s, (uint32_t)(((kb / NSTAGE) - 1) & 1))) {
          s_fail = 1;
          break;
        }
        if (s_fail) break;
        const uint32_t st = base + (uint32_t)s * STAGE_BYTES;
        if (WINDOW) gen_a_tile<T, true>(a, (kb0 + kb) * (TK / 2), (uint32_t)row0, g, lane, st, st + A_TILE);
        else gen_a_rows<T>(a, phi, F, A, (uint32_t)row0, g, lane, st, st + A_TILE);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
      }
    }
    // ---------------- epilogue ----------------
    const bool ok = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lane_base = 32 * (warp % 4);          // TMEM lanes this warp may read
    const int row = lane_base + lane;                // row of the tile = TMEM lane
    const bool go = __all_sync(0xffffffffu, ok && !s_fail);   // warp-uniform: tcgen05.ld is .aligned
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // stage memory becomes the partial tile
    // warps with the same lane quarter take consecutive column ranges of the tile
    constexpr int COLS = TN / (NGEN / 4);
    const int c_begin = ((warp - 2) / 4) * COLS;
    if (go) {
#pragma unroll 1
      for (int c0 = c_begin; c0 < c_begin + COLS; c0 += 32) {
        uint32_t v[32], w[32];
        const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
              "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15]),
              "=r"(w[16]), "=r"(w[17]), "=r"(w[18]), "=r"(w[19]), "=r"(w[20]), "=r"(w[21]), "=r"(w[22]), "=r"(w[23]),
              "=r"(w[24]), "=r"(w[25]), "=r"(w[26]), "=r"(w[27]), "=r"(w[28]), "=r"(w[29]), "=r"(w[30]), "=r"(w[31])
            : "r"(taddr + (uint32_t)TN));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) + __uint_as_float(w[i]));
#pragma unroll
        for (int i = 0; i < 32; ++i) part[row * PART_STRIDE + c0 + i] = __uint_as_float(v[i]);
      }
    }
    if (!ok) s_fail = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && s_fail) atomicExch(a.status, STATUS_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
  }
  cluster.sync();   // every partial tile of the cluster is in shared memory

  // this CTA sums rows [r_lo, r_hi) of the S partial tiles in rank order, then quantises and stores
  const int r_lo = TM * crank / split, r_hi = TM * (crank + 1) / split;
  const int n_el = (r_hi - r_lo) * TN;
  for (int e = threadIdx.x; e < n_el; e += blockDim.x) {
    const int row = r_lo + e / TN, col = e % TN;
    float x = 0.f;
    for (int c = 0; c < split; ++c) x += cluster.map_shared_rank(part, c)[row * PART_STRIDE + col];
    x *= a.inv_a_scale;   // exact: a power of two
    const int64_t n = (a.row_base + row0 + row) * TN + col;   // absolute sample
    if (n < a.win_start || n >= a.win_end) continue;
    if (a.out_q) a.out_q[n - a.win_start] = (int16_t)fminf(fmaxf(rintf(x * a.scale), -32767.f), 32767.f);
    if (a.out_f) a.out_f[n - a.win_start] = x;
  }
  cluster.sync();   // remote reads done before any CTA of the cluster exits
}

// ---------------------------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------------------------
// sin and cos of 2 pi w / 2^64 for a 64-bit phase word, accurate to a few 1e-8: sincospi of the
// word's top bits (exactly representable), corrected to first order by the remaining bits.
__device__ __forceinline__ void sincos_word(uint64_t w, float* s, float* c) {
  const int32_t hi = (int32_t)(w >> 32);                 // half-turns x 2^31
  const int32_t h1 = hi & ~0xFF;                         // <= 23 significant bits: exact in float
  const float x1 = (float)h1 * 4.656612873077392578125e-10f;   // 2^-31
  const float x2 = ((float)(hi - h1) + (float)(uint32_t)w * 2.3283064365386963e-10f) * 4.656612873077392578125e-10f;
  float s1, c1;
  sincospif(x1, &s1, &c1);
  const float d = 3.14159265358979323846f * x2;
  *s = fmaf(c1, d, s1);
  *c = fmaf(-s1, d, c1);
}

template <typename T>
__device__ __forceinline__ T to_half(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_half<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_half<__half>(float v) { return __float2half_rn(v); }
template <typename T>
__device__ __forceinline__ float from_half(T v);
template <>
__device__ __forceinline__ float from_half<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float from_half<__half>(__half v) { return __half2float(v); }

template <typename T>
__device__ __forceinline__ void split_store(T* hi, T* lo, int64_t i, float v) {
  const T h = to_half<T>(v);
  hi[i] = h;
  lo[i] = to_half<T>(v - from_half<T>(h));
}

// Bt[n2][2k] = cos b_k(n2), Bt[n2][2k+1] = sin b_k(n2) (the B operand stored K-major).
template <typename T>
__global__ void prep_b_kernel(const ToneRec* tones, int K, int64_t Kp, T* hi, T* lo, int window_mode) {
  const int64_t pairs = Kp / 2;
  const int64_t total = (int64_t)TN * pairs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n2 = i / pairs, k = i - n2 * pairs;
    float s = 0.f, c = 0.f;
    // static engine: pair k = (tone k / 2, segment k % 2), the segment's frequency word
    const int64_t tone = window_mode ? k >> 1 : k;
    if (tone < K) {
      const uint64_t F = (window_mode && (k & 1)) ? tones[tone].F_end : tones[tone].F;
      sincos_word((uint64_t)n2 * F, &s, &c);
    }
    split_store<T>(hi, lo, n2 * Kp + 2 * k, c);
    split_store<T>(hi, lo, n2 * Kp + 2 * k + 1, s);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_2d(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType dt, void* base, uint64_t inner,
                      uint64_t outer, uint32_t box_inner, uint32_t box_outer) {
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

float table_amp_scale(double amax) {
  if (!(amax > 0) || !std::isfinite(amax)) return 1.f;
  int e = 0;
  (void)std::frexp(amax, &e);                 // amax = m 2^e, m in [0.5, 1)
  e = std::max(-100, std::min(100, e));
  return (float)std::ldexp(1.0, 1 - e);      // amax a_scale in [1, 2)
}

size_t table_kp(int K) { return (((size_t)2 * K + TK - 1) / TK) * TK; }
size_t table_kp_window(int K) { return (((size_t)4 * K + TK - 1) / TK) * TK; }

cudaError_t launch_table_prep(const TableArgs2& t, cudaStream_t s) {
  const int64_t Kp = (int64_t)(t.window_mode ? table_kp_window(t.K) : table_kp(t.K));
  const int threads = 256;
  const int blocks = device_sm_count() * 4;
  if (t.precision == 0)
    prep_b_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(t.tones, t.K, Kp, (__nv_bfloat16*)t.b_hi,
                                                           (__nv_bfloat16*)t.b_lo, t.window_mode);
  else
    prep_b_kernel<__half><<<blocks, threads, 0, s>>>(t.tones, t.K, Kp, (__half*)t.b_hi, (__half*)t.b_lo, t.window_mode);
  return cudaGetLastError();
}

cudaError_t launch_table_gemm(const TableArgs2& t, cudaStream_t s) {
  const int64_t M = t.M;
  const int64_t Kp = (int64_t)(t.window_mode ? table_kp_window(t.K) : table_kp(t.K));
  const bool bf16 = (t.precision == 0);
  cudaError_t e;
  static EncodeTiledFn enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    enc = (EncodeTiledFn)fn;
  }
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUtensorMap mBh, mBl;
  if ((e = encode_2d(enc, &mBh, dt, t.b_hi, (uint64_t)Kp, (uint64_t)TN, TK, TN)) != cudaSuccess) return e;
  if ((e = encode_2d(enc, &mBl, dt, t.b_lo, (uint64_t)Kp, (uint64_t)TN, TK, TN)) != cudaSuccess) return e;

  TableGemmArgs ga;
  ga.n_kb = (int32_t)(Kp / TK);
  ga.out_q = t.out_q;
  ga.out_f = t.out_f;
  ga.scale = t.scale;
  ga.status = t.status;
  ga.tones = t.tones;
  ga.K = t.K;
  ga.nb_log2 = t.nb_log2;
  ga.row_base = t.row_base;
  ga.win_start = t.win_start;
  ga.win_end = t.win_end;
  ga.window_mode = t.window_mode;
  ga.a_scale = t.a_scale > 0.f ? t.a_scale : 1.f;
  ga.inv_a_scale = 1.f / ga.a_scale;
  // instruction descriptor: FP32 accumulate, A/B BF16 (1) or FP16 (0), both K-major, N/8, M/16
  const uint32_t fmt = bf16 ? 1u : 0u;
  ga.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  const size_t smem = (size_t)NSTAGE * STAGE_BYTES + 1024;
  static_assert((size_t)TM * PART_STRIDE * 4 <= (size_t)NSTAGE * STAGE_BYTES, "partial tile fits in the stages");
  // the static engine's window mode is a separate instantiation, so that the table keeps its lean
  // A-operand generator
  auto kern = t.window_mode ? (bf16 ? table_gemm_kernel<__nv_bfloat16, true> : table_gemm_kernel<__half, true>)
                            : (bf16 ? table_gemm_kernel<__nv_bfloat16, false> : table_gemm_kernel<__half, false>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // K split over a cluster of 1, 2 or 4 CTAs per 128-row tile (periodic tables), whichever finishes first by a
  // simple model: waves of co-resident clusters (a cluster of 4 leaves SMs of some GPCs idle: 36
  // clusters = 144 CTAs at once on 152 SMs, against 76 clusters of 2) times the K blocks per CTA
  // plus an epilogue worth about 8 K blocks
  const int64_t tiles = (M + TM - 1) / TM;
  static int active[5] = {0, 0, 0, 0, 0};
  unsigned split = 1;
  double best = 1e300;
  for (unsigned c = 1; c <= 4; c *= 2) {
    if ((int)c > ga.n_kb) break;
    // the static engine sums each sample over a K split that must not depend on the window's
    // length (chunk invariance): always the largest split there
    if (t.invariant && c < 4 && 4 <= ga.n_kb) continue;
    if (!active[c]) {
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(c, 1, 1);
      q.blockDim = dim3(GEMM_THREADS, 1, 1);
      q.dynamicSmemBytes = smem;
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = c;
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.attrs = qa;
      q.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, (const void*)kern, &q) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
      }
      active[c] = n;
    }
    const double waves = (double)((tiles + active[c] - 1) / active[c]);
    const double cost = waves * ((double)ga.n_kb / c + 8.0);
    if (cost < best) {
      best = cost;
      split = c;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tiles * split, 1, 1);
  cfg.blockDim = dim3(GEMM_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, mBh, mBl, ga);
}

}  // namespace awgk
