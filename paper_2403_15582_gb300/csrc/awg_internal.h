// Internal layout shared by the host library (awg_host.cpp) and the kernels (awg_render.cu).
// Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace awgk {

// Work decomposition of the render kernel.  A tile is TILE consecutive samples, cut into RUNS runs
// of RUN samples (run index j, 0 <= j < RUNS: the unit of the chirp records' stride differences).
// A render CTA of RT threads owns one tile; thread j owns run j and keeps its RUN partial sums in
// registers; the tones of a tile are split over several CTAs.  Runs and tiles are aligned to
// absolute sample indices, so a sample's value does not depend on where a render window starts
// (chunk invariance).
constexpr int RUN = 32;
constexpr int RUNS = 128;
constexpr int TILE = RUN * RUNS;   // 4096 samples
constexpr int RT = RUNS;           // threads per render CTA
constexpr int STAGE = 32;          // tones staged in shared memory at a time (double-buffered)
constexpr int SINE_SFU = 0;        // static segments: SFU sine of every sample's phase
constexpr int SINE_ROTATOR = 1;    // static segments: exact sin/cos at the run start, then rotations
constexpr int MAX_SPLIT = 16;      // cluster size limit (non-portable 16 on sm_100-class parts)
constexpr int MAX_ACTIVE_PER_LAUNCH = 7168;   // chirp slots per prep launch (kernel parameters: < 32 KB)

constexpr int64_t NO_CHIRP = INT64_MAX;

// Per-tone record read by the render kernel.  96 bytes, 16-byte aligned (bulk-copied).
struct alignas(16) ToneRec {
  uint64_t phi_ref;       // static segment before the chirp (or the only one): Phi(n) = phi_ref + n F
  uint64_t F;
  uint64_t phi_post_ref;  // static segment after the chirp:  Phi(n) = phi_post_ref + n F_end
  uint64_t F_end;
  int64_t n_s;            // chirp covers samples [n_s, n_e]; NO_CHIRP if none
  int64_t n_e;
  float A;
  int32_t slot;           // chirp slot, -1 if none
  int32_t flags;          // TONE_EXACT / TONE_LINEAR
  int32_t tab_off;        // TONE_EXACT: offset of this chirp's per-sample phase table
  float rot_c, rot_s;     // cos, sin of the per-sample step 2 pi F / 2^64 (rotator sine variant)
  float rot_c_end, rot_s_end;   // the same for F_end
  int64_t a_ns;           // amplitude ramp (TONE_AMP_RAMP): A -> A_end over samples a_ns .. a_ns + a_L
  float A_end;
  int32_t a_L;
};
static_assert(sizeof(ToneRec) == 96, "ToneRec layout");
constexpr int32_t TONE_EXACT = 1;    // chirp read from a per-sample table of exact phases
constexpr int32_t TONE_LINEAR = 2;   // linear chirp: differences of order >= 3 are exactly zero
constexpr int32_t TONE_AMP_RAMP = 4;      // the amplitude ramps (see ToneRec::a_ns)
constexpr int32_t TONE_AMP_MINJERK = 8;   // ... along the minimum-jerk profile (else linear)
constexpr int32_t TONE_FLAT3 = 32;        // the chirp's third unit difference stays below 2^30 words:
                                          // the run cascade's h rounds to 0 in every run
constexpr int32_t TONE_LOW6 = 64;         // FLAT3, and B_6, E_5, G_2..G_4 move a run's phase by
                                          // < 64 units of 2^-32 turn: left out of the run set-up
constexpr int32_t TONE_LOW3 = 256;        // LOW6, and B_5, E_3, E_4 negligible too (< 256 units
                                          // with the others over a two-run cascade): left out as well
constexpr int32_t TONE_PAIR = 128;        // a lane pair may share the chirp's run set-up: linear, or
                                          // LOW6 with C(63,3) max |Delta^3 P| below 512 units of 2^-32
                                          // turn (the render's run set-up, see render_tile)
constexpr int32_t TONE_EXP = 16;          // exponential chirp: ChirpRec::d[0..4] hold F_start, F_end
                                          // and the doubles alpha, C, e^alpha - 1 (bit patterns)

#if defined(__CUDACC__)
#define AWG_HD __host__ __device__
#else
#define AWG_HD
#endif

// Static segments per 4096-sample tile (the tensor-core static engine): tone t is static with a
// constant amplitude over the tile [T0, T0 + TILE) in segment seg (0: before its chirp, or the
// only one; 1: after its chirp).  Returns the segment's phase reference, frequency word and
// amplitude.  A function of the tile and the tone state only, so the split between the engines
// does not depend on how the stream is cut into calls.
AWG_HD inline bool tile_segment_static(const ToneRec& t, int64_t T0, int seg, uint64_t* phi, uint64_t* F, float* A) {
  const int64_t T1 = T0 + TILE - 1;
  if (seg == 0) {
    if (t.slot >= 0 && T1 >= t.n_s) return false;
    *phi = t.phi_ref;
    *F = t.F;
  } else {
    if (t.slot < 0 || T0 <= t.n_e) return false;
    *phi = t.phi_post_ref;
    *F = t.F_end;
  }
  *A = t.A;
  if (t.flags & TONE_AMP_RAMP) {
    if (T1 <= t.a_ns) *A = t.A;
    else if (T0 >= t.a_ns + t.a_L) *A = t.A_end;
    else return false;
  }
  return true;
}
AWG_HD inline bool tile_static(const ToneRec& t, int64_t T0) {
  uint64_t phi, F;
  float A;
  return tile_segment_static(t, T0, 0, &phi, &F, &A) || tile_segment_static(t, T0, 1, &phi, &F, &A);
}

// Per-chirp record (one per live slot): the 192-bit forward-difference words.
struct alignas(16) ChirpRec {
  uint64_t d[21];         // d_0..d_6, 3 little-endian limbs each
  uint64_t phi_start;     // Phi(n_s)
  int64_t n_s;
  int64_t L;
  int32_t tone;
  int32_t flags;
  uint64_t pad;
};
static_assert(sizeof(ChirpRec) == 208, "ChirpRec layout");

// Per (active chirp, tile) record: the chirp phase polynomial re-expressed at the tile start as
// forward differences with stride RUN in the run index j (0 <= j < RUNS), for the phase and its
// first three unit-stride differences.  Words (2^-64 turn), rounded.  B[0] is the phase word.
struct alignas(16) TileRec {
  uint64_t B[7];
  uint64_t E[6];
  uint64_t G[5];
  uint64_t H[4];
};
static_assert(sizeof(TileRec) == 176, "TileRec layout");

// Arguments of one prep launch, the active chirp slots inline (kernel parameters are copied with
// the launch: a launch of up to 1024 slots passes the small form, larger ones the full 7168).
template <int CAP>
struct PrepArgsT {
  const ChirpRec* chirps;
  TileRec* recs;          // [n_active][n_tiles]
  int32_t* act_of_slot;   // slot -> active index (written here)
  int64_t tile0;          // absolute index of the first tile
  int32_t n_tiles;
  int32_t n_active;
  int32_t act_base;       // active index of slots[0]
  uint32_t W[7][7];       // W[q][i] = Delta^q_j C(j RUN, i) at j = 0 (all below 2^32)
  uint64_t inv_odd[3][3]; // inverses mod 2^192 of 3, 15, 45
  int32_t slots[CAP];
};
using PrepArgs = PrepArgsT<MAX_ACTIVE_PER_LAUNCH>;
constexpr int SMALL_PREP = 1024;
static_assert(sizeof(PrepArgs) <= 32764, "prep kernel parameters fit the 32 KB parameter space");

struct RenderArgs {
  const ToneRec* tones;
  const uint32_t* exact_tab;  // per-sample 32-bit phases of TONE_EXACT chirps
  const ChirpRec* chirps;
  const TileRec* recs;
  const int32_t* act_of_slot;
  int32_t K;
  int32_t split;          // CTAs per tile (cluster size)
  int64_t tile0;
  int32_t n_tiles;
  int64_t win_start, win_end;   // [win_start, win_end) absolute samples written
  int16_t* out_q;
  float* out_f;
  float scale;            // 32767 / FS
  int32_t* status;
  uint64_t inv_odd[3][3];
  int32_t sine_mode;      // SINE_SFU or SINE_ROTATOR (static segments)
  int32_t q_stride;       // int16 output: sample i goes to out_q[i * q_stride] (0: 1; channel multiplexing)
  // record rows: the records of active chirp a for window tile t are at recs[a * rec_stride +
  // rec_tile0 + t] (rec_stride 0: n_tiles, the render's own set-up)
  int32_t rec_stride;
  int32_t rec_tile0;
  // pipelined chunk sequences (otherwise 0 / null): pdl 1 waits for the preceding kernel (the
  // records' set-up) and then lets the next kernel launch early; pdl 2 lets it launch early and
  // reads nothing the preceding kernel writes (with split scratch, it waits for that kernel before
  // reusing the scratch); each CTA adds 1 to *exit_ctr once its samples are stored
  int32_t pdl;
  unsigned long long* exit_ctr;
  // tensor-core static engine (otherwise null / 0): tones static over the window are skipped here
  // (their sum comes from the table GEMM) and base[n - win_start] is added before quantising
  const float* base;
  int32_t skip_static;
  // tones to visit (sorted, n_list of them; null: all K): CTA crank of a tile takes the listed
  // tones of [bounds[crank], bounds[crank + 1]) in ascending order (bounds[0] = 0,
  // bounds[split] = K); without a list it takes all of [K crank / split, K (crank + 1) / split)
  const int32_t* tone_list;
  int32_t n_list;
  int32_t bounds[MAX_SPLIT + 1];
  // split sums without clusters (render_split_kernel; null: cluster reduction): partial tiles
  // part[(tile split + rank) TILE + sample] and one counter per tile (a multiple of split between
  // launches: every CTA adds 1)
  float* part;
  unsigned long long* tile_ctr;
};

struct PhaseArgs {
  const ToneRec* tones;
  const ChirpRec* chirps;
  int32_t n;
  int64_t sample;
  uint64_t* out;
  uint64_t inv_odd[3][3];
};

struct TraceArgs {      // per-sample render phases of one tone (test hook)
  const ToneRec* tones;
  const ChirpRec* chirps;
  const TileRec* recs;
  const int32_t* act_of_slot;
  int32_t tone;
  int64_t n0;
  int32_t count;
  int64_t tile0;
  int32_t n_tiles;
  int32_t K, split;       // the render's tone count and split (its CTAs' tone ranges and stages)
  int32_t listed;         // renders go through a tone list (static engine): no shared set-ups
  uint32_t* out;
  uint64_t inv_odd[3][3];
};

struct TableArgs {      // exact per-sample 32-bit phases of one short chirp, m = 0..L
  const ChirpRec* chirps;
  int32_t slot;
  uint32_t* out;          // L + 1 entries
  uint64_t inv_odd[3][3];
};

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);
cudaError_t launch_exact_table(const TableArgs& a, int64_t L, cudaStream_t s);
cudaError_t launch_render(const RenderArgs& a, cudaStream_t s);
cudaError_t launch_replay(const int16_t* tab, int32_t log2_len, int64_t c, int64_t n, int16_t* out, int32_t stride,
                          cudaStream_t s);
// A bounded wait on the device (join of a pipelined sequence): at most limit_ns of wall time, then
// the status word becomes AWG_ETIMEOUT and the kernel returns.
constexpr uint64_t JOIN_LIMIT_NS = 2000000000ull;
cudaError_t launch_join(const unsigned long long* exit_ctr, unsigned long long target, int32_t* status,
                        uint64_t limit_ns, cudaStream_t s);
// items[i] = (request index into reqs, window tile); every request has split == `split`.
// Several renders in one launch (tiles items[i] = (request, tile) of the requests reqs[]; all of
// tone split `split`); every request carries split scratch (part, tile_ctr with n_tiles zeroed
// counters).
cudaError_t launch_render_batch_split(const RenderArgs* reqs, const int2* items, int n_items, int split,
                                      cudaStream_t s);
cudaError_t launch_phase_words(const PhaseArgs& a, cudaStream_t s);
cudaError_t launch_trace(const TraceArgs& a, cudaStream_t s);
cudaError_t launch_sfu_rate(float* out, int blocks, int runs, cudaStream_t s);   // RT threads per block
cudaError_t launch_chirp_rate(float* out, int blocks, int runs, cudaStream_t s); // RT threads per block
cudaError_t render_setup_attributes();
// Number of SMs of the current device (queried once per device, then cached); grid sizes of the
// grid-stride kernels are multiples of it.
int device_sm_count();

// Fixed scratch of the allocation-free render (awg_noalloc.cu): 12 MiB of tile records and a map
// for 16384 chirp slots.  Looks up the arrays' device addresses on first use for `device`, which
// must be the current device.
constexpr size_t NOALLOC_MAX_RECORDS = (12u << 20) / sizeof(TileRec);   // 71493
constexpr int32_t NOALLOC_MAX_SLOTS = 16384;
cudaError_t noalloc_scratch(int device, TileRec** recs, int32_t** act);

// Periodic-table GEMM (awg_table.cu).
struct TableArgs2 {
  const ToneRec* tones;
  int32_t K;
  int64_t M;              // rows of 256 samples
  int32_t nb_log2;        // log2 of the columns (8: 256 samples per row)
  int64_t row_base;       // absolute row index of row 0 (sample row_base * 256)
  int64_t win_start, win_end;   // absolute samples stored (out[n - win_start])
  int32_t window_mode;    // 1: static engine: per tone two segments (4 columns), each taken only
                          //    in the 4096-sample tiles where it is static (tile_segment_static)
  int32_t precision;      // 0 BF16, 1 FP16 hi+lo operands
  int32_t invariant;      // 1: the summation of a sample may not depend on M (static engine: the
                          //    same samples however the stream is cut)
  void* b_hi;             // 256 x Kp (the A operand is generated inside the GEMM kernel)
  void* b_lo;
  int16_t* out_q;
  float* out_f;
  float scale;
  // power of two the A operand is multiplied by before its hi + lo split (the largest amplitude
  // lands in [1, 2), so that the FP16 halves stay in the normal range), divided out exactly in
  // the epilogue
  float a_scale;
  int32_t* status;
};
// a_scale for amplitudes whose largest magnitude is amax (1 for amax 0)
float table_amp_scale(double amax);
size_t table_kp(int K);  // padded inner dimension (2K rounded up to the K tile)
size_t table_kp_window(int K);   // the same for the static engine's 4 columns per tone
cudaError_t launch_table_prep(const TableArgs2& t, cudaStream_t s);   // B operand halves
cudaError_t launch_table_gemm(const TableArgs2& t, cudaStream_t s);   // tensor-core GEMM + epilogue

}  // namespace awgk

struct awg;
namespace awgk {
// Everything awg_render does except the render launch: chirp tile set-up for the window
// [cursor, cursor + n) on stream s, the render descriptor in *ra, and the cursor advance.  The
// caller launches the render (e.g. batched with other handles') on the same stream.  The tile
// records go to `recs` (recs_cap records) and the slot -> record map to `act` (render_slots(h)
// entries) when they are given, so that windows of one handle can be in flight on several streams
// at once; otherwise to the handle's own buffers.  *recs_need (if given) receives the number of
// records the window needs; AWG_ENOMEM if recs_cap is short (the cursor is then unchanged).
int prepare_render(struct awg* h, int64_t n, int16_t* out_q, float* out_f, cudaStream_t s, RenderArgs* ra,
                   TileRec* recs = nullptr, size_t recs_cap = 0, int32_t* act = nullptr,
                   size_t* recs_need = nullptr);
// Tile records prepare_render needs for the window [cursor, cursor + n).
size_t render_recs_needed(const struct awg* h, int64_t n);
// The tensor-core static engine for a served request (its tone state is fixed while it is served):
// engine_setup selects `engine` (AWG_STATIC_GEMM_FP16 / _BF16) for h, prepares its GEMM's B operand
// on stream s (the caller synchronises s before the first render) and returns the tone split of the
// render part (tones that hold a chirp or a ramp).  prepare_render_engine does what prepare_render
// does for the window [cursor, cursor + n), with the engine: the GEMM of the window's static tones
// is launched on s into `base` (n floats), or straight into out_q when no tone chirps or ramps in
// the window (*need_render false: no render item); otherwise the listed tones (d_list, staged
// through the pinned h_list, list_cap entries) are rendered with base added, and the chirp tile
// records go to recs / act as in prepare_render.  engine_list_needed: entries of that list.
int engine_setup(struct awg* h, int32_t engine, cudaStream_t s, int32_t* render_split);
int prepare_render_engine(struct awg* h, int64_t n, int16_t* out_q, cudaStream_t s, RenderArgs* ra, TileRec* recs,
                          size_t recs_cap, int32_t* act, float* base, int32_t* d_list, int32_t* h_list,
                          size_t list_cap, bool* need_render);
size_t engine_list_needed(struct awg* h, int64_t n);
// Entries of the slot -> record map of h (its chirp slots).
size_t render_slots(const struct awg* h);
// CTAs per tile (tone split) for K tones; depends on K only.
int tone_split_for(int K);

// Sets the message awg_last_error() returns on this thread; returns `code`.
int set_error(int code, const std::string& msg);

}  // namespace awgk
