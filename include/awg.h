/*
 * awg.h -- C ABI of a GB300 (sm_103a) multi-tone waveform synthesiser.
 *
 * It computes x[n] = sum_k A_k sin(phi_k(n)) (additive synthesis, Sec. II Eq. main and the
 * dynamic form Eq. dynamicandstatic of Tu & Subhankar, "Fast real-time arbitrary waveform
 * generation using graphic processing units") for static tones and tones chirped along linear,
 * minimum-jerk (Eq. freqchirp) or exponential frequency ramps, and writes scaled int16 DAC samples (and,
 * on request, the FP32 sum) chunk by chunk.
 *
 * Phase model.  A tone's phase is an integer word Phi in units of 2^-64 turn.  Static tones:
 * Phi(n) = Phi_ref + n*F (mod 2^64).  A linear or minimum-jerk chirp over samples n_s..n_s+L
 * follows a degree <= 6 polynomial held as seven 2^128-scaled forward differences (192-bit
 * words); its phase words are exact integers, the same ones a sequential 192-bit accumulator cascade produces, so
 * there is no drift over arbitrarily long streams.  After the chirp the tone is static at the
 * end frequency, continuing from the phase reached at n_s+L (Eq. freqchirp case 2).
 *
 * Conventions for every call below:
 *  - Return value: AWG_OK (0) or a negative AWG_E* code; awg_last_error() then returns a
 *    thread-local message.  A failed call leaves the handle unchanged.
 *  - Host arrays passed in are read during the call only (copied); the caller keeps ownership.
 *  - `out` pointers are caller-owned device memory, or pinned host memory that is mapped into
 *    the device address space (cudaHostAlloc with cudaHostAllocMapped, or any pinned memory on
 *    a system with unified addressing); they are written asynchronously on `stream`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - One handle must not be used from two host threads at once, and the renders of one handle
 *    must be issued to one stream (or ordered by the caller).
 *  - Sample indices are absolute (int64, counted from 0 at creation).
 */
#ifndef AWG_H
#define AWG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct awg awg_t;

enum {
  AWG_OK = 0,
  AWG_EINVAL = -1,    /* bad argument: see awg_last_error() */
  AWG_ENOMEM = -2,    /* device or pinned-host allocation failed, or a fixed capacity is full */
  AWG_ECUDA = -3,     /* a CUDA runtime call failed */
  AWG_ETIMEOUT = -4,  /* a bounded wait in a kernel gave up (status word set on the device) */
  AWG_EDEADLINE = -5, /* admission refused: the request cannot meet its deadline */
  AWG_ESTATE = -6     /* call not valid in the handle's current state */
};

enum { AWG_PROFILE_LINEAR = 0, AWG_PROFILE_MINJERK = 1, AWG_PROFILE_EXPONENTIAL = 2 };

/* Version of this ABI (major*10000 + minor*100 + patch). */
int awg_version(void);

/* Message describing the last failing call on this host thread ("" if none). */
const char* awg_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Host-only set-up arithmetic (no GPU involved).  These are the exact rules the library uses
 * internally; they are exported so that callers and tests can reproduce the words.
 * ---------------------------------------------------------------------------------------- */

/* Frequency word F = rint(f/fs * 2^64) mod 2^64 (IEEE double quotient, ties to even).
 * Tone frequency of Eq. main as a per-sample phase step.  EINVAL if fs is not finite and > 0,
 * or f is not finite, or f < 0 or f >= fs (a tone above fs/2 is rendered as its alias). */
int awg_freq_word(double f_hz, double fs_hz, uint64_t* out_word);

/* Phase word Phi0 = rint(frac(theta / 2pi) * 2^64) mod 2^64 (theta_j of Eq. main).
 * EINVAL if theta is not finite. */
int awg_phase_word(double theta_rad, uint64_t* out_word);

/* Grid word of Eq. freqapprox: j = rint(f/fs * 2^log2_len), F = j << (64 - log2_len), so that
 * the tone completes exactly j cycles in 2^log2_len samples.  1 <= log2_len <= 40.
 * out_j may be NULL. */
int awg_grid_word(double f_hz, double fs_hz, int32_t log2_len, uint64_t* out_word, int64_t* out_j);

/* Chirp length L = rint(duration * fs) samples; the chirp spans m = 0..L (Eq. freqchirp case 1,
 * 0 <= i <= T f_s).  EINVAL unless 1 <= L <= 2^28 - 1. */
int awg_chirp_length(double duration_s, double fs_hz, int64_t* out_L);

/* The seven 192-bit forward-difference words d_0..d_6 of a chirp from word F_start to word F_end
 * over L samples (profile AWG_PROFILE_LINEAR or AWG_PROFILE_MINJERK).  With P(m) the chirp phase
 * in words relative to its start (min-jerk: P(m) = F_start m + D (5 m^4 L^2 - 6 m^5 L + 2 m^6) /
 * (2 L^5), Eq. freqchirp; linear: P(m) = F_start m + D m^2 / (2L), D = F_end - F_start as a
 * signed integer), d_k = rint_half_even(Delta^k P(0) * 2^128) mod 2^192 for k >= 1 and
 * d_0 = 2^127.  out: 21 uint64, little-endian limbs, d_0 first.
 * AWG_PROFILE_EXPONENTIAL (Sec. II names exponential chirps; the phase is the integral of
 * F(t) = F_start r^(t/L), r = F_end / F_start, i.e. R(m) = C (e^(alpha m) - 1) words with
 * alpha = ln(r) / L and C = F_start / alpha): out[0] = F_start, out[1] = F_end and the IEEE
 * doubles alpha, C, e^alpha - 1 as bit patterns in out[2..4]; the rest 0.  EINVAL if F_start or
 * F_end is 0.  With F_start == F_end the chirp is the linear one (the same phase). */
int awg_chirp_coeffs(uint64_t F_start, uint64_t F_end, int64_t L, int32_t profile, uint64_t* out21);

/* Host-only classification hook: the flags the render gives a chirp from word F_start to word
 * F_end over L samples, written to *out_flags, with the bounds that decide them (the paper has no
 * counterpart; its run set-up is the library's own).  AWG_CHIRP_LINEAR / AWG_CHIRP_EXP: the
 * profile; AWG_CHIRP_TABLE: rendered from a per-sample table of exact phases (very short, fast
 * chirps); AWG_CHIRP_FLAT3: the third unit difference stays below 2^30 words (the run cascade's
 * third difference rounds to 0); AWG_CHIRP_LOW6 / AWG_CHIRP_LOW3: the run set-up leaves out the
 * stride differences it proves negligible (below 64 units of 2^-32 turn over a run, and all of
 * them with B_5, E_3, E_4 below 256 units over a two-run cascade); AWG_CHIRP_PAIR: two lanes may
 * share the chirp's run set-up (linear, or LOW6 with C(63,3) max |Delta^3 P| below 512 units).
 * EINVAL as awg_set_chirps (L >= 1, known profile, exponential ends > 0). */
enum { AWG_CHIRP_TABLE = 1, AWG_CHIRP_LINEAR = 2, AWG_CHIRP_EXP = 16, AWG_CHIRP_FLAT3 = 32, AWG_CHIRP_LOW6 = 64,
       AWG_CHIRP_PAIR = 128, AWG_CHIRP_LOW3 = 256 };
int awg_chirp_render_flags(uint64_t F_start, uint64_t F_end, int64_t L, int32_t profile, int32_t* out_flags);

/* ------------------------------------------------------------------------------------------
 * Synthesiser handle (device-resident tone and chirp state).
 * ---------------------------------------------------------------------------------------- */

/* Create a handle for sample rate fs (Hz) on the current CUDA device.  NULL on error. */
awg_t* awg_create(double sample_rate_hz);

/* Release the handle and its device memory (waits for its in-flight work). NULL is allowed. */
void awg_destroy(awg_t* h);

/* Replace the tone set: n tones with frequency (Hz, in [0, fs)), amplitude (finite) and initial
 * phase (rad, the phase at sample 0).  Clears all chirps.  n = 0 is allowed (silence).
 * Full scale returns to its default (sum |A|) unless set explicitly afterwards. */
int awg_set_tones(awg_t* h, const double* freq_hz, const double* amp, const double* phase_rad, int32_t n);

/* As awg_set_tones, with each frequency snapped to the f_s / 2^log2_len grid (Eq. freqapprox),
 * so that the record of 2^log2_len samples is exactly periodic. */
int awg_set_tones_grid(awg_t* h, const double* freq_hz, int32_t log2_len, const double* amp,
                       const double* phase_rad, int32_t n);

/* Schedule n chirps.  Chirp i moves tone[i] from f_start[i] to f_end[i] (Hz, each in [0, fs))
 * over duration[i] seconds (L = rint(duration fs) samples, 1 <= L < 2^28) with the given
 * profile (AWG_PROFILE_LINEAR, AWG_PROFILE_MINJERK, or AWG_PROFILE_EXPONENTIAL: the frequency
 * moves geometrically, both ends > 0 Hz; its phase is evaluated in FP64, within a few 1e-9 turn
 * of the exact integral, where the polynomial profiles are exact integers), starting at absolute
 * sample start_sample[i] from the tone's phase at that sample
 * (a start frequency that differs from the tone's current frequency is a frequency step).
 * A tone holds one chirp at a time: a new chirp on a tone is accepted once the render cursor
 * has passed that tone's previous chirp (previous n_s + L < cursor); the previous chirp's end
 * state then becomes the tone's static state.  Every chirp must start at or after the cursor,
 * and one call may hold at most one chirp per tone.
 * EINVAL on any violation (nothing is applied); ENOMEM if device memory runs out. */
int awg_set_chirps(awg_t* h, const int32_t* tone, const double* f_start_hz, const double* f_end_hz,
                   const double* duration_s, const int32_t* profile, const int64_t* start_sample,
                   int32_t n);

/* Schedule n amplitude ramps (the time-varying amplitude a_j[i] of Eq. dynamicandstatic, e.g. to
 * switch tweezers on and off smoothly).  Ramp i moves tone[i]'s amplitude from its current value
 * to amp_end[i] over L = rint(duration[i] fs) samples (1 <= L < 2^28) starting at absolute sample
 * start_sample[i]: a(n) = A + (amp_end - A) s(tau), tau = (n - start)/L, with s(tau) = tau
 * (AWG_PROFILE_LINEAR) or 10 tau^3 - 15 tau^4 + 6 tau^5 (AWG_PROFILE_MINJERK, the minimum-jerk
 * profile of Eq. freqchirp); a = A before the ramp and amp_end after it.  Ramps and chirps are
 * independent (a tone may do both at once).  A tone holds one ramp at a time: a new ramp is
 * accepted once the cursor has passed the previous one's end, whose amp_end becomes the tone's
 * amplitude.  Ramps start at or after the cursor; one ramp per tone per call.  Full scale is not
 * changed: set it explicitly (awg_set_full_scale) when amplitudes ramp above their initial
 * values, since the default sum |A_k| could then clip.  Tiles in which a ramp is under way are
 * rendered by the kernel's general per-sample path (amplitude in FP32, error <= 6e-7 |amp_end - A|).
 * EINVAL on any violation (nothing is applied). */
int awg_set_amp_ramps(awg_t* h, const int32_t* tone, const double* amp_end, const double* duration_s,
                      const int32_t* profile, const int64_t* start_sample, int32_t n);

/* Full-scale value FS that maps to int16 code 32767 (q = clamp(rint(x * 32767/FS), +-32767)).
 * fs_value <= 0 restores the default sum |A_k|, which can never clip. */
int awg_set_full_scale(awg_t* h, double fs_value);

/* Current full-scale value. */
double awg_full_scale(const awg_t* h);

/* Sample rate the handle was created with (Hz), 0 for NULL. */
double awg_sample_rate(const awg_t* h);

/* Move the render cursor to an absolute sample (>= 0).  Rendering depends only on absolute
 * indices and the current tone and chirp state, so seeking back reproduces earlier output bit
 * for bit as long as no chirp set since then has folded an earlier chirp of the same tone. */
int awg_seek(awg_t* h, int64_t sample);

/* The render cursor (next sample awg_render writes), or -1 for NULL. */
int64_t awg_cursor(const awg_t* h);

/* How static tone segments are evaluated (chirp segments always use the SFU form):
 * AWG_SINE_SFU (default): every sample's sine from its phase word on the SFU, error <= 2^-21.4 per
 *   sample; AWG_SINE_ROTATOR: the exact phase word at the start of each run of 32 samples gives
 *   sin and cos on the SFU, then 31 complex rotations by the per-sample step (cos, sin of
 *   2 pi F / 2^64, rounded to FP32 on the host) on the FP32 pipe, 5 FP32 operations per
 *   tone-sample; error <= 1.2e-5 |A| per tone-sample (rounding of the step and of 4 operations
 *   per rotation over at most 31 rotations).  The mode is part of the handle's state: every
 *   render path uses it, and output depends on it (not bit-identical between modes).  AWG_EINVAL
 *   for other values. */
enum { AWG_SINE_SFU = 0, AWG_SINE_ROTATOR = 1 };
int awg_set_sine_mode(awg_t* h, int32_t mode);
int32_t awg_sine_mode(const awg_t* h);

/* Engine for static tones.  AWG_STATIC_DIRECT (default): every tone through the render kernel.
 * AWG_STATIC_GEMM_FP16 / _BF16: in every 4096-sample tile, the tones that are static there (no
 * chirp and no amplitude ramp under way in the tile; before or after the tone's chirp) are summed
 * on the tensor cores by the table GEMM of awg_table_gemm, over 256-sample rows aligned to
 * absolute sample indices (x[256 r + c] = sum_k [A_k sin a_k(r)] cos b_k(c) + [A_k cos a_k(r)]
 * sin b_k(c) from exact phase words, split-precision operands, FP32 accumulation; two column
 * pairs per tone, one per segment, or one pair while no tone of the handle has ever held a chirp
 * or a ramp); the remaining tones go through the render kernel, which adds the GEMM's FP32 sum
 * before quantising.  Within one engine, and between calls that set tones, chirps or ramps, a
 * sample's value does not depend on how the stream is cut into calls.  Output stays within 1 LSB of the oracle;
 * it is not bit-identical to the direct engine.  awg_render_chunks renders chunk by chunk with a
 * GEMM engine; awg_render_noalloc always uses the direct engine.  AWG_EINVAL for other values. */
enum { AWG_STATIC_DIRECT = 0, AWG_STATIC_GEMM_FP16 = 1, AWG_STATIC_GEMM_BF16 = 2 };
int awg_set_static_engine(awg_t* h, int32_t engine);
int32_t awg_static_engine(const awg_t* h);

/* Periodic hand-off (the end state of the Playback pathway, Sec. IV-C: once the chirps are over
 * the output is a periodic waveform).  When every tone's final frequency (after its chirp, if it
 * has one) lies on the f_s / 2^log2_len grid (Eq. freqapprox), the waveform from
 * n_p = max(cursor, the first 4096-sample tile boundary after the last chirp's end) on is
 * periodic with period N = 2^log2_len.  This call computes that period once into a device table owned by the handle (method
 * AWG_PERIODIC_DIRECT: the render kernel over one period of the static state, in the handle's
 * sine mode, so replayed samples equal the rendered ones bit for bit; AWG_PERIODIC_GEMM_BF16 /
 * _FP16: the split-precision table GEMM, within 1 LSB), synchronising `stream`.  After it,
 * awg_render / awg_render_chunks / awg_render_multiplexed render samples before n_p as usual and
 * replay the table for samples from n_p on (a copy kernel; awg_render_f32 and
 * awg_render_noalloc keep rendering).  awg_set_tones and awg_set_chirps end the hand-off.
 * AWG_EINVAL: log2_len outside 12..30 (15..30 for the GEMM), unknown method, a final frequency
 * off the grid. */
enum { AWG_PERIODIC_DIRECT = 0, AWG_PERIODIC_GEMM_BF16 = 1, AWG_PERIODIC_GEMM_FP16 = 2 };
int awg_set_periodic(awg_t* h, int32_t log2_len, int32_t method, void* stream);
/* n_p of the active hand-off, or -1. */
int64_t awg_periodic_start(const awg_t* h);
int awg_clear_periodic(awg_t* h);

/* Render samples cursor .. cursor+n-1 as int16 codes into out[0..n) on `stream`, then advance
 * the cursor by n.  Asynchronous.  Output is a function of the absolute sample index and the
 * tone set only: render(a) followed by render(b) equals render(a+b) bit for bit. */
int awg_render(awg_t* h, int64_t n, int16_t* out, void* stream);

/* As awg_render, also writing the FP32 sum x[n] (unscaled) to out_f32 (out_q may be NULL). */
int awg_render_f32(awg_t* h, int64_t n, float* out_f32, int16_t* out_q, void* stream);

/* Channel multiplexing for a multi-channel DAC (the WM step of Sec. IV-C, fused into the render's
 * store): handles[c] (n_channels of them, 1..8, distinct, one sample rate, one device) each
 * render n samples from their own cursor; sample i of channel c goes to out[i * n_channels + c],
 * so the buffer holds groups of n_channels samples, one per channel, as the card reads them.
 * Each channel's samples are the same as its awg_render output.  Every cursor advances by n; on
 * an error none does. */
int awg_render_multiplexed(awg_t* const* handles, int32_t n_channels, int64_t n, int16_t* out, void* stream);

/* Render n_chunks consecutive chunks of `chunk` samples (the chunk loop of Sec. IV: the cursor
 * advances chunk by chunk) into out[0 .. n_chunks * chunk), with the same samples as n_chunks
 * calls of awg_render.  The chunks are issued as one pipelined sequence: the chunks go in groups
 * whose chirp tile records fit a fixed budget (4M records); one set-up launch per group computes
 * the records of all its chunks, then the chunk renders follow with programmatic dependent
 * launch, so that each render starts while the one before drains; a join kernel (a bounded wait
 * on a device counter of finished render CTAs) ends each group and restores plain stream order
 * for later work on `stream`.  out is device memory or mapped pinned host memory.  AWG_EINVAL for
 * chunk < 1, n_chunks < 0 or overflow.  A wait that times out inside the sequence (about 2 s)
 * sets the device status to AWG_ETIMEOUT (see awg_device_status). */
int awg_render_chunks(awg_t* h, int64_t chunk, int32_t n_chunks, int16_t* out, void* stream);

/* Render n samples from the cursor as consecutive chunks of `chunk` samples, the last one shorter
 * when chunk does not divide n, in one pipelined sequence as awg_render_chunks (the short last
 * chunk included, so that its render overlaps the one before).  out[0 .. n).  The same samples as
 * awg_render of n samples.  AWG_EINVAL for chunk < 1, n < 0 or overflow. */
int awg_render_stream(awg_t* h, int64_t n, int64_t chunk, int16_t* out, void* stream);

/* Number of kernels the handle has launched so far (every render, set-up, join, table and replay
 * kernel, including those of set-up calls and test hooks); -1 for a null handle.  Read it before
 * and after a region to count that region's launches. */
int64_t awg_launch_count(const awg_t* h);

/* Phase words Phi_k(sample) of the first n tones (n <= tone count), computed on the device by the
 * exact closed form (192-bit, the function that seeds every render tile) and copied to
 * out_host.  Synchronous. */
int awg_phase_words(awg_t* h, int64_t sample, uint64_t* out_host, int32_t n);

/* Per-sample 32-bit phases (units of 2^-32 turn, plus the 2^8 rounding offset of the sine
 * argument) that the render kernel feeds to the sine for tone `tone` at samples
 * cursor-independent [n0, n0+count), count <= 2^20; out_host receives count uint32.  For
 * checking the in-tile phase approximation against exact words.  Synchronous. */
int awg_render_phases(awg_t* h, int32_t tone, int64_t n0, int32_t count, uint32_t* out_host);

/* Tile split used for this handle's tone count: the tones of a tile are summed by this many CTAs,
 * whose partial sums are added in rank order.  For information. */
int32_t awg_tone_split(const awg_t* h);

/* Sum of the device time (ms) of the last render's kernels, recorded with CUDA events; it is
 * valid once that render has completed (e.g. after synchronising its stream).  -1 if none. */
float awg_last_render_ms(awg_t* h);

/* Profiling mode: while on, every render records CUDA events on its stream around its chirp
 * set-up kernels and around its render kernel; a pipelined sequence (awg_render_chunks,
 * awg_render_stream) records them at its start, after the set-up of its first group of chunks
 * and after its last join, so its "render" time spans every chunk render of the sequence (they
 * overlap) and any later group's set-up.  awg_profile_begin clears the record.  awg_profile_end
 * waits for the last recorded event, writes per render call the device time (ms) of the set-up
 * kernel(s) and of the render kernel(s) into prep_ms[i] / render_ms[i] for i < cap (either may be
 * NULL), stores the number of kernels launched in *launches (may be NULL), stops recording and
 * returns the number of render calls recorded (or a negative AWG_E* code). */
int awg_profile_begin(awg_t* h);
int awg_profile_end(awg_t* h, float* prep_ms, float* render_ms, int32_t cap, int64_t* launches);

/* Limits of awg_render_noalloc: (chirps active in the window) x (4096-sample tiles the window
 * touches) tile records, and chirp slots (tones that hold a chirp record). */
#define AWG_NOALLOC_MAX_RECORDS 71493
#define AWG_NOALLOC_MAX_SLOTS 16384

/* As awg_render, but it allocates nothing: no cudaMalloc or cudaFree and, when it succeeds, no
 * host heap either (a rejected call formats its message for awg_last_error).  For callers
 * that cannot allocate while they stream: a real-time thread feeding a DAC must not stall in the
 * device allocator (which can synchronise the whole device and take longer than a chunk's
 * playback time), and some host applications give the library a fixed device-memory budget
 * up front.  Such a caller creates the handle and sets its tones and chirps beforehand, then
 * calls this for every chunk.  The chirp tile records and their slot map go to a fixed 12 MiB
 * scratch array compiled into the library, which every GPU that loads the library holds until
 * the process exits.  awg_create looks up that array's device address on its device (loading
 * the code that holds it), so no call of this function does; it renders on the handle's device
 * only (AWG_EINVAL on another current device).  AWG_ENOMEM (with a message) when the window needs more than
 * AWG_NOALLOC_MAX_RECORDS records or a chirp slot index reaches AWG_NOALLOC_MAX_SLOTS.  All calls
 * in the process share the scratch: each call writes every record it reads, so nothing needs to
 * start at zero, but calls whose kernels overlap on the GPU (other streams, other handles) race
 * -- issue them in order on one stream.  The paper has no counterpart to this entry point. */
int awg_render_noalloc(awg_t* h, int64_t n, int16_t* out, void* stream);

/* Device-side status word of the handle: 0, or the AWG_E* code a kernel raised (for instance
 * AWG_ETIMEOUT when a bounded wait on an mbarrier gave up).  Reading it synchronises.  Clears
 * the word. */
int awg_device_status(awg_t* h);

/* Test hook for the bounded waits on the device: launches on `stream` the join kernel that ends
 * the pipelined chunk sequences (awg_render_chunks), with a target one above the handle's count of
 * finished render CTAs -- a count no kernel will reach -- and a wait limit of limit_us
 * microseconds (1 .. 10^7).  The wait gives up after the limit, sets the device status word to
 * AWG_ETIMEOUT (read it with awg_device_status) and the kernel returns: nothing hangs, and the
 * handle and the CUDA context stay usable.  Asynchronous.  AWG_EINVAL for a limit out of range.
 * (The paper has no counterpart: this checks the library's own failure path.) */
int awg_test_wait_timeout(awg_t* h, int64_t limit_us, void* stream);

/* Measurement hook: the rate the SFU sustains in the render kernel's own static-tone loop, with
 * none of the render's staging, set-up or split sums around it -- a measured ceiling to set a
 * render's sines per second against, beside the nominal SFU rate.  Launches on `stream` `blocks`
 * CTAs of 128 threads; each thread runs `runs` runs of 32 samples of one static tone (one SFU
 * sine per sample: blocks x 128 x runs x 32 sines) and writes one float (the sum of its partial
 * sums) to out[thread], a caller-owned device buffer of blocks x 128 floats.  Asynchronous; time
 * it with events on `stream`.  AWG_EINVAL for a null buffer or blocks, runs outside 1 .. 2^20.
 * (The paper has no counterpart.) */
int awg_sfu_rate_probe(float* out, int32_t blocks, int32_t runs, void* stream);

/* Measurement hook: the same for the render kernel's chirp loop (the 32-bit phase cascade
 * p += f, f += g of linear and LOW6 chirps, then the sine and the multiply-add): each thread
 * runs `runs` runs of 32 samples of one chirp state (blocks x 128 x runs x 32 sines) and writes
 * the sum of its partial sums to out[thread].  Same buffer, stream and error rules as
 * awg_sfu_rate_probe.  (The paper has no counterpart.) */
int awg_chirp_rate_probe(float* out, int32_t blocks, int32_t runs, void* stream);

/* ------------------------------------------------------------------------------------------
 * Periodic table on tensor cores.
 * ---------------------------------------------------------------------------------------- */
enum { AWG_PREC_BF16 = 0, AWG_PREC_FP16 = 1 };

/* The whole periodic record x[0 .. 2^log2_len) of the handle's tones as a split-precision GEMM:
 * with n = n1 * 256 + n2, x = sum_k [A_k sin a_k(n1)] cos b_k(n2) + [A_k cos a_k(n1)] sin b_k(n2)
 * (the angle-addition form of Eq. main), a_k, b_k from exact phase words; operands split into
 * hi + lo halves of the chosen precision, products hi*hi + hi*lo + lo*hi accumulated in FP32 on
 * tcgen05 tensor cores.  Requires every tone on the f_s / 2^log2_len grid (awg_set_tones_grid,
 * Eq. freqapprox) and no chirps; 15 <= log2_len <= 30.  Writes int16 codes (full scale of the
 * handle) to out_q and/or the FP32 sum to out_f (either may be NULL, not both), sample n at
 * index n, asynchronously on `stream`.  The cursor is not used or moved.  Operand buffers
 * (2 x 2^(log2_len-8) x 2K 16-bit values, 5.2 GB for 10,000 tones and 2^24 samples) are kept by
 * the handle between calls. */
int awg_table_gemm(awg_t* h, int32_t log2_len, int32_t precision, int16_t* out_q, float* out_f, void* stream);

/* ------------------------------------------------------------------------------------------
 * Streaming ring (the Streaming pathway, Sec. IV-B, with the DAC card replaced by a host sink).
 * n_slots chunk slots of int16 samples live in pinned, device-mapped host memory; awg_ring_push
 * renders the handle's next chunk straight into the next slot; a sink thread plays chunk c at
 * t_start + c * chunk / fs (t_start: when the first `prefill` chunks are complete), reading every
 * sample of the slot, and frees the slot.  A chunk that is not complete at its play time is an
 * underrun (the card's FIFO would have run dry).
 * ---------------------------------------------------------------------------------------- */
typedef struct awg_ring awg_ring_t;

typedef struct {
  int64_t played;            /* chunks played */
  int64_t underruns;         /* chunks that were not complete at their play time */
  double latency_p50_ms;     /* GPU completion minus push time (host clock), per chunk */
  double latency_p99_ms;
  double latency_max_ms;
  double lead_min_ms;        /* play time minus GPU completion: the smallest margin seen */
  double lead_p50_ms;
  double chunk_playback_ms;  /* chunk / fs */
  uint64_t checksum;         /* FNV-style hash over every played sample, in play order */
} awg_ring_stats_t;

/* Ring of n_slots (2..1024) chunks of `chunk` samples (1..2^30) fed by handle h.  NULL on error. */
awg_ring_t* awg_ring_create(awg_t* h, int64_t chunk, int32_t n_slots);

/* Stop the sink (if running), wait for outstanding renders and free the ring.  NULL is allowed. */
void awg_ring_destroy(awg_ring_t* r);

/* Render the handle's next chunk into the next slot on `stream` (asynchronously) and hand it to
 * the sink.  Waits up to timeout_ms while that slot still holds a chunk the sink has not played;
 * AWG_ETIMEOUT if it stays occupied.  Advances the handle's cursor by one chunk. */
int awg_ring_push(awg_ring_t* r, void* stream, int32_t timeout_ms);

/* Start the sink thread: it waits for `prefill` (1..n_slots) chunks, then plays n_chunks chunks
 * (n_chunks < 0: until awg_ring_finish).  If capture is non-NULL, the played samples are also
 * copied there in play order, up to capture_samples. */
int awg_ring_start(awg_ring_t* r, int32_t prefill, int64_t n_chunks, int16_t* capture, int64_t capture_samples);

/* Wait up to timeout_ms for the sink to play its n_chunks, stop it, and fill *out (may be NULL).
 * AWG_ETIMEOUT if the chunks were not all played, or the sink gave up waiting for a chunk. */
int awg_ring_finish(awg_ring_t* r, int32_t timeout_ms, awg_ring_stats_t* out);

/* Host pointer to the samples of slot i (NULL if out of range). */
const int16_t* awg_ring_slot(const awg_ring_t* r, int32_t i);

/* ------------------------------------------------------------------------------------------
 * Served request stream with continuous batching.  A request is a waveform (a comb of tones, some
 * of them chirped, as in the rearrangement of Sec. V-B) that asks for n_chunks consecutive chunks
 * of `chunk` samples, played back at fs one after another (the chunked streaming of Sec. IV).
 * Timing: the first `depth` chunks (awg_server_set_prefetch; default 2; fewer if the request has
 * fewer) are the start-up: rendered as soon as the request is set up on the device; playback
 * starts when they are all complete (t_play; its latency from submission is reported as the
 * first-chunk time), like a FIFO ahead of the DAC that is filled before the DAC starts.  Every
 * later chunk c is due when chunk c-1 ends playing, t_play + c chunk/fs (a chunk completed after
 * that is a deadline miss: an underrun of the player), and is released for rendering `depth`
 * chunk periods earlier.
 * Admission: a request is admitted while the device-memory budget and max_active allow and the
 * real-time budget holds with it: each chunk's window (its look-ahead less the queue horizon, the
 * round cost, twice the longest CTA that cannot be preempted and an allowance for the host's
 * scheduling delay) must hold the chunk's own device time, and the set's device time per period
 * must stay below 85 % of the windows (a cost model fitted at creation).  A request that does not fit waits up to max_queue_ms (without blocking the requests
 * behind it) and is then rejected; one that could never fit is rejected at once.
 * Rounds: the scheduler keeps two rounds in flight; each round takes the released chunks of all
 * active requests in earliest-deadline-first order, cuts the ones that do not fit the round's work
 * budget into whole 4096-sample tiles, and renders them in one batched grid per tone-split size.
 * A request's samples are the same as a standalone render of it (awg_render), whatever runs
 * beside it and however its chunks are cut.
 * ---------------------------------------------------------------------------------------- */
typedef struct awg_server awg_server_t;

enum { AWG_REQ_QUEUED = 0, AWG_REQ_ACTIVE = 1, AWG_REQ_DONE = 2, AWG_REQ_REJECTED = 3 };

typedef struct {
  const double* freq_hz;            /* n_tones: as awg_set_tones */
  const double* amp;
  const double* phase_rad;
  int32_t n_tones;
  const int32_t* chirp_tone;        /* n_chirps: as awg_set_chirps (start samples relative to the
                                       request's first sample) */
  const double* chirp_f_start_hz;
  const double* chirp_f_end_hz;
  const double* chirp_duration_s;
  const int32_t* chirp_profile;
  const int64_t* chirp_start_sample;
  int32_t n_chirps;
  int64_t chunk;                    /* samples per chunk, 1 .. 2^26 */
  int32_t n_chunks;
  double full_scale;                /* <= 0: sum |A| */
} awg_request_t;

typedef struct {
  int64_t submitted, admitted, rejected_deadline, rejected_memory, completed;
  int64_t chunks, deadline_misses;  /* chunks rendered; of those, completed after their deadline */
  double latency_p50_ms;            /* streamed chunks (c >= depth): completion minus release */
  double latency_p99_ms;
  double latency_max_ms;
  double latency_p99_of_period;     /* streamed chunks: p99 of (completion - release) / playback period */
  double first_chunk_p50_ms;        /* playback start (start-up complete) minus submission */
  double first_chunk_p99_ms;
  int64_t rounds;
  double mean_batch;                /* pieces (requests) per round */
  int64_t max_batch;
  double tone_samples_per_s;        /* tones x samples rendered, over the span from the first round to the last */
  double samples_per_s;
  double busy_fraction;             /* device time of the rounds / that span */
  double est_throughput;            /* cost model: static-tone samples/s of a busy device */
  double est_round_cost_ms;         /* cost model: fixed device time of one round */
  double est_cta_rate;              /* cost model: tone-samples/s of one render CTA alone on an SM */
  double est_engine_throughput;     /* cost model: static tone-samples/s of the tensor-core engine */
} awg_server_stats_t;

/* Server for sample rate fs on the current device, with a device-memory budget (bytes) for the
 * requests' state and outputs, at most max_active concurrent requests, and at most max_queue_ms
 * of waiting for admission.  NULL on error (see awg_last_error). */
awg_server_t* awg_server_create(double sample_rate_hz, int64_t mem_budget_bytes, int32_t max_active,
                                double max_queue_ms);

/* Static tones of requests with at least min_tones tones on the tensor-core engine (engine
 * AWG_STATIC_GEMM_FP16 or _BF16, as awg_set_static_engine): each piece's static tones are summed by
 * the split-precision GEMM over the piece (within 1 LSB of the oracle, not bit-identical to the
 * direct render), only the tones that chirp or ramp in it go through the batched render kernel.
 * A served request equals a standalone render with the same engine bit for bit.  AWG_STATIC_DIRECT
 * (the default) renders every tone directly.  Set before the first request; AWG_ESTATE after. */
int awg_server_set_static_engine(awg_server_t* s, int32_t engine, int32_t min_tones);

/* Chunks rendered ahead of playback (1 .. 16, default 2): the first `depth` chunks are rendered
 * before playback starts, and chunk c is released when chunk c - depth starts playing.  Set
 * before the first request; AWG_ESTATE after. */
int awg_server_set_prefetch(awg_server_t* s, int32_t chunks);

/* Stop the scheduler, wait for in-flight work and free everything.  NULL is allowed. */
void awg_server_destroy(awg_server_t* s);

/* Queue a request (arrays are copied); returns its id (>= 0) or a negative AWG_E* code. */
int64_t awg_server_submit(awg_server_t* s, const awg_request_t* req);

/* State (AWG_REQ_*) and number of rendered chunks of request id. */
int awg_server_poll(awg_server_t* s, int64_t id, int32_t* state, int32_t* chunks_done);

/* Copy the first n_samples samples of a finished request to host memory (AWG_ESTATE if not done). */
int awg_server_read(awg_server_t* s, int64_t id, int16_t* host_out, int64_t n_samples);

/* Forget a finished or rejected request and free its output (done by the scheduler thread). */
int awg_server_release(awg_server_t* s, int64_t id);

/* Wait up to timeout_ms until no request is queued or active. */
int awg_server_drain(awg_server_t* s, int32_t timeout_ms);

/* Counters and latency percentiles so far. */
int awg_server_stats(awg_server_t* s, awg_server_stats_t* out);

/* Trace of the most recent rounds and chunk completions (the last 65,536 of each; times on the
 * server clock, seconds since awg_server_create; device times mapped through an event recorded at
 * creation).  Each call copies up to cap records, oldest first, and returns how many (or a
 * negative AWG_E* code). */
typedef struct {
  double t_plan;                    /* host: planning started */
  double t_issued;                  /* host: all launches of the round issued */
  double t_start, t_done;           /* device: round start and end */
  double work;                      /* tone-samples */
  double first_due;                 /* earliest due time among the round's streamed chunks */
  int32_t pieces, tiles;
} awg_round_record_t;

typedef struct {
  int64_t id;                       /* request */
  int32_t chunk, late;              /* late: completed after its due time */
  double release, due, done;        /* start-up chunk c: release = set-up done, due = release + (c+1) period */
} awg_chunk_record_t;

int32_t awg_server_trace_rounds(awg_server_t* s, awg_round_record_t* out, int32_t cap);
int32_t awg_server_trace_chunks(awg_server_t* s, awg_chunk_record_t* out, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* AWG_H */
