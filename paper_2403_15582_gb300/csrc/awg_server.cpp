// Served request stream with continuous batching (C ABI in include/awg.h).
//
// A request is a tweezer-rearrangement waveform (Sec. V-B: a comb of static tones, some of them
// chirped) that asks for n_chunks consecutive chunks of `chunk` samples.  Chunk c is released at
// arrival + c * chunk / fs (when the previous chunk would start playing) and is due one playback
// period later.  A scheduler thread admits requests while device memory and the real-time budget
// allow, keeps each admitted request's tone and chirp state resident on the device (one handle
// per request), and in every round renders all released chunks of all active requests in one
// batched grid per tone-split size.  Each (request, tile) is computed exactly as a standalone
// render of that request would compute it, so a result does not depend on its co-runners.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/awg.h"
#include "awg_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  // description (host copies)
  std::vector<double> f, a, th, c_f0, c_f1, c_dur;
  std::vector<int32_t> c_tone, c_prof;
  std::vector<int64_t> c_start;
  int64_t chunk = 0;
  int32_t n_chunks = 0;
  double full_scale = 0;
  double t_arrival = 0;        // server clock, seconds
  double period = 0;           // playback time of one chunk, s
  // state
  int32_t state = AWG_REQ_QUEUED;
  awg_t* h = nullptr;
  int16_t* d_out = nullptr;
  size_t mem = 0, out_bytes = 0;
  bool ready = false;          // set-up done: renderable
  bool release_requested = false;
  int32_t split = 1;           // tone split of its render (of the render part, with the engine)
  bool engine = false;         // static tones on the tensor-core engine (awg_server_set_static_engine)
  double weight = 0;           // device cost per sample, in static-tone units: K + n_chirps / 2, or
                               // with the engine K / engine_gain + 1.5 n_chirps
  double cta_tones = 0;        // tones one CTA sums (K / tone split, rounded up)
  int32_t issue_chunk = 0;     // next piece to issue: chunk index and offset in it
  int64_t issue_off = 0;
  int32_t done_chunks = 0;     // chunks complete on the device
  double t_ready = -1;         // set-up finished
  int32_t n_start = 1;         // start-up chunks (min(depth, n_chunks)), rendered before playback
  int32_t start_done = 0;      // start-up chunks complete
  double t_start_max = 0;      // latest completion among them
  double t_play = -1;          // every start-up chunk complete: playback starts
  double t_pieces = 0;         // latest completion among the pieces of the chunk being completed
};

// One round: pieces (a request's chunk, or a tile-aligned part of it) rendered by one batched
// grid per tone-split size.
struct Piece {
  Request* r;
  int32_t chunk;
  int64_t off, n;
  bool last;                   // completes its chunk
};

struct Round {
  int set = 0;                 // staging buffers and events in use
  std::vector<Piece> pieces;
  double work = 0;             // cost in static-tone samples (Request::weight x samples)
  double tone_samples = 0;     // tone-samples rendered (tones x samples)
  double host_s = 0;           // host time to plan and issue
  awg_round_record_t rec{};
};

// Fixed-capacity trace of the most recent records.
template <class T>
struct TraceRing {
  static constexpr size_t CAP = 1u << 16;
  std::vector<T> buf;
  size_t n = 0;                // records written so far
  void push(const T& x) {
    if (buf.size() < CAP) buf.push_back(x);
    else buf[n % CAP] = x;
    ++n;
  }
  int32_t copy(T* out, int32_t cap) const {
    const size_t have = std::min(n, CAP), take = std::min(have, (size_t)std::max(0, cap));
    const size_t first = n - have + (have - take);   // skip the oldest when cap is short
    for (size_t i = 0; i < take; ++i) out[i] = buf[(first + i) % CAP];
    return (int32_t)take;
  }
};

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

constexpr int NSETS = 3;       // rounds in flight, each on its own stream with its own buffers
constexpr int RESIDENT = 5;    // render CTAs resident per SM
// partial tiles of the split sums per round set, allocated up front (256 MiB each): a round of a
// full 2 ms horizon at ~3e12 tone-samples/s is ~15,000 CTAs of 96 tones; larger rounds grow it
constexpr size_t PART_TILES = 16384;

struct awg_server {
  double fs = 0;
  int64_t budget = 0;
  int32_t max_active = 0;
  int32_t depth = 2;           // chunks rendered ahead of playback (awg_server_set_prefetch)
  int32_t engine = AWG_STATIC_DIRECT;   // static-tone engine for requests of >= engine_min_tones tones
  int32_t engine_min_tones = 0;
  cudaStream_t setup_stream = nullptr;  // the worker's stream (engine operands at set-up)
  double max_queue_s = 0;
  int device = 0;
  clk::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::atomic<int64_t> epoch{0};                  // bumped by submit / set-up done / release / stop
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<int64_t, Request*> all;
  int64_t next_id = 0;
  int64_t used = 0;
  std::thread sched, worker;
  std::atomic<bool> stop{false};
  std::deque<Request*> to_setup;                  // admitted, waiting for set-up (worker thread)
  std::vector<awg_t*> idle_handles;               // pooled handles (state is replaced on reuse)
  std::map<size_t, std::vector<int16_t*>> idle_out;   // pooled output buffers by byte size
  // per set: stream, events, staging and device copies of the round's descriptors, tile records
  cudaStream_t streams[NSETS] = {};
  cudaEvent_t ev_ref = nullptr, ev_beg[NSETS] = {}, ev_end[NSETS] = {};
  double t_ref = 0;                               // server clock when ev_ref completed
  awgk::RenderArgs* h_reqs[NSETS] = {};
  int2* h_items[NSETS] = {};
  awgk::RenderArgs* d_reqs[NSETS] = {};
  int2* d_items[NSETS] = {};
  awgk::TileRec* d_arena[NSETS] = {};
  int32_t* d_act[NSETS] = {};
  size_t cap_reqs[NSETS] = {}, cap_items[NSETS] = {}, cap_arena[NSETS] = {}, cap_act[NSETS] = {};
  // split sums of the batched renders: partial tiles (items x split x TILE floats) and a counter
  // per item, per set
  float* d_part[NSETS] = {};
  unsigned long long* d_tctr[NSETS] = {};
  size_t cap_part[NSETS] = {}, cap_tctr[NSETS] = {};
  // tensor-core engine pieces: the GEMM's FP32 sums and the tone lists of the round (device, and
  // the lists' pinned staging)
  float* d_base[NSETS] = {};
  int32_t* d_list[NSETS] = {};
  int32_t* h_list[NSETS] = {};
  size_t cap_base[NSETS] = {}, cap_list[NSETS] = {};
  std::deque<Round> flight;
  int64_t round_seq = 0;
  double queued_work = 0;      // tone-samples issued and not yet accounted complete (rounds on the
                               // three streams overlap: the queue drains at the busy-device rate P)
  double busy_end = -1;        // end of the device's current busy interval (server clock)
  // cost model (calibrated at creation): the device renders P static-tone samples/s when it is
  // kept busy (updated from busy rounds within [0.6, 1.2] of the calibration); a round costs a_gpu
  // more (descriptor copies, launches)
  double P = 2.5e12, P_cal = 2.5e12;
  double a_gpu = 20e-6;
  double r_cta = 1e10;         // tone-samples/s of one CTA alone on its SM
  double P_engine = 0;         // static tone-samples/s of the tensor-core engine on a busy device
  double host_s = 30e-6;
  // statistics
  int64_t submitted = 0, admitted = 0, rej_deadline = 0, rej_memory = 0, completed = 0;
  int64_t chunks = 0, misses = 0, rounds = 0, batched = 0, max_batch = 0;
  std::vector<double> lat, ttfc, lat_frac;
  TraceRing<awg_round_record_t> trace_rounds;
  TraceRing<awg_chunk_record_t> trace_chunks;
  double busy_s = 0, tone_samples = 0, samples = 0;
  double first_t = -1, last_t = 0;
  std::string error;
};

namespace {

double now_s(const awg_server_t* s) { return std::chrono::duration<double>(clk::now() - s->t0).count(); }

// Release and due time of a streamed chunk c >= depth of a playing request (server clock): due
// when chunk c-1 ends playing, t_play + c period; released a look-ahead of `depth` periods
// earlier, which is never before t_play.  The first `depth` chunks (the start-up) are rendered
// before playback starts, so every streamed chunk has the whole look-ahead.  (With playback
// starting after chunk 0 alone, chunk 1 had one period instead of `depth`: the chunks that missed
// at low load.  A minimum look-ahead of 1 ms for short chunks was tried as well: chunks released
// that early crowded the device queue and more of them missed.)
double lookahead(const awg_server_t* s, const Request* r) { return (double)s->depth * r->period; }
double chunk_due(const Request* r, int32_t c) { return r->t_play + (double)c * r->period; }
double chunk_release(const awg_server_t* s, const Request* r, int32_t c) {
  return std::max(r->t_play, chunk_due(r, c) - lookahead(s, r));
}

// The request's cost in static-tone units per sample and its longest CTA in tones: direct render
// K + n_chirps / 2 (a chirping tone costs about one and a half static ones) and K / split tones per
// CTA; with the engine, K times the engine's cost ratio plus the chirping tones, and the longer of
// a render CTA and a GEMM CTA (128 rows of 256 samples over a quarter of the tones) in the same
// units.
void set_cost(const awg_server_t* s, Request* r) {
  const double K = (double)r->f.size(), nc = (double)r->c_tone.size();
  if (r->engine && s->P_engine > 0) {
    r->weight = K * s->P / s->P_engine + 1.5 * nc;
    const int split = awgk::tone_split_for((int)r->c_tone.size());
    const double render_cta = std::ceil(nc / split);
    const double gemm_cta_s = 32768.0 * std::max(1.0, K / 4.0) / (s->P_engine / (double)awgk::device_sm_count());
    r->cta_tones = std::max(render_cta, gemm_cta_s * s->r_cta / awgk::TILE);
  } else {
    r->weight = K + 0.5 * nc;
    const int split = awgk::tone_split_for((int)r->f.size());
    r->cta_tones = (double)(((int)r->f.size() + split - 1) / split);
  }
}

// Device time of one CTA of request r alone on an SM (its tones per CTA over the calibrated rate
// of a lone CTA), and of a chunk or a round alone: its fixed cost plus the larger of its work at
// the busy-device rate and its longest CTA (a small round cannot spread over the device).
double cta_time(const awg_server_t* s, const Request* r) { return r->cta_tones * awgk::TILE / s->r_cta; }
double round_time(const awg_server_t* s, double work, double t_cta_max) {
  return s->a_gpu + std::max(work / s->P, t_cta_max);
}

size_t footprint(const Request* r) {
  const size_t tiles = (size_t)(r->chunk + 2 * awgk::TILE - 1) / awgk::TILE;
  return (size_t)r->f.size() * sizeof(awgk::ToneRec) + r->c_tone.size() * sizeof(awgk::ChirpRec) +
         r->c_tone.size() * tiles * sizeof(awgk::TileRec) + (size_t)r->n_chunks * (size_t)r->chunk * 2 + (64u << 10);
}

// Queue horizon for a set whose shortest chunk period is min_period: the scheduler issues work
// only while the device has less than this much queued, so a newly released chunk starts within
// about one horizon.
double horizon(double min_period) { return std::min(2e-3, std::max(40e-6, min_period / 3.0)); }

// Admission by the real-time budget (EDF with release jitter): chunk i needs C_i = K_i chunk_i / P
// of device time per period T_i and must be done within its window W_i = lookahead_i - H - a_gpu -
// 2 t_cta - J (released a look-ahead before its due time, less the queue horizon H, the round
// cost a_gpu, twice the longest non-preemptible CTA and the host's release jitter J), which must
// also hold the chunk's own time alone (round_time).  The set is accepted while that holds for
// every request and sum C_i / min(T_i, W_i) <= 0.85 (the density test where windows are short, the
// utilisation test where they exceed a period), and one tile of the largest request fits in a
// horizon.
constexpr double HOST_JITTER_S = 150e-6;   // release-to-plan delay the host may add (scheduler wake-up)

bool fits_set(const awg_server_t* s, const std::vector<const Request*>& set) {
  double min_period = 1e30, kmax = 0, ctamax = 0, load = 0;
  for (const Request* q : set) {
    min_period = std::min(min_period, q->period);
    kmax = std::max(kmax, (double)q->f.size());
    ctamax = std::max(ctamax, q->cta_tones);
    load += q->weight * s->fs / s->P;
  }
  if (set.empty()) return true;
  const double H = horizon(min_period);
  // A CTA cannot be preempted: a chunk may wait for the longest CTA in flight and takes at least
  // one CTA time itself.  A CTA shares its SM with up to RESIDENT others as the load grows.
  const double t_cta = ctamax * awgk::TILE / s->r_cta * (1.0 + (RESIDENT - 1) * std::min(1.0, load));
  double density = 0;
  for (const Request* q : set) {
    const double window = lookahead(s, q) - H - s->a_gpu - 2.0 * t_cta - HOST_JITTER_S;
    if (window <= round_time(s, q->weight * (double)q->chunk, cta_time(s, q))) return false;
    density += q->weight * (double)q->chunk / s->P / std::min(q->period, window);
  }
  return density <= 0.85 && kmax * awgk::TILE / s->P <= H;
}

bool fits_deadline(const awg_server_t* s, const Request* extra) {
  std::vector<const Request*> set(s->active.begin(), s->active.end());
  if (extra) set.push_back(extra);
  return fits_set(s, set);
}

// Could `r` ever be admitted (alone, with an idle device)?
bool fits_alone(const awg_server_t* s, const Request* r) { return fits_set(s, {r}); }

bool start_request(awg_server_t* s, Request* r) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->idle_handles.empty()) {
      r->h = s->idle_handles.back();
      s->idle_handles.pop_back();
    }
  }
  if (!r->h) r->h = awg_create(s->fs);
  if (!r->h) return false;
  if (awg_seek(r->h, 0)) return false;
  const int32_t K = (int32_t)r->f.size();
  if (awg_set_tones(r->h, r->f.data(), r->a.data(), r->th.data(), K)) return false;
  if (!r->c_tone.empty() &&
      awg_set_chirps(r->h, r->c_tone.data(), r->c_f0.data(), r->c_f1.data(), r->c_dur.data(), r->c_prof.data(),
                     r->c_start.data(), (int32_t)r->c_tone.size()))
    return false;
  if (awg_set_full_scale(r->h, r->full_scale)) return false;
  r->split = awg_tone_split(r->h);
  awg_set_static_engine(r->h, AWG_STATIC_DIRECT);
  if (r->engine) {   // B operand of the request's GEMM, once: its tone state is fixed from here on
    if (awgk::engine_setup(r->h, s->engine, s->setup_stream, &r->split) != AWG_OK) return false;
    if (cudaStreamSynchronize(s->setup_stream) != cudaSuccess) return false;
  }
  r->out_bytes = std::max<size_t>((size_t)r->n_chunks * (size_t)r->chunk * sizeof(int16_t), 16);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->idle_out.find(r->out_bytes);
    if (it != s->idle_out.end() && !it->second.empty()) {
      r->d_out = it->second.back();
      it->second.pop_back();
    }
  }
  if (!r->d_out && cudaMalloc((void**)&r->d_out, r->out_bytes) != cudaSuccess) return false;
  return true;
}

// Handles go back to the pool instead of being destroyed (no device allocation in steady state).
void recycle_handle(awg_server_t* s, Request* r) {
  if (r->h) s->idle_handles.push_back(r->h);
  r->h = nullptr;
}

void destroy_handle(Request* r) {
  if (r->h) awg_destroy(r->h);
  r->h = nullptr;
}

void bump(awg_server_t* s) {
  s->epoch.fetch_add(1);
  s->cv.notify_all();
}

// Set-up of admitted requests (handle, tone and chirp state, output buffer) off the scheduler's
// critical path.
void worker_main(awg_server_t* s) {
  cudaSetDevice(s->device);
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop.load() || !s->to_setup.empty(); });
      if (s->stop.load()) return;
      if (s->to_setup.empty()) continue;
      r = s->to_setup.front();
      s->to_setup.pop_front();
    }
    const bool ok = start_request(s, r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (ok) {
        r->ready = true;
        r->t_ready = now_s(s);
        r->n_start = std::max<int32_t>(1, std::min(s->depth, r->n_chunks));
      } else {
        s->error = std::string("request set-up failed: ") + awg_last_error();
        r->state = AWG_REQ_REJECTED;
        ++s->rej_memory;
        s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        s->used -= (int64_t)r->mem;
        if (r->d_out) s->idle_out[r->out_bytes].push_back(r->d_out);
        r->d_out = nullptr;
        recycle_handle(s, r);
      }
    }
    bump(s);
  }
}

template <class T>
bool grow(T** dev, T** host, size_t* cap, size_t need) {
  if (need <= *cap) return true;
  size_t ncap = std::max(need, *cap * 2);
  T *d = nullptr, *h = nullptr;
  if (cudaMalloc((void**)&d, ncap * sizeof(T)) != cudaSuccess) return false;
  if (cudaHostAlloc((void**)&h, ncap * sizeof(T), cudaHostAllocDefault) != cudaSuccess) {
    cudaFree(d);
    return false;
  }
  cudaFree(*dev);
  cudaFreeHost(*host);
  *dev = d;
  *host = h;
  *cap = ncap;
  return true;
}

// Retire released outputs; admit queued requests (any order: a request that does not fit yet
// waits, up to max_queue_s, without blocking those behind it).  Lock held.
void admit(awg_server_t* s) {
  for (auto it = s->all.begin(); it != s->all.end();) {
    Request* r = it->second;
    if (r->release_requested && (r->state == AWG_REQ_DONE || r->state == AWG_REQ_REJECTED)) {
      if (r->d_out) {
        s->idle_out[r->out_bytes].push_back(r->d_out);
        s->used -= (int64_t)r->out_bytes;
      }
      delete r;
      it = s->all.erase(it);
    } else {
      ++it;
    }
  }
  const double now = now_s(s);
  bool changed = false;
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request* r = *it;
    const size_t mem = footprint(r);
    int decision = 0;   // 0 wait, 1 admit, -1 reject (deadline), -2 reject (memory)
    if (!fits_alone(s, r)) {
      decision = -1;
    } else if ((int64_t)mem > s->budget) {
      decision = -2;
    } else {
      const bool mem_ok = s->used + (int64_t)mem <= s->budget && (int32_t)s->active.size() < s->max_active;
      const bool rt_ok = fits_deadline(s, r);
      if (mem_ok && rt_ok) decision = 1;
      else if (now - r->t_arrival > s->max_queue_s) decision = rt_ok ? -2 : -1;
    }
    if (decision == 0) {
      ++it;
      continue;
    }
    changed = true;
    if (decision == 1) {
      r->mem = mem;
      s->used += (int64_t)mem;
      r->state = AWG_REQ_ACTIVE;
      ++s->admitted;
      s->active.push_back(r);
      s->to_setup.push_back(r);
    } else {
      r->state = AWG_REQ_REJECTED;
      ++(decision == -1 ? s->rej_deadline : s->rej_memory);
    }
    it = s->pending.erase(it);
  }
  if (changed) s->cv.notify_all();   // worker; awg_server_drain / poll
}

// Earliest-deadline-first plan of one round at time `now`.  The start-up chunks of a request
// (the first min(depth, n_chunks)) are released when its set-up is done; it starts playback when
// they are all complete (t_play), and chunk c >= depth is due when chunk c-1 ends (t_play + c
// period) and released `depth` periods earlier (chunk_release).  A round takes what fills the device's queue up to the horizon; a chunk
// that does not fit is cut into whole tiles and continued in later rounds.
// Returns the earliest future release in *next_release.  Lock held.
void plan_round(awg_server_t* s, double now, Round* rd, double* next_release) {
  struct Cand {
    double due;
    Request* r;
  };
  std::vector<Cand> cands;
  double min_period = 1e30;
  *next_release = 1e30;
  for (Request* r : s->active) {
    min_period = std::min(min_period, r->period);
    if (!r->ready || r->issue_chunk >= r->n_chunks) continue;
    const int32_t c = r->issue_chunk;
    double rel, due;
    if (c < r->n_start) {            // start-up chunk: released at once, ordered by index
      rel = r->t_ready;
      due = r->t_ready + (double)(c + 1) * r->period;
    } else {
      if (r->t_play < 0) continue;   // start-up still in flight
      rel = chunk_release(s, r, c);
      due = chunk_due(r, c);
    }
    if (rel <= now) cands.push_back({due, r});
    else *next_release = std::min(*next_release, rel);
  }
  if (cands.empty()) return;
  // work the device may take on now: fill the queue up to the horizon
  const double H = horizon(min_period);
  const double queued = s->queued_work / s->P;
  if (!s->flight.empty() && queued >= H) return;
  double w_left = std::max(0.5 * H, H - queued - s->a_gpu) * s->P;
  std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.due < y.due; });
  rd->rec.first_due = 1e30;
  for (const Cand& cd : cands)
    if (cd.r->issue_chunk >= cd.r->n_start) {
      rd->rec.first_due = cd.due;
      break;
    }
  for (const Cand& cd : cands) {
    if (w_left <= 0 && !rd->pieces.empty()) break;
    Request* r = cd.r;
    const double K = std::max(1.0, r->weight);
    const int64_t remaining = r->chunk - r->issue_off;
    int64_t take = remaining;
    if (K * (double)take > w_left) {
      const int64_t tiles = std::max<int64_t>(1, (int64_t)(w_left / K) / awgk::TILE);
      take = std::min(remaining, tiles * awgk::TILE);
    }
    rd->pieces.push_back({r, r->issue_chunk, r->issue_off, take, take == remaining});
    rd->work += K * (double)take;
    rd->tone_samples += (double)r->f.size() * (double)take;
    w_left -= K * (double)take;
    r->issue_off += take;
    if (r->issue_off == r->chunk) {
      r->issue_off = 0;
      ++r->issue_chunk;
    }
  }
}

// Issue a planned round on its set's stream (outside the lock: only this thread touches active
// requests' handles).  The round's tile records live in the set's arena, so rounds on the other
// streams (including other pieces of the same request) can run at the same time.
bool issue_round(awg_server_t* s, Round* rd) {
  const int set = rd->set;
  cudaStream_t st = s->streams[set];
  std::sort(rd->pieces.begin(), rd->pieces.end(),
            [](const Piece& x, const Piece& y) { return x.r->split < y.r->split; });
  std::vector<size_t> rec0(rd->pieces.size() + 1, 0), act0(rd->pieces.size() + 1, 0);
  for (size_t i = 0; i < rd->pieces.size(); ++i) {
    rec0[i + 1] = rec0[i] + awgk::render_recs_needed(rd->pieces[i].r->h, rd->pieces[i].n);
    act0[i + 1] = act0[i] + awgk::render_slots(rd->pieces[i].r->h);
  }
  // grow: the set's previous round is complete (it left the flight queue), so nothing uses them
  if (rec0.back() > s->cap_arena[set]) {
    const size_t ncap = std::max(rec0.back(), 2 * s->cap_arena[set]);
    awgk::TileRec* a = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(awgk::TileRec)) != cudaSuccess) return false;
    cudaFree(s->d_arena[set]);
    s->d_arena[set] = a;
    s->cap_arena[set] = ncap;
  }
  if (act0.back() > s->cap_act[set]) {
    const size_t ncap = std::max(act0.back(), 2 * s->cap_act[set]);
    int32_t* a = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(int32_t)) != cudaSuccess) return false;
    cudaFree(s->d_act[set]);
    s->d_act[set] = a;
    s->cap_act[set] = ncap;
  }
  // engine pieces: the GEMM's sum of the piece's samples and its tone list
  std::vector<size_t> base0(rd->pieces.size() + 1, 0), list0(rd->pieces.size() + 1, 0);
  for (size_t i = 0; i < rd->pieces.size(); ++i) {
    const Piece& p = rd->pieces[i];
    base0[i + 1] = base0[i] + (p.r->engine ? (size_t)p.n : 0);
    list0[i + 1] = list0[i] + (p.r->engine ? awgk::engine_list_needed(p.r->h, p.n) : 0);
  }
  if (base0.back() > s->cap_base[set]) {
    const size_t ncap = std::max(base0.back(), 2 * s->cap_base[set]);
    float* a = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(float)) != cudaSuccess) return false;
    cudaFree(s->d_base[set]);
    s->d_base[set] = a;
    s->cap_base[set] = ncap;
  }
  if (list0.back() > s->cap_list[set]) {
    const size_t ncap = std::max(list0.back(), 2 * s->cap_list[set]);
    int32_t *a = nullptr, *b = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(int32_t)) != cudaSuccess) return false;
    if (cudaHostAlloc((void**)&b, ncap * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
      cudaFree(a);
      return false;
    }
    cudaFree(s->d_list[set]);
    cudaFreeHost(s->h_list[set]);
    s->d_list[set] = a;
    s->h_list[set] = b;
    s->cap_list[set] = ncap;
  }
  std::vector<awgk::RenderArgs> ra(rd->pieces.size());
  size_t n_items = 0;
  bool ok = cudaEventRecord(s->ev_beg[set], st) == cudaSuccess;
  for (size_t i = 0; i < rd->pieces.size() && ok; ++i) {
    const Piece& p = rd->pieces[i];
    int16_t* out = p.r->d_out + (size_t)p.chunk * (size_t)p.r->chunk + (size_t)p.off;
    const bool own = rec0[i + 1] > rec0[i];   // chirp tile records in this piece
    if (p.r->engine) {
      bool need = false;
      ok = awgk::prepare_render_engine(p.r->h, p.n, out, st, &ra[i], own ? s->d_arena[set] + rec0[i] : nullptr,
                                       rec0[i + 1] - rec0[i], own ? s->d_act[set] + act0[i] : nullptr,
                                       s->d_base[set] + base0[i], s->d_list[set] + list0[i],
                                       s->h_list[set] + list0[i], list0[i + 1] - list0[i], &need) == AWG_OK;
      if (!need) ra[i].n_tiles = 0;   // the GEMM wrote the samples: no render item
    } else {
      ok = awgk::prepare_render(p.r->h, p.n, out, nullptr, st, &ra[i], own ? s->d_arena[set] + rec0[i] : nullptr,
                                rec0[i + 1] - rec0[i], own ? s->d_act[set] + act0[i] : nullptr) == AWG_OK;
    }
    n_items += (size_t)ra[i].n_tiles;
  }
  rd->rec.pieces = (int32_t)rd->pieces.size();
  rd->rec.tiles = (int32_t)n_items;
  // the split sums' scratch: piece i's partial tiles and tile counters after those of pieces < i
  size_t part_need = 0, ctr_need = 0;
  for (size_t i = 0; i < rd->pieces.size(); ++i) {
    part_need += (size_t)ra[i].n_tiles * (size_t)ra[i].split * awgk::TILE;
    ctr_need += (size_t)ra[i].n_tiles;
  }
  if (ok && part_need > s->cap_part[set]) {   // the set's previous round is complete
    const size_t ncap = std::max(part_need, 2 * s->cap_part[set]);
    float* a = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(float)) != cudaSuccess) return false;
    cudaFree(s->d_part[set]);
    s->d_part[set] = a;
    s->cap_part[set] = ncap;
  }
  if (ok && ctr_need > s->cap_tctr[set]) {
    const size_t ncap = std::max(ctr_need, 2 * s->cap_tctr[set]);
    unsigned long long* a = nullptr;
    if (cudaMalloc((void**)&a, ncap * sizeof(unsigned long long)) != cudaSuccess) return false;
    cudaFree(s->d_tctr[set]);
    s->d_tctr[set] = a;
    s->cap_tctr[set] = ncap;
  }
  size_t part_off = 0, ctr_off = 0;
  for (size_t i = 0; i < rd->pieces.size(); ++i) {
    ra[i].part = s->d_part[set] + part_off;
    ra[i].tile_ctr = s->d_tctr[set] + ctr_off;
    part_off += (size_t)ra[i].n_tiles * (size_t)ra[i].split * awgk::TILE;
    ctr_off += (size_t)ra[i].n_tiles;
  }
  ok = ok && cudaMemsetAsync(s->d_tctr[set], 0, ctr_need * sizeof(unsigned long long), st) == cudaSuccess;
  ok = ok && grow(&s->d_reqs[set], &s->h_reqs[set], &s->cap_reqs[set], rd->pieces.size()) &&
       grow(&s->d_items[set], &s->h_items[set], &s->cap_items[set], n_items);
  if (!ok) return false;
  size_t it = 0;
  for (size_t i = 0; i < rd->pieces.size(); ++i) {
    s->h_reqs[set][i] = ra[i];
    for (int32_t t = 0; t < ra[i].n_tiles; ++t) s->h_items[set][it++] = make_int2((int)i, t);
  }
  ok = cudaMemcpyAsync(s->d_reqs[set], s->h_reqs[set], rd->pieces.size() * sizeof(awgk::RenderArgs),
                       cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(s->d_items[set], s->h_items[set], n_items * sizeof(int2), cudaMemcpyHostToDevice, st) ==
           cudaSuccess;
  size_t b = 0, item0 = 0;
  while (ok && b < rd->pieces.size()) {
    size_t e = b, items = 0;
    while (e < rd->pieces.size() && rd->pieces[e].r->split == rd->pieces[b].r->split)
      items += (size_t)ra[e++].n_tiles;
    ok = awgk::launch_render_batch_split(s->d_reqs[set], s->d_items[set] + item0, (int)items,
                                         rd->pieces[b].r->split, st) == cudaSuccess;
    item0 += items;
    b = e;
  }
  return ok && cudaEventRecord(s->ev_end[set], st) == cudaSuccess;
}

// Account for the oldest round once its end event has completed.
void complete_round(awg_server_t* s) {
  Round rd = std::move(s->flight.front());
  s->flight.pop_front();
  float end_ms = 0.f, gpu_ms = 0.f;
  cudaEventElapsedTime(&end_ms, s->ev_ref, s->ev_end[rd.set]);
  cudaEventElapsedTime(&gpu_ms, s->ev_beg[rd.set], s->ev_end[rd.set]);
  const double t_done = s->t_ref + 1e-3 * (double)end_ms;   // device completion, server clock
  const double t_start = t_done - 1e-3 * (double)gpu_ms;    // the round's stream reached it
  std::vector<Request*> finished;
  std::lock_guard<std::mutex> lk(s->mu);
  rd.rec.t_start = t_start;
  rd.rec.t_done = t_done;
  rd.rec.work = rd.work;
  s->trace_rounds.push(rd.rec);
  s->queued_work = std::max(0.0, s->queued_work - rd.work);
  ++s->rounds;
  s->batched += (int64_t)rd.pieces.size();
  s->max_batch = std::max(s->max_batch, (int64_t)rd.pieces.size());
  s->tone_samples += rd.tone_samples;
  if (s->first_t < 0) s->first_t = t_start;
  s->last_t = std::max(s->last_t, t_done);
  // a round that found the device busy measures the sustained rate: its work over the advance of
  // the busy interval's end
  if (t_done > s->busy_end && rd.work > 0) {
    if (t_start < s->busy_end) {
      const double rate = rd.work / (t_done - s->busy_end);
      s->P = std::min(1.2 * s->P_cal, std::max(0.6 * s->P_cal, 0.95 * s->P + 0.05 * rate));
      s->busy_s += t_done - s->busy_end;
    } else {
      s->busy_s += t_done - t_start;
    }
    s->busy_end = t_done;
  }
  s->host_s = 0.9 * s->host_s + 0.1 * rd.host_s;
  for (const Piece& p : rd.pieces) {
    Request* r = p.r;
    r->t_pieces = std::max(r->t_pieces, t_done);
    if (!p.last) continue;
    const double t_chunk = r->t_pieces;   // all pieces of the chunk are complete
    r->t_pieces = 0;
    awg_chunk_record_t cr{};
    cr.id = r->id;
    cr.chunk = p.chunk;
    cr.done = t_chunk;
    if (p.chunk < r->n_start) {
      r->t_start_max = std::max(r->t_start_max, t_chunk);
      if (++r->start_done == r->n_start) {   // the player's buffer is full: playback starts
        r->t_play = r->t_start_max;
        s->ttfc.push_back(r->t_play - r->t_arrival);
      }
      cr.release = r->t_ready;
      cr.due = r->t_ready + (double)(p.chunk + 1) * r->period;
    } else {
      const double rel = chunk_release(s, r, p.chunk);
      s->lat.push_back(t_chunk - rel);
      s->lat_frac.push_back((t_chunk - rel) / r->period);
      cr.release = rel;
      cr.due = chunk_due(r, p.chunk);
      cr.late = t_chunk > cr.due;
      if (cr.late) ++s->misses;
    }
    s->trace_chunks.push(cr);
    ++s->chunks;
    s->samples += (double)r->chunk;
    r->done_chunks = p.chunk + 1;
    if (r->done_chunks == r->n_chunks) finished.push_back(r);
  }
  for (Request* r : finished) {
    r->state = AWG_REQ_DONE;
    ++s->completed;
    s->active.erase(std::find(s->active.begin(), s->active.end(), r));
    recycle_handle(s, r);
    s->used -= (int64_t)(r->mem - r->out_bytes);
  }
  s->cv.notify_all();
}

void fail_rounds(awg_server_t* s, const std::string& what) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->error = what + ": " + awg_last_error();
  s->stop.store(true);
  s->cv.notify_all();
}

// The tensor-core engine's rate: rounds of one request of K static tones over N samples with the
// engine (best of three, after a warm-up), through the same path as the served rounds.
int calibrate_engine(awg_server_t* s, int32_t K, int64_t N) {
  std::vector<double> f(K), a(K, 1.0 / K), th(K, 0.0);
  for (int32_t k = 0; k < K; ++k) f[k] = s->fs * (0.01 + 0.4 * (double)k / K);
  awg_t* h = awg_create(s->fs);
  int16_t* out = nullptr;
  int st = h ? AWG_OK : AWG_ECUDA;
  if (!st && cudaMalloc((void**)&out, (size_t)N * sizeof(int16_t)) != cudaSuccess)
    st = awgk::set_error(AWG_ENOMEM, "calibration buffer");
  if (!st) st = awg_set_tones(h, f.data(), a.data(), th.data(), K);
  Request r;
  r.h = h;
  r.d_out = out;
  r.chunk = N;
  r.n_chunks = 1;
  r.engine = true;
  if (!st) st = awgk::engine_setup(h, AWG_STATIC_GEMM_FP16, s->streams[0], &r.split);
  double best = 1e30;
  for (int rep = 0; rep < 4 && !st; ++rep) {
    awg_seek(h, 0);
    Round rd;
    rd.set = 0;
    rd.pieces.push_back({&r, 0, 0, N, true});
    float ms = 0.f;
    if (!issue_round(s, &rd) || cudaEventSynchronize(s->ev_end[0]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, s->ev_beg[0], s->ev_end[0]) != cudaSuccess) {
      st = awgk::set_error(AWG_ECUDA, "engine calibration round failed");
      break;
    }
    if (rep > 0) best = std::min(best, 1e-3 * (double)ms);
  }
  if (out) cudaFree(out);
  if (h) awg_destroy(h);
  if (st) return st;
  s->P_engine = (double)K * (double)N / std::max(1e-6, best - s->a_gpu);
  return AWG_OK;
}

// Cost model calibration, through the same path as the served rounds (best of three each): a round
// of one tile of one tone (fixed cost a_gpu), of 2048 static tones over 2^19 samples (rate P), and
// of one tile of 96 x MAX_SPLIT tones (one CTA of 96 tones per SM: the rate of a CTA alone).
int calibrate(awg_server_t* s) {
  const int32_t K = 2048;
  const int64_t N = (int64_t)1 << 19;
  std::vector<double> f(K), a(K, 1.0 / K), th(K, 0.0);
  for (int32_t k = 0; k < K; ++k) f[k] = s->fs * (0.01 + 0.4 * (double)k / K);
  awg_t* h = awg_create(s->fs);
  int16_t* out = nullptr;
  int st = h ? AWG_OK : AWG_ECUDA;
  if (!st && cudaMalloc((void**)&out, (size_t)N * sizeof(int16_t)) != cudaSuccess)
    st = awgk::set_error(AWG_ENOMEM, "calibration buffer");
  double best[3] = {1e30, 1e30, 1e30};
  for (int pass = 0; pass < 3 && !st; ++pass) {
    const int32_t k = pass == 0 ? 1 : pass == 1 ? K : 96 * awgk::MAX_SPLIT;   // pass 2: one CTA per SM
    const int64_t n = pass == 1 ? N : awgk::TILE;
    if ((st = awg_set_tones(h, f.data(), a.data(), th.data(), k))) break;
    Request r;
    r.h = h;
    r.d_out = out;
    r.chunk = n;
    r.n_chunks = 1;
    r.split = awg_tone_split(h);
    for (int rep = 0; rep < 4 && !st; ++rep) {
      awg_seek(h, 0);
      Round rd;
      rd.set = 0;
      rd.pieces.push_back({&r, 0, 0, n, true});
      float ms = 0.f;
      if (!issue_round(s, &rd) || cudaEventSynchronize(s->ev_end[0]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, s->ev_beg[0], s->ev_end[0]) != cudaSuccess) {
        st = awgk::set_error(AWG_ECUDA, "calibration round failed");
        break;
      }
      if (rep > 0) best[pass] = std::min(best[pass], 1e-3 * (double)ms);   // the first is a warm-up
    }
  }
  if (out) cudaFree(out);
  if (h) awg_destroy(h);
  if (st) return st;
  s->a_gpu = std::max(2e-6, best[0]);
  s->P = s->P_cal = (double)K * (double)N / std::max(1e-6, best[1] - s->a_gpu);
  s->r_cta = 96.0 * awgk::TILE / std::max(1e-6, best[2] - s->a_gpu);
  return calibrate_engine(s, K, N);
}

// Scheduler: up to NSETS rounds in flight on their own streams; the host plans the next round
// while earlier ones run, and rounds overlap on the device when one alone does not fill it.
void sched_main(awg_server_t* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    const int64_t ep = s->epoch.load();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      admit(s);
    }
    while (!s->flight.empty() && cudaEventQuery(s->ev_end[s->flight.front().set]) == cudaSuccess) complete_round(s);

    double next_release = 1e30;
    if ((int)s->flight.size() < NSETS) {
      const double t_plan = now_s(s);
      Round rd;
      rd.set = (int)(s->round_seq % NSETS);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        plan_round(s, t_plan, &rd, &next_release);
        s->queued_work += rd.work;
      }
      if (!rd.pieces.empty()) {
        if (!issue_round(s, &rd)) {
          fail_rounds(s, "round failed");
          break;
        }
        const double t_issued = now_s(s);
        rd.host_s = t_issued - t_plan;
        rd.rec.t_plan = t_plan;
        rd.rec.t_issued = t_issued;
        s->flight.push_back(std::move(rd));
        ++s->round_seq;
        continue;
      }
    }
    // Nothing to issue now: wait for the oldest round, the next release or new work.
    if (!s->flight.empty()) {
      const cudaEvent_t ev = s->ev_end[s->flight.front().set];
      while (!s->stop.load()) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) {
          fail_rounds(s, "round failed");
          break;
        }
        if ((int)s->flight.size() < NSETS && (now_s(s) >= next_release || s->epoch.load() != ep)) break;
        std::this_thread::yield();
      }
      continue;
    }
    const double wait = next_release - now_s(s);
    if (wait > 1e-3) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::duration<double>(std::min(0.05, wait - 0.5e-3)),
                     [&] { return s->stop.load() || s->epoch.load() != ep; });
    } else {
      while (!s->stop.load() && now_s(s) < next_release && s->epoch.load() == ep) std::this_thread::yield();
    }
  }
  for (int i = 0; i < NSETS; ++i)
    if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
}

}  // namespace

extern "C" {

awg_server_t* awg_server_create(double sample_rate_hz, int64_t mem_budget_bytes, int32_t max_active,
                                double max_queue_ms) {
  if (!(sample_rate_hz > 0) || mem_budget_bytes <= 0 || max_active < 1 || !(max_queue_ms >= 0)) {
    awgk::set_error(AWG_EINVAL, "server needs fs > 0, a memory budget, max_active >= 1 and max_queue_ms >= 0");
    return nullptr;
  }
  awg_server_t* s = new awg_server();
  s->fs = sample_rate_hz;
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->max_queue_s = 1e-3 * max_queue_ms;
  s->t0 = clk::now();
  cudaError_t e = cudaGetDevice(&s->device);
  for (int i = 0; i < NSETS && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_beg[i]);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_end[i]);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_ref);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->setup_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = awgk::render_setup_attributes();
  // reference point between the device's event clock and the server clock
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_ref, s->streams[0]);
  if (e == cudaSuccess) e = cudaEventSynchronize(s->ev_ref);
  s->t_ref = now_s(s);
  if (e != cudaSuccess) {
    awgk::set_error(AWG_ECUDA, std::string("server set-up: ") + cudaGetErrorString(e));
    awg_server_destroy(s);
    return nullptr;
  }
  // staging sized for typical rounds up front, so that the first rounds do not allocate
  for (int i = 0; i < NSETS && e == cudaSuccess; ++i) {
    if (!grow(&s->d_reqs[i], &s->h_reqs[i], &s->cap_reqs[i], 1024) ||
        !grow(&s->d_items[i], &s->h_items[i], &s->cap_items[i], 1 << 16) ||
        cudaMalloc((void**)&s->d_arena[i], (1u << 16) * sizeof(awgk::TileRec)) != cudaSuccess ||
        cudaMalloc((void**)&s->d_act[i], (1u << 16) * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&s->d_part[i], (size_t)PART_TILES * awgk::TILE * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&s->d_tctr[i], (1u << 16) * sizeof(unsigned long long)) != cudaSuccess) {
      e = cudaErrorMemoryAllocation;
      break;
    }
    s->cap_arena[i] = s->cap_act[i] = s->cap_tctr[i] = 1u << 16;
    s->cap_part[i] = (size_t)PART_TILES * awgk::TILE;
  }
  if (e != cudaSuccess) awgk::set_error(AWG_ENOMEM, "staging buffers");
  if (e != cudaSuccess || calibrate(s) != AWG_OK) {
    const std::string why = awg_last_error();
    awg_server_destroy(s);
    awgk::set_error(AWG_ECUDA, "server calibration: " + why);
    return nullptr;
  }
  s->sched = std::thread(sched_main, s);
  s->worker = std::thread(worker_main, s);
  return s;
}

int awg_server_set_static_engine(awg_server_t* s, int32_t engine, int32_t min_tones) {
  if (!s) return awgk::set_error(AWG_EINVAL, "null server");
  if (engine != AWG_STATIC_DIRECT && engine != AWG_STATIC_GEMM_FP16 && engine != AWG_STATIC_GEMM_BF16)
    return awgk::set_error(AWG_EINVAL, "unknown static engine");
  if (min_tones < 1) return awgk::set_error(AWG_EINVAL, "min_tones must be >= 1");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->all.empty()) return awgk::set_error(AWG_ESTATE, "the static engine is set before the first request");
  s->engine = engine;
  s->engine_min_tones = min_tones;
  return AWG_OK;
}

int awg_server_set_prefetch(awg_server_t* s, int32_t chunks) {
  if (!s) return awgk::set_error(AWG_EINVAL, "null server");
  if (chunks < 1 || chunks > 16) return awgk::set_error(AWG_EINVAL, "prefetch depth must be 1 .. 16 chunks");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->all.empty()) return awgk::set_error(AWG_ESTATE, "prefetch depth is set before the first request");
  s->depth = chunks;
  return AWG_OK;
}

void awg_server_destroy(awg_server_t* s) {
  if (!s) return;
  s->stop.store(true);
  bump(s);
  if (s->sched.joinable()) s->sched.join();
  if (s->worker.joinable()) s->worker.join();
  for (int i = 0; i < NSETS; ++i)
    if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
  for (auto& kv : s->all) {
    destroy_handle(kv.second);
    if (kv.second->d_out) cudaFree(kv.second->d_out);
    delete kv.second;
  }
  for (awg_t* h : s->idle_handles) awg_destroy(h);
  for (auto& kv : s->idle_out)
    for (int16_t* p : kv.second) cudaFree(p);
  for (int i = 0; i < NSETS; ++i) {
    cudaFree(s->d_arena[i]);
    cudaFree(s->d_act[i]);
    cudaFree(s->d_part[i]);
    cudaFree(s->d_tctr[i]);
    cudaFree(s->d_reqs[i]);
    cudaFree(s->d_items[i]);
    cudaFree(s->d_base[i]);
    cudaFree(s->d_list[i]);
    cudaFreeHost(s->h_list[i]);
    cudaFreeHost(s->h_reqs[i]);
    cudaFreeHost(s->h_items[i]);
    if (s->ev_beg[i]) cudaEventDestroy(s->ev_beg[i]);
    if (s->ev_end[i]) cudaEventDestroy(s->ev_end[i]);
  }
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  if (s->setup_stream) cudaStreamDestroy(s->setup_stream);
  for (int i = 0; i < NSETS; ++i)
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
  delete s;
}

int64_t awg_server_submit(awg_server_t* s, const awg_request_t* q) {
  if (!s || !q) return awgk::set_error(AWG_EINVAL, "null server or request");
  if (q->n_tones < 0 || q->n_chirps < 0 || q->chunk < 1 || q->n_chunks < 1 || q->chunk > ((int64_t)1 << 26))
    return awgk::set_error(AWG_EINVAL, "bad request sizes");
  if ((q->n_tones > 0 && (!q->freq_hz || !q->amp || !q->phase_rad)) ||
      (q->n_chirps > 0 && (!q->chirp_tone || !q->chirp_f_start_hz || !q->chirp_f_end_hz || !q->chirp_duration_s ||
                           !q->chirp_profile || !q->chirp_start_sample)))
    return awgk::set_error(AWG_EINVAL, "null request array");
  Request* r = new Request();
  r->f.assign(q->freq_hz, q->freq_hz + q->n_tones);
  r->a.assign(q->amp, q->amp + q->n_tones);
  r->th.assign(q->phase_rad, q->phase_rad + q->n_tones);
  r->c_tone.assign(q->chirp_tone, q->chirp_tone + q->n_chirps);
  r->c_f0.assign(q->chirp_f_start_hz, q->chirp_f_start_hz + q->n_chirps);
  r->c_f1.assign(q->chirp_f_end_hz, q->chirp_f_end_hz + q->n_chirps);
  r->c_dur.assign(q->chirp_duration_s, q->chirp_duration_s + q->n_chirps);
  r->c_prof.assign(q->chirp_profile, q->chirp_profile + q->n_chirps);
  r->c_start.assign(q->chirp_start_sample, q->chirp_start_sample + q->n_chirps);
  r->chunk = q->chunk;
  r->n_chunks = q->n_chunks;
  r->full_scale = q->full_scale;
  r->period = (double)q->chunk / s->fs;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->engine = s->engine != AWG_STATIC_DIRECT && q->n_tones > 0 && q->n_tones >= s->engine_min_tones;
    set_cost(s, r);
    r->id = s->next_id++;
    r->t_arrival = now_s(s);
    s->all[r->id] = r;
    s->pending.push_back(r);
    ++s->submitted;
  }
  bump(s);
  return r->id;
}

int awg_server_poll(awg_server_t* s, int64_t id, int32_t* state, int32_t* chunks_done) {
  if (!s) return awgk::set_error(AWG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return awgk::set_error(AWG_EINVAL, "unknown request id");
  if (state) *state = it->second->state;
  if (chunks_done) *chunks_done = it->second->done_chunks;
  return AWG_OK;
}

int awg_server_read(awg_server_t* s, int64_t id, int16_t* host_out, int64_t n_samples) {
  if (!s || !host_out) return awgk::set_error(AWG_EINVAL, "null argument");
  int16_t* src = nullptr;
  int64_t total = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return awgk::set_error(AWG_EINVAL, "unknown request id");
    Request* r = it->second;
    if (r->state != AWG_REQ_DONE) return awgk::set_error(AWG_ESTATE, "request not done");
    src = r->d_out;
    total = (int64_t)r->n_chunks * r->chunk;
  }
  if (n_samples < 0 || n_samples > total) return awgk::set_error(AWG_EINVAL, "sample count out of range");
  cudaError_t e = cudaMemcpy(host_out, src, (size_t)n_samples * sizeof(int16_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return awgk::set_error(AWG_ECUDA, std::string("read: ") + cudaGetErrorString(e));
  return AWG_OK;
}

int awg_server_release(awg_server_t* s, int64_t id) {
  if (!s) return awgk::set_error(AWG_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return awgk::set_error(AWG_EINVAL, "unknown request id");
    it->second->release_requested = true;
  }
  bump(s);
  return AWG_OK;
}

int awg_server_drain(awg_server_t* s, int32_t timeout_ms) {
  if (!s) return awgk::set_error(AWG_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] {
    if (s->stop.load()) return true;
    if (!s->pending.empty() || !s->active.empty()) return false;
    return true;
  });
  if (!s->error.empty()) return awgk::set_error(AWG_ECUDA, s->error);
  return ok ? AWG_OK : awgk::set_error(AWG_ETIMEOUT, "requests still in flight");
}

int awg_server_stats(awg_server_t* s, awg_server_stats_t* out) {
  if (!s || !out) return awgk::set_error(AWG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->rejected_deadline = s->rej_deadline;
  out->rejected_memory = s->rej_memory;
  out->completed = s->completed;
  out->chunks = s->chunks;
  out->deadline_misses = s->misses;
  out->latency_p50_ms = 1e3 * percentile(s->lat, 0.50);
  out->latency_p99_ms = 1e3 * percentile(s->lat, 0.99);
  out->latency_max_ms = s->lat.empty() ? 0 : 1e3 * *std::max_element(s->lat.begin(), s->lat.end());
  out->latency_p99_of_period = percentile(s->lat_frac, 0.99);
  out->first_chunk_p50_ms = 1e3 * percentile(s->ttfc, 0.50);
  out->first_chunk_p99_ms = 1e3 * percentile(s->ttfc, 0.99);
  out->rounds = s->rounds;
  out->mean_batch = s->rounds ? (double)s->batched / (double)s->rounds : 0.0;
  out->max_batch = s->max_batch;
  const double span = s->first_t >= 0 ? std::max(1e-9, s->last_t - s->first_t) : 1e-9;
  out->tone_samples_per_s = s->tone_samples / span;
  out->samples_per_s = s->samples / span;
  out->busy_fraction = s->busy_s / span;
  out->est_throughput = s->P;
  out->est_round_cost_ms = 1e3 * s->a_gpu;
  out->est_cta_rate = s->r_cta;
  out->est_engine_throughput = s->P_engine;
  return AWG_OK;
}

int32_t awg_server_trace_rounds(awg_server_t* s, awg_round_record_t* out, int32_t cap) {
  if (!s || (cap > 0 && !out)) return awgk::set_error(AWG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  return s->trace_rounds.copy(out, cap);
}

int32_t awg_server_trace_chunks(awg_server_t* s, awg_chunk_record_t* out, int32_t cap) {
  if (!s || (cap > 0 && !out)) return awgk::set_error(AWG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  return s->trace_chunks.copy(out, cap);
}

}  // extern "C"
