// Streaming ring (C ABI in include/awg.h): chunk slots in pinned, device-mapped host memory that
// the render kernel writes directly, and a sink thread that plays them at the sample rate -- the
// host-side stand-in for the DAC card's FIFO of the Streaming pathway (Sec. IV-B).  A chunk that is
// not complete when its play time comes is an underrun.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/awg.h"
#include "awg_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Slot {
  int64_t chunk = -1;            // chunk index held, -1 if free
  cudaEvent_t done = nullptr;    // recorded after the chunk's render
  double t_submit_ms = 0;        // host time of the push (ms since ring creation)
};

}  // namespace

struct awg_ring {
  awg_t* h = nullptr;
  int64_t chunk = 0;
  int32_t n_slots = 0;
  double fs = 0;
  int16_t* host = nullptr;       // n_slots * chunk samples, pinned + mapped
  std::vector<Slot> slots;
  cudaEvent_t ref = nullptr;     // timing reference recorded at creation
  double ref_host_ms = 0;        // host time at which `ref` completed
  clk::time_point t_origin;
  // producer / sink shared state
  std::mutex mu;
  std::condition_variable cv;
  int64_t pushed = 0;            // chunks handed to the GPU
  int64_t played = 0;            // chunks consumed by the sink
  std::thread sink;
  std::atomic<bool> stop{false};
  bool sink_running = false;
  int32_t prefill = 1;
  int64_t target = -1;           // stop after this many chunks (-1: until stopped)
  // stats
  int64_t underruns = 0;
  int64_t sink_error = 0;
  std::vector<double> latency_ms;  // GPU completion - push, per played chunk
  std::vector<double> lead_ms;     // play time - GPU completion, per played chunk
  uint64_t checksum = 0;
  int16_t* capture = nullptr;
  int64_t capture_cap = 0;
};

namespace {

double now_ms(const awg_ring_t* r) {
  return std::chrono::duration<double, std::milli>(clk::now() - r->t_origin).count();
}

int ring_fail(int code, const std::string& msg) { return awgk::set_error(code, msg); }

// Host time (ring clock) at which the GPU completed `ev`, via the reference event.
double gpu_done_ms(awg_ring_t* r, cudaEvent_t ev) {
  float el = 0.f;
  if (cudaEventElapsedTime(&el, r->ref, ev) != cudaSuccess) return now_ms(r);
  return r->ref_host_ms + el;
}

// Poll an event until it completes or `limit_ms` passes.
bool wait_event(cudaEvent_t ev, double limit_ms) {
  const auto t0 = clk::now();
  while (true) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return true;
    if (e != cudaErrorNotReady) return false;
    if (std::chrono::duration<double, std::milli>(clk::now() - t0).count() > limit_ms) return false;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void sink_main(awg_ring_t* r) {
  const double period_ms = 1e3 * (double)r->chunk / r->fs;
  // wait for the prefill chunks to be complete, then start the play clock
  for (int64_t c = 0; c < r->prefill; ++c) {
    Slot* s = nullptr;
    {
      std::unique_lock<std::mutex> lk(r->mu);
      if (!r->cv.wait_for(lk, std::chrono::seconds(10), [&] { return r->stop.load() || r->pushed > c; })) {
        r->sink_error = AWG_ETIMEOUT;
        return;
      }
      if (r->stop.load()) return;
      s = &r->slots[(size_t)(c % r->n_slots)];
    }
    if (!wait_event(s->done, 10000.0)) {
      r->sink_error = AWG_ETIMEOUT;
      return;
    }
  }
  const double t_start = now_ms(r);
  for (int64_t c = 0; r->target < 0 || c < r->target; ++c) {
    const double deadline = t_start + (double)c * period_ms;
    // sleep until the play time of chunk c (coarse sleep, then a short spin)
    while (true) {
      if (r->stop.load()) return;
      const double left = deadline - now_ms(r);
      if (left <= 0) break;
      if (left > 0.3) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((left - 0.2) * 1000)));
      else std::this_thread::yield();
    }
    Slot* s = nullptr;
    bool queued;
    {
      std::lock_guard<std::mutex> lk(r->mu);
      queued = r->pushed > c;
      s = &r->slots[(size_t)(c % r->n_slots)];
    }
    bool late = !queued || cudaEventQuery(s->done) != cudaSuccess;
    if (late) {
      ++r->underruns;
      // the DAC would have played stale data; wait (bounded) for the chunk, then go on
      {
        std::unique_lock<std::mutex> lk(r->mu);
        if (!r->cv.wait_for(lk, std::chrono::seconds(10), [&] { return r->stop.load() || r->pushed > c; })) {
          r->sink_error = AWG_ETIMEOUT;
          return;
        }
        if (r->stop.load()) return;
      }
      if (!wait_event(s->done, 10000.0)) {
        r->sink_error = AWG_ETIMEOUT;
        return;
      }
    }
    const double done = gpu_done_ms(r, s->done);
    r->latency_ms.push_back(done - s->t_submit_ms);
    r->lead_ms.push_back(deadline - done);
    // play: read every sample of the slot (as the DMA to the card would), optionally capture
    const int16_t* src = r->host + (size_t)(c % r->n_slots) * (size_t)r->chunk;
    uint64_t acc = r->checksum;
    for (int64_t i = 0; i < r->chunk; ++i) acc = acc * 1099511628211ull + (uint16_t)src[i];
    r->checksum = acc;
    if (r->capture && (c + 1) * r->chunk <= r->capture_cap)
      std::memcpy(r->capture + c * r->chunk, src, (size_t)r->chunk * sizeof(int16_t));
    {
      std::lock_guard<std::mutex> lk(r->mu);
      s->chunk = -1;
      r->played = c + 1;
    }
    r->cv.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

awg_ring_t* awg_ring_create(awg_t* h, int64_t chunk, int32_t n_slots) {
  if (!h || chunk < 1 || n_slots < 2 || chunk > (int64_t)1 << 30 || n_slots > 1024) {
    ring_fail(AWG_EINVAL, "ring needs a handle, chunk >= 1 and 2..1024 slots");
    return nullptr;
  }
  awg_ring_t* r = new awg_ring();
  r->h = h;
  r->chunk = chunk;
  r->n_slots = n_slots;
  r->fs = awg_sample_rate(h);
  r->t_origin = clk::now();
  r->slots.resize((size_t)n_slots);
  cudaError_t e = cudaHostAlloc((void**)&r->host, (size_t)n_slots * (size_t)chunk * sizeof(int16_t),
                                cudaHostAllocMapped | cudaHostAllocPortable);
  for (int32_t i = 0; e == cudaSuccess && i < n_slots; ++i) e = cudaEventCreate(&r->slots[(size_t)i].done);
  if (e == cudaSuccess) e = cudaEventCreate(&r->ref);
  if (e == cudaSuccess) e = cudaEventRecord(r->ref, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(r->ref);
  if (e != cudaSuccess) {
    ring_fail(AWG_ECUDA, std::string("ring set-up: ") + cudaGetErrorString(e));
    awg_ring_destroy(r);
    return nullptr;
  }
  r->ref_host_ms = now_ms(r);
  return r;
}

void awg_ring_destroy(awg_ring_t* r) {
  if (!r) return;
  r->stop.store(true);
  r->cv.notify_all();
  if (r->sink.joinable()) r->sink.join();
  for (Slot& s : r->slots) {
    if (s.done) {
      cudaEventSynchronize(s.done);
      cudaEventDestroy(s.done);
    }
  }
  if (r->ref) cudaEventDestroy(r->ref);
  if (r->host) cudaFreeHost(r->host);
  delete r;
}

int awg_ring_push(awg_ring_t* r, void* stream, int32_t timeout_ms) {
  if (!r) return ring_fail(AWG_EINVAL, "null ring");
  const int64_t c = r->pushed;
  Slot& s = r->slots[(size_t)(c % r->n_slots)];
  {
    std::unique_lock<std::mutex> lk(r->mu);
    // the slot is free once the sink has played the chunk n_slots back
    if (!r->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                        [&] { return r->played > c - r->n_slots; }))
      return ring_fail(AWG_ETIMEOUT, "ring full: the sink did not free a slot in time");
  }
  int16_t* dst = r->host + (size_t)(c % r->n_slots) * (size_t)r->chunk;
  s.t_submit_ms = now_ms(r);
  int st = awg_render(r->h, r->chunk, dst, stream);
  if (st) return ring_fail(st, std::string("render: ") + awg_last_error());
  cudaError_t e = cudaEventRecord(s.done, (cudaStream_t)stream);
  if (e != cudaSuccess) return ring_fail(AWG_ECUDA, std::string("event: ") + cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lk(r->mu);
    s.chunk = c;
    r->pushed = c + 1;
  }
  r->cv.notify_all();
  return AWG_OK;
}

int awg_ring_start(awg_ring_t* r, int32_t prefill, int64_t n_chunks, int16_t* capture, int64_t capture_samples) {
  if (!r) return ring_fail(AWG_EINVAL, "null ring");
  if (r->sink_running) return ring_fail(AWG_ESTATE, "sink already running");
  if (prefill < 1 || prefill > r->n_slots) return ring_fail(AWG_EINVAL, "prefill must be 1..n_slots");
  r->prefill = prefill;
  r->target = n_chunks;
  r->capture = capture;
  r->capture_cap = capture ? capture_samples : 0;
  r->stop.store(false);
  r->sink_running = true;
  r->sink = std::thread(sink_main, r);
  return AWG_OK;
}

int awg_ring_finish(awg_ring_t* r, int32_t timeout_ms, awg_ring_stats_t* out) {
  if (!r) return ring_fail(AWG_EINVAL, "null ring");
  if (!r->sink_running) return ring_fail(AWG_ESTATE, "sink not running");
  int rc = AWG_OK;
  {
    std::unique_lock<std::mutex> lk(r->mu);
    if (r->target >= 0 &&
        !r->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return r->played >= r->target; }))
      rc = ring_fail(AWG_ETIMEOUT, "sink did not play all chunks in time");
  }
  r->stop.store(true);
  r->cv.notify_all();
  r->sink.join();
  r->sink_running = false;
  if (rc == AWG_OK && r->sink_error) rc = ring_fail((int)r->sink_error, "sink gave up waiting for a chunk");
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->played = r->played;
    out->underruns = r->underruns;
    out->latency_p50_ms = percentile(r->latency_ms, 0.50);
    out->latency_p99_ms = percentile(r->latency_ms, 0.99);
    out->latency_max_ms = r->latency_ms.empty() ? 0 : *std::max_element(r->latency_ms.begin(), r->latency_ms.end());
    out->lead_min_ms = r->lead_ms.empty() ? 0 : *std::min_element(r->lead_ms.begin(), r->lead_ms.end());
    out->lead_p50_ms = percentile(r->lead_ms, 0.50);
    out->chunk_playback_ms = 1e3 * (double)r->chunk / r->fs;
    out->checksum = r->checksum;
  }
  return rc;
}

const int16_t* awg_ring_slot(const awg_ring_t* r, int32_t i) {
  if (!r || i < 0 || i >= r->n_slots) return nullptr;
  return r->host + (size_t)i * (size_t)r->chunk;
}

}  // extern "C"
