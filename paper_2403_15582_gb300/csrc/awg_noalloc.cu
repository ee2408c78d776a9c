// Fixed scratch for the allocation-free render (awg_render_noalloc).
//
// The chirp tile records and the slot -> record map that a render needs live here, in static
// device arrays compiled into the library, instead of in memory the handle allocates on demand.
// Every GPU that loads the library holds these arrays until the process exits.  In host code the
// array names are host-side stand-ins, not device addresses: the device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "awg_internal.h"

namespace awgk {

namespace {

static __device__ __align__(256) TileRec g_noalloc_recs[NOALLOC_MAX_RECORDS];
static __device__ __align__(256) int32_t g_noalloc_act[NOALLOC_MAX_SLOTS];

constexpr int MAX_DEVICES = 64;
struct DeviceScratch {
  TileRec* recs;
  int32_t* act;
  bool ready;
};
DeviceScratch g_scratch[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

}  // namespace

cudaError_t noalloc_scratch(int device, TileRec** recs, int32_t** act) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  DeviceScratch& s = g_scratch[device];
  if (!s.ready) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    if (cur != device) return cudaErrorInvalidDevice;
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_recs);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_noalloc_act);
    if (e != cudaSuccess) return e;
    s.recs = static_cast<TileRec*>(p);
    s.act = static_cast<int32_t*>(q);
    s.ready = true;
  }
  *recs = s.recs;
  *act = s.act;
  return cudaSuccess;
}

}  // namespace awgk
