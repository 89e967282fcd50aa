// query_static.cu -- gv_query_fp32_static: the FP32 + refinement query pass with
// its scratch (refinement worklist and counter) in a fixed device array that
// the library owns for the life of the process, so that the call itself never
// allocates device memory.
//
// Who needs it: callers that must not call cudaMalloc on their hot path -- a
// host framework that owns every byte of device memory through its own pool,
// a real-time or serving loop that cannot afford cudaMalloc's implicit device
// synchronisation, or a plug-in that has no allocator to call.  Such callers
// cannot create a gv_workspace (which allocates); this entry point takes the
// place of one.
//
// Limits and sharing rules (also stated in gv.h):
//  - at most kStaticMaxTracks tracks per call (larger baskets are rejected
//    with GV_ERR_INVALID_ARG before anything is enqueued);
//  - the array is a static __device__ object: every GPU that loads the library
//    holds it (4 MiB + 256 B) until the process exits;
//  - all calls share the one array; the counter is cleared (cudaMemsetAsync on
//    the caller's stream) at the start of every call and the worklist keeps
//    whatever the last call left in it.  Calls that overlap on the GPU (on
//    different streams, or from different threads) race on the array and give
//    wrong results: serialise them;
//  - the first call on a device with a non-empty basket resolves the array's
//    device address with cudaGetSymbolAddress (host code cannot use the symbol
//    itself: in host code its name stands for a host-side shadow, not a device
//    address) and keeps it for that device.  Make that first call before any
//    stream capture.  The kept address belongs to the device's primary context as
//    it was when first resolved: it does not survive cudaDeviceReset, and a caller
//    running in another (driver-API) context must not use this entry point.
#include <mutex>
#include "gv_internal.h"

namespace gv {

constexpr int64_t kStaticMaxTracks = int64_t(1) << 20;
constexpr size_t kStaticCounterBytes = 256;  // counter, padded to keep the worklist aligned

static __device__ __align__(256) unsigned char g_static_scratch[kStaticCounterBytes + sizeof(uint32_t) * kStaticMaxTracks];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device (resolved once per device).
static gv_status static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "gv_query_fp32_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(GV_ERR_UNSUPPORTED, "gv_query_fp32_static: device index beyond 63");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "gv_query_fp32_static: cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return GV_OK;
}

}  // namespace gv

using namespace gv;

extern "C" gv_status gv_query_fp32_static(const gv_solid* s, const gv_tracks* t, const gv_results* res,
                                          void* stream) {
  const gv::Range range("gv_query_fp32_static");
  if (!s || !t || !res) return set_error(GV_ERR_INVALID_ARG, "gv_query_fp32_static: NULL solid, tracks or results");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "gv_query_fp32_static: negative track count");
  if (t->n > kStaticMaxTracks)
    return set_error(GV_ERR_INVALID_ARG,
                     "gv_query_fp32_static: basket larger than the fixed scratch (at most 1048576 tracks per call)");
  QueryArgs a{t->x, t->y, t->z, t->dx, t->dy, t->dz, res->inside, res->dist_in, res->dist_out,
              res->safety_in, res->safety_out, t->n};
  if (t->n > 0) {
    if (!a.x || !a.y || !a.z) return set_error(GV_ERR_INVALID_ARG, "gv_query_fp32_static: NULL point array");
    if ((a.din || a.dout) && (!a.u || !a.v || !a.w))
      return set_error(GV_ERR_INVALID_ARG, "gv_query_fp32_static: distances requested without directions");
    const void* ptrs[10] = {a.x, a.y, a.z, a.u, a.v, a.w, a.din, a.dout, a.sin, a.sout};
    for (int i = 0; i < 10; i++)
      if (ptrs[i] && ((uintptr_t)ptrs[i] & 7u))
        return set_error(GV_ERR_INVALID_ARG, "gv_query_fp32_static: arrays must be 8-byte aligned");
  }
  if (t->n == 0) return GV_OK;  // nothing to do: nothing enqueued, no address looked up
  void* base = nullptr;
  gv_status st = static_scratch(&base);
  if (st != GV_OK) return st;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
  uint32_t* worklist = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + kStaticCounterBytes);
  // launch_query_fp32 clears the counter on the stream before the bulk pass
  const cudaError_t e = launch_query_fp32(s, a, worklist, counter, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "gv_query_fp32_static launch");
  return GV_OK;
}
