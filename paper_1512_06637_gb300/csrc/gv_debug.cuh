// gv_debug.cuh -- device-side checks of a GV_DEBUG build.
//
// Built with GV_DEBUG defined (build.py with GV_DEBUG=1, producing libgvgeo_debug.so), the query
// passes check their inputs and their own bookkeeping on the device: directions are unit vectors
// (| |d|^2 - 1 | <= 1e-6), a refinement worklist holds no more entries than the basket, and every
// track index it names exists.  A failed check records its code and the smallest offending track
// index in a device word of the translation unit (atomic OR / atomic min) and the pass goes on;
// gv_debug_status reads the words back.  In a release build the checks compile to nothing.
#pragma once
#include <cuda_runtime.h>

namespace gv {

enum : unsigned { kDbgDirection = 1u, kDbgWorklist = 2u, kDbgIndex = 4u };

#ifdef GV_DEBUG
static __device__ unsigned long long g_dbg[2] = {0ull, 0xFFFFFFFFFFFFFFFFull};
__device__ __forceinline__ void dbg_record(unsigned code, long long i) {
  atomicOr(&g_dbg[0], (unsigned long long)code);
  atomicMin(&g_dbg[1], (unsigned long long)(i < 0 ? 0 : i));
}
#define GV_DCHECK(cond, code, i)                                  \
  do {                                                            \
    if (!(cond)) ::gv::dbg_record((code), (long long)(i));        \
  } while (0)
// |d|^2 within 1e-6 of 1
__device__ __forceinline__ bool dbg_unit(double u, double v, double w) {
  return fabs((u * u + v * v + w * w) - 1.0) <= 1e-6;
}
// This translation unit's word (codes, smallest index), cleared afterwards if asked.
static cudaError_t dbg_read(unsigned long long out[2], bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_dbg, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && clear) {
    const unsigned long long z[2] = {0ull, 0xFFFFFFFFFFFFFFFFull};
    e = cudaMemcpyToSymbol(g_dbg, z, sizeof(z));
  }
  return e;
}
#else
#define GV_DCHECK(cond, code, i) \
  do {                           \
  } while (0)
#endif

}  // namespace gv
