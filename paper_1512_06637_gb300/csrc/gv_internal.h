// gv_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "gv.h"
#include "gv_desc.h"

struct gv_solid {
  gv::Desc h;          // host copy
  gv::Desc* d;         // device copy (on `device`)
  int device;
  gv::Desc ph[2];      // boolean: host copies of the two components
};

struct gv_workspace {
  uint32_t* idx;                 // refinement worklist, `cap` entries
  unsigned long long* counter;   // worklist length (device)
  int64_t cap;
  int device;
  int fused_blocks;              // last query: blocks of the one-launch small-basket pass (0: none)
};

namespace gv {

// Arguments of one single-solid query pass (device pointers).
struct QueryArgs {
  const double *x, *y, *z, *u, *v, *w;
  int8_t* inside;
  double *din, *dout, *sin, *sout;
  int64_t n;
};

gv_status set_error(gv_status st, const std::string& msg);

// An NVTX range around one call of the C ABI (visible to a profiler's timeline; a no-op
// unless a tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Records of a device table of solids (a batch's or a geometry's): one per solid, then the
// two component records of every boolean, whose parts pointer is set to them, so that the
// table does not depend on the lifetime of the solids' handles.  d_table is the device
// address the table will be copied to; returns the records to copy.
std::vector<Desc> table_records(const gv_solid* const* solids, int n, Desc* d_table);
int table_size(const gv_solid* const* solids, int n);
gv_status cuda_error(cudaError_t e, const char* where);
int sm_count();

#ifdef GV_DEBUG
// The device-check words of the query passes' translation units (gv_debug.cuh).
cudaError_t debug_read_query32(unsigned long long out[2], bool clear);
cudaError_t debug_read_query64(unsigned long long out[2], bool clear);
cudaError_t debug_read_query_small(unsigned long long out[2], bool clear);
#endif

// Launchers (async on `stream`); return cudaGetLastError() of the launch.
cudaError_t launch_query_fp64(const gv_solid* s, const QueryArgs& a, cudaStream_t stream);
// Baskets of at most 65536 tracks of a primitive solid take one launch that evaluates uncertain
// tracks in binary64 on the spot; it writes each block's count of such tracks to worklist[block]
// (not the counter) and reports its number of blocks in *fused_blocks (0: the two-pass path).
cudaError_t launch_query_fp32(const gv_solid* s, const QueryArgs& a, uint32_t* worklist,
                              unsigned long long* counter, cudaStream_t stream, int* fused_blocks = nullptr);
// The one-launch pass when the basket qualifies (returns false and launches nothing otherwise).
bool launch_query_small(const gv_solid* s, const QueryArgs& a, uint32_t* slots, cudaStream_t stream,
                        int* fused_blocks);

}  // namespace gv
