// gv_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include "gv.h"
#include "gv_desc.h"

struct gv_solid {
  gv::Desc h;          // host copy
  gv::Desc* d;         // device copy (on `device`)
  int device;
};

struct gv_workspace {
  uint32_t* idx;                 // refinement worklist, `cap` entries
  unsigned long long* counter;   // worklist length (device)
  int64_t cap;
  int device;
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
gv_status cuda_error(cudaError_t e, const char* where);
int sm_count();

// Launchers (async on `stream`); return cudaGetLastError() of the launch.
cudaError_t launch_query_fp64(const gv_solid* s, const QueryArgs& a, cudaStream_t stream);
cudaError_t launch_query_fp32(const gv_solid* s, const QueryArgs& a, uint32_t* worklist,
                              unsigned long long* counter, cudaStream_t stream);

}  // namespace gv
