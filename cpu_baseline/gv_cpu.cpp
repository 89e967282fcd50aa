// gv_cpu.cpp -- the CPU baseline of the benchmark: the library's binary64 closed-form
// solid code (solid_fp64.cuh, descriptors from desc_build.h) compiled for the host and
// run one track per loop iteration, OpenMP over tracks.  It is the fair CPU counterpart
// of the GPU's plain binary64 pass (same algorithm, same bits), timed beside the GPU and
// checked against the oracle by the tests.  Measurement infrastructure only: the
// geometry library never calls it.
#include <cuda_runtime.h>  // the host stand-ins (shim/): qualifiers and intrinsics
#include <cstdint>
#include <cstring>
#include "desc_build.h"
#include "solid_fp64.cuh"

using namespace gv;

extern "C" {

int gvcpu_desc_size(void) { return (int)sizeof(Desc); }

// Build a descriptor into `out` (gvcpu_desc_size() bytes).  kind: 0 box (p: dx dy dz),
// 1 trd (dx1 dx2 dy1 dy2 dz), 2 trap (11 parameters), 3 tube (rmin rmax dz sphi dphi),
// 4 cone (rmin1 rmax1 rmin2 rmax2 dz sphi dphi), 5 polycone (nz, then z[nz], rmin[nz],
// rmax[nz], sphi, dphi).  Returns the gv_status of the construction.
int gvcpu_build(int kind, const double* p, void* out) {
  Desc h;
  Built b = built_err(GV_ERR_INVALID_ARG, "unknown kind");
  switch (kind) {
    case 0: b = build_box(p[0], p[1], p[2], h); break;
    case 1: {
      const double q[11] = {p[4], 0, 0, p[2], p[0], p[0], 0, p[3], p[1], p[1], 0};
      b = build_trap(q, kTrd, h);
      break;
    }
    case 2: b = build_trap(p, kTrap, h); break;
    case 3: b = build_tube(p[0], p[1], p[2], p[3], p[4], h); break;
    case 4: b = build_cone(p[0], p[1], p[2], p[3], p[4], p[5], p[6], h); break;
    case 5: {
      const int nz = (int)p[0];
      b = build_pcon(kPcon, nz, p + 1, p + 1 + nz, p + 1 + 2 * nz, p[1 + 3 * nz], p[2 + 3 * nz], h);
      break;
    }
  }
  if (b.st == GV_OK) std::memcpy(out, &h, sizeof(Desc));
  return (int)b.st;
}

// All five queries for n tracks (any output may be NULL); nthreads OpenMP threads.
void gvcpu_query(const void* desc, int64_t n, const double* x, const double* y, const double* z,
                 const double* u, const double* v, const double* w, int8_t* inside, double* din,
                 double* dout, double* sin, double* sout, int nthreads) {
  Desc S;
  std::memcpy(&S, desc, sizeof(Desc));
  const unsigned want = (inside ? f64::kWantCode : 0u) | (din ? f64::kWantDin : 0u) |
                        (dout ? f64::kWantDout : 0u) | (sin ? f64::kWantSin : 0u) |
                        (sout ? f64::kWantSout : 0u);
  const bool dirs = din || dout;
#pragma omp parallel for schedule(static, 4096) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t i = 0; i < n; i++) {
    f64::Track T{x[i], y[i], z[i], dirs ? u[i] : 0.0, dirs ? v[i] : 0.0, dirs ? w[i] : 0.0};
    f64::Result R;
    f64::query(S, T, want, R);
    if (inside) inside[i] = (int8_t)R.code;
    if (din) din[i] = R.din;
    if (dout) dout[i] = R.dout;
    if (sin) sin[i] = R.sin;
    if (sout) sout[i] = R.sout;
  }
}

}  // extern "C"
