// gv_host.cu -- host side of the C ABI: solid constructors (the descriptors built by
// desc_build.h, then uploaded), workspaces, argument checks and launch dispatch.
// This file is compiled with -ffp-contract=off so that every expression rounds
// exactly as written.  Every rule below is stated in gv.h.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include "desc_build.h"
#include "gv_internal.h"

namespace gv {

static thread_local std::string g_last_error;

gv_status set_error(gv_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

gv_status cuda_error(cudaError_t e, const char* where) {
  return set_error(GV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 152;
  return n;
}

static gv_status upload(const Desc& h, gv_solid** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "out handle pointer is NULL");
  gv_solid* s = new (std::nothrow) gv_solid;
  if (!s) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->h = h;
  s->d = nullptr;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d, sizeof(Desc));
  if (e == cudaSuccess) e = cudaMemcpy(s->d, &s->h, sizeof(Desc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (s->d) cudaFree(s->d);
    delete s;
    return e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "cudaMalloc of a solid failed")
                                          : cuda_error(e, "solid upload");
  }
  *out = s;
  return GV_OK;
}

// A built descriptor uploaded as a new handle; a failed construction reports its message.
static gv_status make(const Built& b, const Desc& h, gv_solid** out) {
  if (b.st != GV_OK) return set_error(b.st, b.msg);
  return upload(h, out);
}

}  // namespace gv

using namespace gv;

namespace gv {

int table_size(const gv_solid* const* solids, int n) {
  int m = n;
  for (int i = 0; i < n; i++) if (solids[i]->h.type == kBool) m += 2;
  return m;
}

std::vector<Desc> table_records(const gv_solid* const* solids, int n, Desc* d_table) {
  std::vector<Desc> recs;
  recs.reserve(table_size(solids, n));
  for (int i = 0; i < n; i++) recs.push_back(solids[i]->h);
  for (int i = 0; i < n; i++) {
    if (solids[i]->h.type != kBool) continue;
    recs[i].parts = d_table + recs.size();
    recs.push_back(solids[i]->ph[0]);
    recs.push_back(solids[i]->ph[1]);
  }
  return recs;
}

}  // namespace gv

extern "C" {

gv_status gv_solid_box(double dx, double dy, double dz, gv_solid** out) {
  Desc h;
  const Built b = build_box(dx, dy, dz, h);
  return make(b, h, out);
}

gv_status gv_solid_trap(const double p[11], gv_solid** out) {
  if (!p) return set_error(GV_ERR_INVALID_ARG, "trap: NULL parameter array");
  Desc h;
  const Built b = build_trap(p, kTrap, h);
  return make(b, h, out);
}

gv_status gv_solid_trd(double dx1, double dx2, double dy1, double dy2, double dz, gv_solid** out) {
  const double p[11] = {dz, 0, 0, dy1, dx1, dx1, 0, dy2, dx2, dx2, 0};
  Desc h;
  const Built b = build_trap(p, kTrd, h);
  return make(b, h, out);
}

gv_status gv_solid_tube(double rmin, double rmax, double dz, double sphi, double dphi, gv_solid** out) {
  Desc h;
  const Built b = build_tube(rmin, rmax, dz, sphi, dphi, h);
  return make(b, h, out);
}

gv_status gv_solid_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz, double sphi,
                        double dphi, gv_solid** out) {
  Desc h;
  const Built b = build_cone(rmin1, rmax1, rmin2, rmax2, dz, sphi, dphi, h);
  return make(b, h, out);
}

gv_status gv_solid_polycone(int nz, const double* z, const double* rmin, const double* rmax, double sphi,
                            double dphi, gv_solid** out) {
  Desc h;
  const Built b = build_pcon(kPcon, nz, z, rmin, rmax, sphi, dphi, h);
  return make(b, h, out);
}

gv_status gv_solid_boolean(int32_t op, const gv_solid* a, const gv_solid* c, const double R[9], const double t[3],
                           gv_solid** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "out handle pointer is NULL");
  if (!a || !c || !R || !t) return set_error(GV_ERR_INVALID_ARG, "boolean: NULL component or placement");
  if (op != GV_UNION && op != GV_SUBTRACTION && op != GV_INTERSECTION)
    return set_error(GV_ERR_INVALID_ARG, "boolean: unknown operation");
  if (a->h.type == kBool || c->h.type == kBool)
    return set_error(GV_ERR_UNSUPPORTED, "boolean: components must be primitive solids");
  if (a->device != c->device) return set_error(GV_ERR_INVALID_ARG, "boolean: components on different devices");
  for (int i = 0; i < 9; i++) if (!std::isfinite(R[i])) return set_error(GV_ERR_INVALID_ARG, "boolean: non-finite rotation");
  for (int i = 0; i < 3; i++) if (!std::isfinite(t[i])) return set_error(GV_ERR_INVALID_ARG, "boolean: non-finite shift");
  for (int i = 0; i < 3; i++)  // R must be a rotation: orthonormal rows, determinant +1
    for (int j = 0; j < 3; j++) {
      const double d = R[3 * i] * R[3 * j] + R[3 * i + 1] * R[3 * j + 1] + R[3 * i + 2] * R[3 * j + 2];
      if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-9) return set_error(GV_ERR_INVALID_ARG, "boolean: R is not orthonormal");
    }
  const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                     R[2] * (R[3] * R[7] - R[4] * R[6]);
  if (det < 0) return set_error(GV_ERR_INVALID_ARG, "boolean: R is a reflection");
  gv_solid* s = new (std::nothrow) gv_solid;
  if (!s) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  init_desc(s->h, kBool);
  s->h.bop = op;
  std::memcpy(s->h.bR, R, sizeof(s->h.bR));
  std::memcpy(s->h.bt, t, sizeof(s->h.bt));
  s->h.size = std::fmax(a->h.size, c->h.size);
  for (int i = 0; i < 3; i++) {  // a's box and the box around c's placed box
    const double hc = std::fabs(R[3 * i]) * c->h.ext[0] + std::fabs(R[3 * i + 1]) * c->h.ext[1] +
                      std::fabs(R[3 * i + 2]) * c->h.ext[2];
    s->h.ext[i] = std::fmax(a->h.ext[i], std::fabs(t[i]) + hc);
  }
  s->ph[0] = a->h;
  s->ph[1] = c->h;
  s->d = nullptr;
  s->device = a->device;
  // one allocation: the boolean's record, then copies of the two component records
  cudaError_t e = cudaMalloc(&s->d, 3 * sizeof(Desc));
  if (e == cudaSuccess) {
    s->h.parts = s->d + 1;
    const Desc recs[3] = {s->h, a->h, c->h};
    e = cudaMemcpy(s->d, recs, sizeof(recs), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    if (s->d) cudaFree(s->d);
    delete s;
    return e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "cudaMalloc of a solid failed")
                                          : cuda_error(e, "boolean upload");
  }
  *out = s;
  return GV_OK;
}

void gv_solid_destroy(gv_solid* s) {
  if (!s) return;
  if (s->d) cudaFree(s->d);
  delete s;
}

gv_status gv_workspace_create(int64_t max_tracks, gv_workspace** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "out handle pointer is NULL");
  if (max_tracks < 0 || max_tracks > ((int64_t)1 << 32))
    return set_error(GV_ERR_INVALID_ARG, "workspace size must be in [0, 2^32]");
  gv_workspace* w = new (std::nothrow) gv_workspace;
  if (!w) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  w->idx = nullptr;
  w->counter = nullptr;
  w->cap = max_tracks;
  w->fused_blocks = 0;
  cudaError_t e = cudaGetDevice(&w->device);
  if (e == cudaSuccess) e = cudaMalloc(&w->idx, sizeof(uint32_t) * (size_t)(max_tracks > 0 ? max_tracks : 1));
  if (e == cudaSuccess) e = cudaMalloc(&w->counter, 64);
  if (e == cudaSuccess) e = cudaMemset(w->counter, 0, 64);
  if (e != cudaSuccess) {
    if (w->idx) cudaFree(w->idx);
    if (w->counter) cudaFree(w->counter);
    delete w;
    return e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "cudaMalloc of a workspace failed")
                                          : cuda_error(e, "workspace");
  }
  *out = w;
  return GV_OK;
}

void gv_workspace_destroy(gv_workspace* w) {
  if (!w) return;
  if (w->idx) cudaFree(w->idx);
  if (w->counter) cudaFree(w->counter);
  delete w;
}

gv_status gv_workspace_refined(gv_workspace* w, void* stream, int64_t* n_refined) {
  if (!w || !n_refined) return set_error(GV_ERR_INVALID_ARG, "NULL workspace or output");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (w->fused_blocks > 0) {  // the one-launch pass left one count per block
    uint32_t h[256];
    const int nb = w->fused_blocks < 256 ? w->fused_blocks : 256;
    e = cudaMemcpyAsync(h, w->idx, sizeof(uint32_t) * (size_t)nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "gv_workspace_refined");
    int64_t sum = 0;
    for (int b = 0; b < nb; b++) sum += h[b];
    *n_refined = sum;
    return GV_OK;
  }
  unsigned long long h = 0;
  e = cudaMemcpyAsync(&h, w->counter, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "gv_workspace_refined");
  *n_refined = (int64_t)h;
  return GV_OK;
}

gv_status gv_query(const gv_solid* s, const gv_tracks* t, gv_precision prec, const gv_results* res,
                   gv_workspace* ws, void* stream) {
  const gv::Range range("gv_query");
  if (!s || !t || !res) return set_error(GV_ERR_INVALID_ARG, "NULL solid, tracks or results");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "negative track count");
  if (prec != GV_FP64 && prec != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "unknown precision");
  QueryArgs a{t->x, t->y, t->z, t->dx, t->dy, t->dz, res->inside, res->dist_in, res->dist_out,
              res->safety_in, res->safety_out, t->n};
  if (t->n == 0) return GV_OK;
  if (!a.x || !a.y || !a.z) return set_error(GV_ERR_INVALID_ARG, "NULL point array");
  if ((a.din || a.dout) && (!a.u || !a.v || !a.w))
    return set_error(GV_ERR_INVALID_ARG, "distances requested without directions");
  const void* ptrs[11] = {a.x, a.y, a.z, a.u, a.v, a.w, a.din, a.dout, a.sin, a.sout, nullptr};
  for (int i = 0; i < 10; i++)
    if (ptrs[i] && ((uintptr_t)ptrs[i] & 7u)) return set_error(GV_ERR_INVALID_ARG, "arrays must be 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (prec == GV_FP64) {
    e = launch_query_fp64(s, a, st);
  } else {
    if (!ws) return set_error(GV_ERR_INVALID_ARG, "GV_FP32_REFINE needs a workspace");
    if (ws->cap < t->n) return set_error(GV_ERR_OUT_OF_MEMORY, "workspace smaller than the basket");
    e = launch_query_fp32(s, a, ws->idx, ws->counter, st, &ws->fused_blocks);
  }
  if (e != cudaSuccess) return cuda_error(e, "gv_query launch");
  return GV_OK;
}

gv_status gv_debug_status(uint32_t* codes, int64_t* first_index, int32_t clear) {
  if (!codes || !first_index) return set_error(GV_ERR_INVALID_ARG, "gv_debug_status: NULL output");
#ifdef GV_DEBUG
  cudaError_t e = cudaDeviceSynchronize();
  unsigned long long w32[2] = {0ull, ~0ull}, w64[2] = {0ull, ~0ull}, ws[2] = {0ull, ~0ull};
  if (e == cudaSuccess) e = debug_read_query32(w32, clear != 0);
  if (e == cudaSuccess) e = debug_read_query64(w64, clear != 0);
  if (e == cudaSuccess) e = debug_read_query_small(ws, clear != 0);
  if (e != cudaSuccess) return cuda_error(e, "gv_debug_status");
  *codes = (uint32_t)(w32[0] | w64[0] | ws[0]);
  unsigned long long m = w32[1] < w64[1] ? w32[1] : w64[1];
  if (ws[1] < m) m = ws[1];
  *first_index = m == ~0ull ? -1 : (int64_t)m;
  return GV_OK;
#else
  (void)clear;
  *codes = 0;
  *first_index = -1;
  return set_error(GV_ERR_UNSUPPORTED, "gv_debug_status: built without GV_DEBUG");
#endif
}

const char* gv_last_error(void) { return g_last_error.c_str(); }

const char* gv_version(void) { return "gvgeo 0.1 (sm_103a)"; }

}  // extern "C"
