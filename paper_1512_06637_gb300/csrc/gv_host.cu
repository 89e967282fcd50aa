// gv_host.cu -- host side of the C ABI: solid constructors (validation and
// derived constants), workspaces, argument checks and launch dispatch.
//
// The derived constants (plane normals and offsets of the trapezoid faces, cone
// slopes, phi-plane normals) are computed here in binary64 with the host libm;
// this file is compiled with -ffp-contract=off so that every expression rounds
// exactly as written.  Every rule below is stated in gv.h.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
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

static bool finite(double v) { return std::isfinite(v); }

static void set_plane(double* P, double nx, double ny, double nz, double c) {
  P[0] = nx; P[1] = ny; P[2] = nz; P[3] = c;
}

static double dot3(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

// Side face through the quad (A, B, C, D): n = (C - A) x (D - B), turned away
// from the vertex centroid cs, normalised; offset = mean of n.V over the quad.
static bool face_plane(const double* A, const double* B, const double* C, const double* D,
                       const double* cs, double* P) {
  double u[3], w[3], n[3], e[3];
  for (int i = 0; i < 3; i++) { u[i] = C[i] - A[i]; w[i] = D[i] - B[i]; }
  n[0] = u[1] * w[2] - u[2] * w[1];
  n[1] = u[2] * w[0] - u[0] * w[2];
  n[2] = u[0] * w[1] - u[1] * w[0];
  for (int i = 0; i < 3; i++) e[i] = ((A[i] + B[i]) + (C[i] + D[i])) * 0.25 - cs[i];
  if (dot3(n, e) < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  const double len = std::sqrt(dot3(n, n));
  if (!(len > 0)) return false;
  for (int i = 0; i < 3; i++) n[i] = n[i] / len;
  const double c = ((dot3(n, A) + dot3(n, B)) + (dot3(n, C) + dot3(n, D))) * 0.25;
  const double* V[4] = {A, B, C, D};
  for (int i = 0; i < 4; i++)
    if (std::fabs(dot3(n, V[i]) - c) > 1e-9) return false;
  set_plane(P, n[0], n[1], n[2], c);
  return true;
}

static void split_f(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// Binary32 split constants of every binary64 constant of the descriptor.
static void fill_f32(Desc& h) {
  for (int i = 0; i < 3; i++) split_f(h.D[i], h.Dh[i], h.Dl[i]);
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) split_f(h.pl[i][j], h.plh[i][j], h.pll[i][j]);
  split_f(h.dz, h.dzh, h.dzl);
  for (int i = 0; i < 2; i++) {
    split_f(h.ns[i], h.nsh[i], h.nsl[i]);
    split_f(h.ne[i], h.neh[i], h.nel[i]);
  }
  float size = 0;
  for (int i = 0; i < 3; i++) size = std::fmax(size, (float)h.D[i]);
  for (int k = 0; k < h.nz; k++) {
    split_f(h.z[k], h.zh[k], h.zl[k]);
    long long bits;
    std::memcpy(&bits, &h.z[k], sizeof(bits));
    h.zkey[k] = order_key(bits);
    size = std::fmax(size, (float)std::fabs(h.z[k]));
  }
  for (int k = 0; k + 1 < h.nz; k++) {
    split_f(h.out[k].a, h.oah[k], h.oal[k]);
    split_f(h.out[k].b, h.obh[k], h.obl[k]);
    h.ok_[k] = (float)h.out[k].k;
    split_f(h.in[k].a, h.iah[k], h.ial[k]);
    split_f(h.in[k].b, h.ibh[k], h.ibl[k]);
    h.ik_[k] = (float)h.in[k].k;
  }
  h.size = size;
}

static gv_status upload(Desc h, gv_solid** out) {
  fill_f32(h);
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

static void init_desc(Desc& h, int type) {
  std::memset(&h, 0, sizeof(h));
  h.type = type;
}

static gv_status make_trap(const double p[11], int type, gv_solid** out) {
  for (int i = 0; i < 11; i++)
    if (!finite(p[i])) return set_error(GV_ERR_INVALID_ARG, "trap: non-finite parameter");
  const double dz = p[0], th = p[1], ph = p[2];
  if (!(dz > 0 && p[3] > 0 && p[4] > 0 && p[5] > 0 && p[7] > 0 && p[8] > 0 && p[9] > 0))
    return set_error(GV_ERR_INVALID_ARG, "trap: half-lengths must be positive");
  if (!(std::fabs(th) < 1.5707963267948966 && std::fabs(p[6]) < 1.5707963267948966 &&
        std::fabs(p[10]) < 1.5707963267948966))
    return set_error(GV_ERR_INVALID_ARG, "trap: |theta|, |alpha| must be below pi/2");
  Desc h;
  init_desc(h, type);
  const double tthc = std::tan(th) * std::cos(ph), tths = std::tan(th) * std::sin(ph);
  double v[8][3];
  for (int j = 0; j < 2; j++) {
    const double zf = j == 0 ? -dz : dz;
    const double dy = j == 0 ? p[3] : p[7];
    const double dxa = j == 0 ? p[4] : p[8];
    const double dxb = j == 0 ? p[5] : p[9];
    const double ta = std::tan(j == 0 ? p[6] : p[10]);
    const double cx = zf * tthc, cy = zf * tths;
    const double xm = cx - dy * ta, xp = cx + dy * ta;
    v[4 * j + 0][0] = xm - dxa; v[4 * j + 0][1] = cy - dy; v[4 * j + 0][2] = zf;
    v[4 * j + 1][0] = xm + dxa; v[4 * j + 1][1] = cy - dy; v[4 * j + 1][2] = zf;
    v[4 * j + 2][0] = xp - dxb; v[4 * j + 2][1] = cy + dy; v[4 * j + 2][2] = zf;
    v[4 * j + 3][0] = xp + dxb; v[4 * j + 3][1] = cy + dy; v[4 * j + 3][2] = zf;
  }
  double cs[3];
  for (int i = 0; i < 3; i++) {
    double acc = 0;
    for (int k = 0; k < 8; k++) acc = acc + v[k][i];
    cs[i] = acc * 0.125;
  }
  if (!face_plane(v[0], v[1], v[5], v[4], cs, h.pl[0]) ||  // -y
      !face_plane(v[2], v[6], v[7], v[3], cs, h.pl[1]) ||  // +y
      !face_plane(v[0], v[4], v[6], v[2], cs, h.pl[2]) ||  // -x
      !face_plane(v[1], v[3], v[7], v[5], cs, h.pl[3]))    // +x
    return set_error(GV_ERR_INVALID_ARG, "trap: a side face is not planar (or is degenerate)");
  h.dz = dz;
  for (int k = 0; k < 8; k++)
    for (int i = 0; i < 3; i++) h.ext[i] = std::fmax(h.ext[i], std::fabs(v[k][i]));
  return upload(h, out);
}

static void set_line(Line& L, double r0, double r1, double z0, double z1) {
  L.a = (r1 - r0) / (z1 - z0);
  L.b = r0 - L.a * z0;
  L.k = 1.0 / std::sqrt(1.0 + L.a * L.a);
}

static gv_status make_pcon(int type, int nz, const double* z, const double* rmin, const double* rmax,
                           double sphi, double dphi, gv_solid** out) {
  if (nz < 2) return set_error(GV_ERR_INVALID_ARG, "polycone: at least two z-planes");
  if (nz > kMaxZ) return set_error(GV_ERR_UNSUPPORTED, "polycone: more than GV_MAX_ZPLANES z-planes");
  if (!z || !rmin || !rmax) return set_error(GV_ERR_INVALID_ARG, "polycone: NULL array");
  if (!finite(sphi) || !finite(dphi) || !(dphi > 0))
    return set_error(GV_ERR_INVALID_ARG, "phi range must be finite with dphi > 0");
  for (int k = 0; k < nz; k++) {
    if (!finite(z[k]) || !finite(rmin[k]) || !finite(rmax[k]))
      return set_error(GV_ERR_INVALID_ARG, "non-finite z or radius");
    if (!(rmin[k] >= 0 && rmin[k] < rmax[k]))
      return set_error(GV_ERR_INVALID_ARG, "radii must satisfy 0 <= rmin < rmax");
    if (k > 0 && !(z[k] > z[k - 1]))
      return set_error(GV_ERR_INVALID_ARG, "z-planes must be strictly increasing");
  }
  Desc h;
  init_desc(h, type);
  h.nz = nz;
  for (int k = 0; k < nz; k++) h.z[k] = z[k];
  for (int k = 0; k + 1 < nz; k++) {
    set_line(h.out[k], rmax[k], rmax[k + 1], z[k], z[k + 1]);
    set_line(h.in[k], rmin[k], rmin[k + 1], z[k], z[k + 1]);
    if (rmin[k] > 0 || rmin[k + 1] > 0) h.inner |= 1u << k;
  }
  const double twopi = 6.283185307179586, pi = 3.141592653589793;
  if (dphi < twopi) h.flags |= kHasPhi;
  if (dphi > pi) h.flags |= kPhiWide;
  const double ephi = sphi + dphi;
  h.ns[0] = std::sin(sphi);
  h.ns[1] = -std::cos(sphi);
  h.ne[0] = -std::sin(ephi);
  h.ne[1] = std::cos(ephi);
  h.dz = 0.5 * (z[nz - 1] - z[0]);
  double rm = 0;
  for (int k = 0; k < nz; k++) rm = std::fmax(rm, rmax[k]);
  h.ext[0] = h.ext[1] = rm;
  h.ext[2] = std::fmax(std::fabs(z[0]), std::fabs(z[nz - 1]));
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
  if (!(dx > 0 && dy > 0 && dz > 0) || !std::isfinite(dx + dy + dz))
    return set_error(GV_ERR_INVALID_ARG, "box: half-lengths must be finite and positive");
  Desc h;
  init_desc(h, kBox);
  h.D[0] = dx; h.D[1] = dy; h.D[2] = dz;
  h.dz = dz;
  h.ext[0] = dx; h.ext[1] = dy; h.ext[2] = dz;
  return upload(h, out);
}

gv_status gv_solid_trap(const double p[11], gv_solid** out) {
  if (!p) return set_error(GV_ERR_INVALID_ARG, "trap: NULL parameter array");
  return make_trap(p, kTrap, out);
}

gv_status gv_solid_trd(double dx1, double dx2, double dy1, double dy2, double dz, gv_solid** out) {
  const double p[11] = {dz, 0, 0, dy1, dx1, dx1, 0, dy2, dx2, dx2, 0};
  return make_trap(p, kTrd, out);
}

gv_status gv_solid_tube(double rmin, double rmax, double dz, double sphi, double dphi, gv_solid** out) {
  if (!(dz > 0) || !std::isfinite(dz)) return set_error(GV_ERR_INVALID_ARG, "tube: dz must be positive");
  const double z[2] = {-dz, dz}, rn[2] = {rmin, rmin}, rx[2] = {rmax, rmax};
  return make_pcon(kTube, 2, z, rn, rx, sphi, dphi, out);
}

gv_status gv_solid_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz, double sphi,
                        double dphi, gv_solid** out) {
  if (!(dz > 0) || !std::isfinite(dz)) return set_error(GV_ERR_INVALID_ARG, "cone: dz must be positive");
  const double z[2] = {-dz, dz}, rn[2] = {rmin1, rmin2}, rx[2] = {rmax1, rmax2};
  return make_pcon(kCone, 2, z, rn, rx, sphi, dphi, out);
}

gv_status gv_solid_polycone(int nz, const double* z, const double* rmin, const double* rmax, double sphi,
                            double dphi, gv_solid** out) {
  return make_pcon(kPcon, nz, z, rmin, rmax, sphi, dphi, out);
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
  unsigned long long h = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, w->counter, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "gv_workspace_refined");
  *n_refined = (int64_t)h;
  return GV_OK;
}

gv_status gv_query(const gv_solid* s, const gv_tracks* t, gv_precision prec, const gv_results* res,
                   gv_workspace* ws, void* stream) {
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
    e = launch_query_fp32(s, a, ws->idx, ws->counter, st);
  }
  if (e != cudaSuccess) return cuda_error(e, "gv_query launch");
  return GV_OK;
}

const char* gv_last_error(void) { return g_last_error.c_str(); }

const char* gv_version(void) { return "gvgeo 0.1 (sm_103a)"; }

}  // extern "C"
