// desc_build.h -- host construction of the solid descriptors: validation and the
// derived constants (plane normals and offsets of the trapezoid faces, section lines,
// phi-plane normals, binary32 splits), with no CUDA call, so that the library's
// constructors and the benchmark's CPU loop build the same records.
//
// The derived constants are computed in binary64 with the host libm; every file that
// includes this header is compiled with -ffp-contract=off so that every expression
// rounds exactly as written.  Every rule below is stated in gv.h.
#pragma once
#include <cmath>
#include <cstring>
#include "gv.h"
#include "gv_desc.h"

namespace gv {

// Outcome of a construction: GV_OK, or a status with a message.
struct Built {
  gv_status st;
  const char* msg;
};
inline Built built_ok() { return {GV_OK, ""}; }
inline Built built_err(gv_status st, const char* msg) { return {st, msg}; }

inline bool finite(double v) { return std::isfinite(v); }

inline void set_plane(double* P, double nx, double ny, double nz, double c) {
  P[0] = nx; P[1] = ny; P[2] = nz; P[3] = c;
}

inline double dot3(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

// Side face through the quad (A, B, C, D): n = (C - A) x (D - B), turned away
// from the vertex centroid cs, normalised; offset = mean of n.V over the quad.
inline bool face_plane(const double* A, const double* B, const double* C, const double* D,
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

inline void split_f(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// Binary32 split constants of every binary64 constant of the descriptor.
inline void fill_f32(Desc& h) {
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

// Features finer than 2^-16 of the solid's size: binary64 only (kFp64Only).
constexpr double kFineFeature = 1.0 / 65536.0;
inline void mark_fine_features(Desc& h) {
  if (h.type == kBox) {
    const double big = std::fmax(h.D[0], std::fmax(h.D[1], h.D[2]));
    if (std::fmin(h.D[0], std::fmin(h.D[1], h.D[2])) < kFineFeature * big) h.flags |= kFp64Only;
    return;
  }
  if (h.type == kTrd || h.type == kTrap) {
    const double big = std::fmax(h.ext[0], std::fmax(h.ext[1], h.ext[2]));
    if (h.dz < kFineFeature * big) h.flags |= kFp64Only;
    return;
  }
  const double big = std::fmax(h.ext[0], h.ext[2]);
  for (int k = 0; k + 1 < h.nz; k++) {
    if (h.z[k + 1] - h.z[k] < kFineFeature * big) h.flags |= kFp64Only;
    if ((h.inner >> k) & 1u) {
      for (int j = k; j <= k + 1; j++) {  // wall thickness at both planes of the section
        const double ro = h.out[k].a * h.z[j] + h.out[k].b, ri = h.in[k].a * h.z[j] + h.in[k].b;
        if (ri > 0 && ro - ri < kFineFeature * big) h.flags |= kFp64Only;
      }
    }
  }
}

inline void init_desc(Desc& h, int type) {
  std::memset(&h, 0, sizeof(h));
  h.type = type;
}

inline Built build_box(double dx, double dy, double dz, Desc& h) {
  if (!(dx > 0 && dy > 0 && dz > 0) || !std::isfinite(dx + dy + dz))
    return built_err(GV_ERR_INVALID_ARG, "box: half-lengths must be finite and positive");
  init_desc(h, kBox);
  h.D[0] = dx; h.D[1] = dy; h.D[2] = dz;
  h.dz = dz;
  h.ext[0] = dx; h.ext[1] = dy; h.ext[2] = dz;
  mark_fine_features(h);
  fill_f32(h);
  return built_ok();
}

inline Built build_trap(const double p[11], int type, Desc& h) {
  for (int i = 0; i < 11; i++)
    if (!finite(p[i])) return built_err(GV_ERR_INVALID_ARG, "trap: non-finite parameter");
  const double dz = p[0], th = p[1], ph = p[2];
  if (!(dz > 0 && p[3] > 0 && p[4] > 0 && p[5] > 0 && p[7] > 0 && p[8] > 0 && p[9] > 0))
    return built_err(GV_ERR_INVALID_ARG, "trap: half-lengths must be positive");
  if (!(std::fabs(th) < 1.5707963267948966 && std::fabs(p[6]) < 1.5707963267948966 &&
        std::fabs(p[10]) < 1.5707963267948966))
    return built_err(GV_ERR_INVALID_ARG, "trap: |theta|, |alpha| must be below pi/2");
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
    return built_err(GV_ERR_INVALID_ARG, "trap: a side face is not planar (or is degenerate)");
  h.dz = dz;
  for (int k = 0; k < 8; k++)
    for (int i = 0; i < 3; i++) h.ext[i] = std::fmax(h.ext[i], std::fabs(v[k][i]));
  mark_fine_features(h);
  fill_f32(h);
  return built_ok();
}

inline void set_line(Line& L, double r0, double r1, double z0, double z1) {
  L.a = (r1 - r0) / (z1 - z0);
  L.b = r0 - L.a * z0;
  L.k = 1.0 / std::sqrt(1.0 + L.a * L.a);
}

inline Built build_pcon(int type, int nz, const double* z, const double* rmin, const double* rmax,
                        double sphi, double dphi, Desc& h) {
  if (nz < 2) return built_err(GV_ERR_INVALID_ARG, "polycone: at least two z-planes");
  if (nz > kMaxZ) return built_err(GV_ERR_UNSUPPORTED, "polycone: more than GV_MAX_ZPLANES z-planes");
  if (!z || !rmin || !rmax) return built_err(GV_ERR_INVALID_ARG, "polycone: NULL array");
  if (!finite(sphi) || !finite(dphi) || !(dphi > 0))
    return built_err(GV_ERR_INVALID_ARG, "phi range must be finite with dphi > 0");
  for (int k = 0; k < nz; k++) {
    if (!finite(z[k]) || !finite(rmin[k]) || !finite(rmax[k]))
      return built_err(GV_ERR_INVALID_ARG, "non-finite z or radius");
    if (!(rmin[k] >= 0 && rmin[k] < rmax[k]))
      return built_err(GV_ERR_INVALID_ARG, "radii must satisfy 0 <= rmin < rmax");
    if (k > 0 && !(z[k] > z[k - 1]))
      return built_err(GV_ERR_INVALID_ARG, "z-planes must be strictly increasing");
  }
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
  if (dphi < twopi && (dphi < kFineFeature || twopi - dphi < kFineFeature)) h.flags |= kFp64Only;
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
  mark_fine_features(h);
  fill_f32(h);
  return built_ok();
}

inline Built build_tube(double rmin, double rmax, double dz, double sphi, double dphi, Desc& h) {
  if (!(dz > 0) || !std::isfinite(dz)) return built_err(GV_ERR_INVALID_ARG, "tube: dz must be positive");
  const double z[2] = {-dz, dz}, rn[2] = {rmin, rmin}, rx[2] = {rmax, rmax};
  return build_pcon(kTube, 2, z, rn, rx, sphi, dphi, h);
}

inline Built build_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz, double sphi,
                        double dphi, Desc& h) {
  if (!(dz > 0) || !std::isfinite(dz)) return built_err(GV_ERR_INVALID_ARG, "cone: dz must be positive");
  const double z[2] = {-dz, dz}, rn[2] = {rmin1, rmin2}, rx[2] = {rmax1, rmax2};
  return build_pcon(kCone, 2, z, rn, rx, sphi, dphi, h);
}

}  // namespace gv
