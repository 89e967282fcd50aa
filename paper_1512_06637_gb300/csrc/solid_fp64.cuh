// solid_fp64.cuh -- binary64 device evaluation of the five queries per solid.
//
// The three questions of the paper's VecGeom section, per track:
//   Inside      s = max of the solid's constraint values; INSIDE if s < -h,
//               OUTSIDE if s > h, SURFACE otherwise (h = 0.5e-9 mm).
//   Safety      SafetyToIn = s (OUTSIDE) / SafetyToOut = -s (INSIDE); 0 on the
//               surface; -1 from the wrong side.  Polycone: the sections taken
//               as closed pieces (minimum over pieces outside, the containing
//               piece inside).
//   Distance    closed forms: slab intervals for the planar solids, a walk over
//               the z-sections with exit roots for the polycone family, and for
//               DistanceToIn a candidate entry per surface checked against the
//               other constraints at the entry point.
// A SURFACE point enters when every constraint within the band shrinks along d; one
// that does not enter has DistanceToOut 0, one that enters DistanceToIn 0.  Grazing
// rays: a derivative per unit length within kTangent of zero is tangent (a curved
// wall is then left if convex, entered if concave, unless the ray runs along its
// straight generator); a constraint within the band whose surface the ray runs along
// slides: the ray stays on the boundary, so it never enters through it; a double
// root within its rounding bound is a touch; chords shorter than kMerge are touches.
// Decision quantities use __dadd_rn/__dmul_rn so that no multiply-add is fused
// into them.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include "gv_desc.h"

namespace gv {
namespace f64 {

constexpr double H = kHalfTol;
#define GV_INF CUDART_INF

__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ int code_of(double s) { return s < -H ? 0 : (s > H ? 2 : 1); }

enum : unsigned { kWantCode = 1, kWantDin = 2, kWantDout = 4, kWantSin = 8, kWantSout = 16 };

struct Track { double x, y, z, u, v, w; };
struct Result { int code; double din, dout, sin, sout; };

// Motion of a constraint along d: +1 grows, -1 shrinks, 0 runs along its surface.
__device__ __forceinline__ int plane_motion(double gd) {
  return gd > kTangent ? 1 : (gd < -kTangent ? -1 : 0);
}
// Derivative per unit length of a wall r = a z + b, outward: (dr/dt - a w) k; on the axis
// dr/dt is the length of the direction's xy part.
__device__ __forceinline__ double wall_gd(const Line& L, const Track& T, double r, double radial) {
  const double rd = r > 0 ? radial / r : __dsqrt_rn(xadd(xmul(T.u, T.u), xmul(T.v, T.v)));
  return xmul(xsub(rd, xmul(L.a, T.w)), L.k);
}
// A tangent wall curves away from the ray (left if outer, entered if inner) unless the ray
// lies in the meridian plane of the point, along the wall's straight generator.
__device__ __forceinline__ int wall_motion(double gd, const Track& T, double r, bool outer) {
  if (gd > kTangent) return 1;
  if (gd < -kTangent) return -1;
  if (r > 0 && fabs(xsub(xmul(T.x, T.v), xmul(T.y, T.u))) > kTangent * r) return outer ? 1 : -1;
  return 0;
}

// Surface start: does every constraint within the band shrink along d?
struct Motion {
  bool all_in = true;
  __device__ __forceinline__ void add(double g, int m) {
    if (g >= -H && m != -1) all_in = false;
  }
};
// A constraint the ray slides along: within the band, running along its surface.
__device__ __forceinline__ bool slides(double g, int m) { return fabs(g) <= H && m == 0; }
// The motion of a wall, computed only for a wall within the band (|g| <= h): elsewhere neither
// the surface-start rule nor sliding looks at it (-1 stands in), and the division is skipped.
__device__ __forceinline__ int wall_motion_near(double g, const Line& L, const Track& T, double r, double radial,
                                                bool outer) {
  if (!(fabs(g) <= H)) return -1;
  const double gd = wall_gd(L, T, r, radial);
  return wall_motion(outer ? gd : -gd, T, r, outer);
}

__device__ __forceinline__ void finish_safety(int code, double s_out_side, double s_in_side,
                                              Result& R) {
  R.sin = code == 0 ? -1.0 : (code == 1 ? 0.0 : s_out_side);
  R.sout = code == 2 ? -1.0 : (code == 1 ? 0.0 : s_in_side);
}

// Decision quantity s at an arbitrary point (no tolerance applied), per family.
__device__ inline double box_s(const Desc& S, double x, double y, double z) {
  return dmax(dmax(xsub(fabs(x), S.D[0]), xsub(fabs(y), S.D[1])), xsub(fabs(z), S.D[2]));
}
__device__ inline double planar_s(const Desc& S, double x, double y, double z) {
  double v = xsub(fabs(z), S.dz);
  for (int i = 0; i < 4; i++) {
    const double* P = S.pl[i];
    v = dmax(v, xsub(xadd(xadd(xmul(P[0], x), xmul(P[1], y)), xmul(P[2], z)), P[3]));
  }
  return v;
}

// An entering surface point: the exit t found is meaningful only if the ray is inside
// (no tolerance) just before it; a ray that never gets inside (a point a hair outside
// that enters too slowly to get in before the exit) leaves at once.  Checked at t / 2.
template <class SF>
__device__ __forceinline__ bool inside_before(const Desc& S, const Track& T, double t, SF sf) {
  if (!(t < GV_INF)) return false;
  const double h = 0.5 * t;
  return sf(S, T.x + h * T.u, T.y + h * T.v, T.z + h * T.w) <= 0;
}

// ------------------------------------------------------------------- box

__device__ inline void box_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  const double p[3] = {T.x, T.y, T.z}, d[3] = {T.u, T.v, T.w};
  double g[3];
  for (int i = 0; i < 3; i++) g[i] = xsub(fabs(p[i]), S.D[i]);
  const double s = dmax(dmax(g[0], g[1]), g[2]);
  R.code = code_of(s);
  finish_safety(R.code, s, -s, R);
  if (!(want & (kWantDin | kWantDout))) return;
  Motion m;
  bool slide = false;
  for (int i = 0; i < 3; i++) {
    const int mi = plane_motion(p[i] < 0 ? -d[i] : d[i]);
    m.add(g[i], mi);
    slide |= slides(g[i], mi);
  }
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && !m.all_in) R.dout = 0.0;
    else {
      double t = GV_INF;
      for (int i = 0; i < 3; i++)
        if (d[i] != 0) t = dmin(t, (copysign(S.D[i], d[i]) - p[i]) / d[i]);
      if (R.code == 1 && !inside_before(S, T, t, box_s)) t = 0.0;
      R.dout = t;
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.0;
    else if (R.code == 1) R.din = m.all_in ? 0.0 : GV_INF;  // convex: no later entry
    else if (slide) R.din = GV_INF;  // runs along a face plane: never in the interior
    else {
      double tn = -GV_INF, tf = GV_INF;
      bool miss = false;
      for (int i = 0; i < 3; i++) {
        if (d[i] == 0) { if (g[i] > 0) miss = true; continue; }
        tn = dmax(tn, (-copysign(S.D[i], d[i]) - p[i]) / d[i]);
        tf = dmin(tf, (copysign(S.D[i], d[i]) - p[i]) / d[i]);
      }
      R.din = (!miss && tf - tn > kMerge && tf > 0) ? tn : GV_INF;
    }
  }
}

// ------------------------------------------------------------ trd / trap

__device__ inline void planar_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  double g[5], gd[5];
  for (int i = 0; i < 4; i++) {
    const double* P = S.pl[i];
    g[i] = xsub(xadd(xadd(xmul(P[0], T.x), xmul(P[1], T.y)), xmul(P[2], T.z)), P[3]);
    gd[i] = xadd(xadd(xmul(P[0], T.u), xmul(P[1], T.v)), xmul(P[2], T.w));
  }
  g[4] = xsub(fabs(T.z), S.dz);
  gd[4] = T.z < 0 ? -T.w : T.w;
  double s = g[0];
  for (int i = 1; i < 5; i++) s = dmax(s, g[i]);
  R.code = code_of(s);
  finish_safety(R.code, s, -s, R);
  if (!(want & (kWantDin | kWantDout))) return;
  Motion m;
  bool slide = false;
  for (int i = 0; i < 5; i++) {
    const int mi = plane_motion(gd[i]);
    m.add(g[i], mi);
    slide |= slides(g[i], mi);
  }
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && !m.all_in) R.dout = 0.0;
    else {
      double t = GV_INF;
      for (int i = 0; i < 4; i++)
        if (gd[i] > 0) t = dmin(t, -g[i] / gd[i]);
      if (T.w != 0) t = dmin(t, (copysign(S.dz, T.w) - T.z) / T.w);
      if (R.code == 1 && !inside_before(S, T, t, planar_s)) t = 0.0;
      R.dout = t;
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.0;
    else if (R.code == 1) R.din = m.all_in ? 0.0 : GV_INF;  // convex: no later entry
    else if (slide) R.din = GV_INF;  // runs along a face plane: never in the interior
    else {
      double tn = -GV_INF, tf = GV_INF;
      bool miss = false;
      for (int i = 0; i < 4; i++) {
        if (gd[i] == 0) { if (g[i] > 0) miss = true; continue; }
        const double t = -g[i] / gd[i];
        if (gd[i] < 0) tn = dmax(tn, t); else tf = dmin(tf, t);
      }
      if (T.w == 0) { if (g[4] > 0) miss = true; }
      else {
        tn = dmax(tn, (-copysign(S.dz, T.w) - T.z) / T.w);
        tf = dmin(tf, (copysign(S.dz, T.w) - T.z) / T.w);
      }
      R.din = (!miss && tf - tn > kMerge && tf > 0) ? tn : GV_INF;
    }
  }
}

// ------------------------------------- polycone family (tube, cone, polycone)

struct Phi { double a, b; };
__device__ __forceinline__ Phi phi_eval(const Desc& S, double x, double y) {
  return {xadd(xmul(S.ns[0], x), xmul(S.ns[1], y)), xadd(xmul(S.ne[0], x), xmul(S.ne[1], y))};
}
__device__ __forceinline__ double phi_g(const Desc& S, const Phi& f) {
  return (S.flags & kPhiWide) ? dmin(f.a, f.b) : dmax(f.a, f.b);
}

// Sliding constraints of a polycone-family track (bits), its start section k0.
enum : unsigned { kSlOut = 1, kSlIn = 2, kSlZ0 = 4, kSlZL = 8, kSlPs = 16, kSlPe = 32 };

// Entry checks.  An entry at t through one surface counts when the ray is inside every other
// constraint at t + kMerge: g + kMerge g' < 0 at the entry point.  A constraint left within
// kMerge of t gives a chord shorter than kMerge (a touch); one entered within kMerge of t is
// entered at the same crossing (crossings closer than kMerge merge).  A sliding constraint
// never holds the interior.
struct Entry {
  double u, v, w;     // direction
  double nds, nde;    // phi normals . d
  unsigned sl;        // sliding bits
  int k0;
};
// Phi membership of an entry point.
__device__ __forceinline__ bool phi_ok(const Desc& S, const Entry& E, double x, double y) {
  if (!(S.flags & kHasPhi)) return true;
  const bool a_ok = !(E.sl & kSlPs) && xadd(xadd(xmul(S.ns[0], x), xmul(S.ns[1], y)), kMerge * E.nds) < 0;
  const bool b_ok = !(E.sl & kSlPe) && xadd(xadd(xmul(S.ne[0], x), xmul(S.ne[1], y)), kMerge * E.nde) < 0;
  return (S.flags & kPhiWide) ? (a_ok || b_ok) : (a_ok && b_ok);
}
// Between the end planes at an entry point.
__device__ __forceinline__ bool zends_ok(const Desc& S, const Entry& E, double z) {
  const int last = S.nz - 1;
  return xsub(z, S.z[0]) > kMerge * -E.w && xsub(S.z[last], z) > kMerge * E.w;
}

__device__ __forceinline__ int section_of(const Desc& S, double z) {
  int k = 0;
  while (k < S.nz - 2 && z >= S.z[k + 1]) k++;
  return k;
}

__device__ __forceinline__ double g_out(const Line& L, double r, double z) {
  return xmul(xsub(r, xadd(xmul(L.a, z), L.b)), L.k);
}
__device__ __forceinline__ double g_in(const Line& L, double r, double z) {
  return xmul(xsub(xadd(xmul(L.a, z), L.b), r), L.k);
}

// Crossings of r = a z + b (on the nappe a z + b >= 0) along the track: tm where the
// track enters {r <= R}, tp where it leaves it.  Roots of A t^2 + 2 B t + C = 0 by the
// cancellation-free pair; A t + B = -/+ sqrt(disc) tells entry from exit.  The
// coefficients and the discriminant are rounded operation by operation (no fused
// multiply-add); a discriminant within its rounding bound kDisc (|B| Bs + |A| Cs + |C| As),
// As, Bs, Cs the magnitudes of the terms of A, B, C, is a double root: a touch.
struct Cross { double tm, tp; bool hm, hp; };
__device__ inline Cross line_cross(const Line& L, const Track& T, double r2, double radial,
                                   double A0, double bs0) {
  const double P = xadd(xmul(L.a, T.z), L.b), D = xmul(L.a, T.w);
  const double A = xsub(A0, xmul(D, D)), B = xsub(radial, xmul(P, D)), C = xsub(r2, xmul(P, P));
  Cross c{0, 0, false, false};
  if (A == 0) {
    if (B != 0) {
      const double t = -C / (2 * B);
      if (B > 0) { c.tp = t; c.hp = true; } else { c.tm = t; c.hm = true; }
    }
  } else {
    const double disc = xsub(xmul(B, B), xmul(A, C));
    const double As = xadd(A0, xmul(D, D)), Cs = xadd(r2, xmul(P, P));
    const double Bs = xadd(bs0, fabs(xmul(P, D)));
    const double eps = xmul(kDisc, xadd(xadd(xmul(fabs(B), Bs), xmul(fabs(A), Cs)), xmul(fabs(C), As)));
    if (disc > eps) {
      const double sq = sqrt(disc);
      if (B >= 0) { const double q = -(B + sq); c.tm = q / A; c.tp = C / q; }
      else        { const double q = sq - B;    c.tp = q / A; c.tm = C / q; }
      c.hm = c.hp = true;
    }
  }
  if (c.hm && !(L.a * (T.z + c.tm * T.w) + L.b >= 0)) c.hm = false;
  if (c.hp && !(L.a * (T.z + c.tp * T.w) + L.b >= 0)) c.hp = false;
  return c;
}

__device__ __forceinline__ bool inner_has(const Desc& S, int k) { return (S.inner >> k) & 1u; }

// Lateral membership of an entry point in section k (skip_out / skip_in: the surface
// entered through), with the entry margin: (r^2 - R^2) + 2 kMerge d(r^2 - R^2)/dt / 2 < 0
// for the outer wall and the reverse for the inner one.  The walls of the start section
// slide when their bit is set: never inside there.
__device__ __forceinline__ bool radial_ok(const Desc& S, const Entry& E, int k, double x, double y, double z,
                                          bool skip_out, bool skip_in) {
  const double r2 = x * x + y * y, rd = x * E.u + y * E.v;
  if (!skip_out) {
    if (k == E.k0 && (E.sl & kSlOut)) return false;
    const double R = S.out[k].a * z + S.out[k].b;
    if (!(R > 0 && (r2 - R * R) + 2 * kMerge * (rd - R * (S.out[k].a * E.w)) < 0)) return false;
  }
  if (!skip_in && inner_has(S, k)) {
    if (k == E.k0 && (E.sl & kSlIn)) return false;
    const double R = S.in[k].a * z + S.in[k].b;
    if (R >= 0 && !((r2 - R * R) - 2 * kMerge * (R * (S.in[k].a * E.w) - rd) > 0)) return false;
  }
  return true;
}

// Closed piece k: lateral, its own two planes, phi.
__device__ inline double s_closed(const Desc& S, int k, double r, double z, double gphi) {
  double v = g_out(S.out[k], r, z);
  v = dmax(v, xsub(S.z[k], z));
  v = dmax(v, xsub(z, S.z[k + 1]));
  if (inner_has(S, k)) v = dmax(v, g_in(S.in[k], r, z));
  if (S.flags & kHasPhi) v = dmax(v, gphi);
  return v;
}

__device__ inline double pcon_s(const Desc& S, double x, double y, double z) {
  const int last = S.nz - 1;
  const double r = __dsqrt_rn(xadd(xmul(x, x), xmul(y, y)));
  const int k = section_of(S, z);
  double v = dmax(g_out(S.out[k], r, z), dmax(xsub(S.z[0], z), xsub(z, S.z[last])));
  if (inner_has(S, k)) v = dmax(v, g_in(S.in[k], r, z));
  if (S.flags & kHasPhi) v = dmax(v, phi_g(S, phi_eval(S, x, y)));
  return v;
}
// The same with the phi planes of a wide segment that the ray slides along taken as
// violated (the only sliding constraints a track that travels inside can have).
__device__ inline double pcon_s_wide(const Desc& S, double x, double y, double z, unsigned sl) {
  const int last = S.nz - 1;
  const double r = __dsqrt_rn(xadd(xmul(x, x), xmul(y, y)));
  const int k = section_of(S, z);
  double v = dmax(g_out(S.out[k], r, z), dmax(xsub(S.z[0], z), xsub(z, S.z[last])));
  if (inner_has(S, k)) v = dmax(v, g_in(S.in[k], r, z));
  if (S.flags & kHasPhi) {
    Phi f = phi_eval(S, x, y);
    if (sl & kSlPs) f.a = GV_INF;
    if (sl & kSlPe) f.b = GV_INF;
    v = dmax(v, phi_g(S, f));
  }
  return v;
}

__device__ inline void pcon_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  const int nz = S.nz, last = nz - 1;
  const double r2 = xadd(xmul(T.x, T.x), xmul(T.y, T.y));
  const double r = __dsqrt_rn(r2);
  const int k0 = section_of(S, T.z);
  const bool has_phi = S.flags & kHasPhi, wide = S.flags & kPhiWide;
  Phi f{0, 0};
  double gphi = -GV_INF;
  if (has_phi) { f = phi_eval(S, T.x, T.y); gphi = phi_g(S, f); }
  const double go = g_out(S.out[k0], r, T.z);
  const double gi = inner_has(S, k0) ? g_in(S.in[k0], r, T.z) : -GV_INF;
  const double gz0 = xsub(S.z[0], T.z), gz1 = xsub(T.z, S.z[last]);
  const double s = dmax(dmax(dmax(go, gi), dmax(gz0, gz1)), gphi);
  R.code = code_of(s);
  if (want & (kWantSin | kWantSout)) {
    double sin_v = s, sout_v = -s;
    if (nz > 2) {
      if (R.code == 2) {
        sin_v = s_closed(S, 0, r, T.z, gphi);
        for (int k = 1; k < last; k++) sin_v = dmin(sin_v, s_closed(S, k, r, T.z, gphi));
      } else if (R.code == 0) {
        sout_v = -s_closed(S, k0, r, T.z, gphi);
      }
    }
    finish_safety(R.code, sin_v, sout_v, R);
  }
  if (!(want & (kWantDin | kWantDout))) return;

  const double radial = xadd(xmul(T.x, T.u), xmul(T.y, T.v));
  double nds = 0, nde = 0;
  Motion m;
  unsigned sl = 0;
  {
    const int mo = wall_motion_near(go, S.out[k0], T, r, radial, true);
    m.add(go, mo);
    if (slides(go, mo)) sl |= kSlOut;
    if (inner_has(S, k0)) {
      const int mi = wall_motion_near(gi, S.in[k0], T, r, radial, false);
      m.add(gi, mi);
      if (slides(gi, mi)) sl |= kSlIn;
    }
    const int m0 = plane_motion(-T.w), m1 = plane_motion(T.w);
    m.add(gz0, m0);
    m.add(gz1, m1);
    if (slides(gz0, m0)) sl |= kSlZ0;
    if (slides(gz1, m1)) sl |= kSlZL;
    if (has_phi) {
      nds = xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v));
      nde = xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v));
      const int ms = plane_motion(nds), me = plane_motion(nde);
      if (wide) { if (f.a <= f.b) m.add(f.a, ms); else m.add(f.b, me); }
      else { m.add(f.a, ms); m.add(f.b, me); }
      if (slides(f.a, ms)) sl |= kSlPs;
      if (slides(f.b, me)) sl |= kSlPe;
    }
  }
  const double A0 = xadd(xmul(T.u, T.u), xmul(T.v, T.v));
  const double bs0 = xadd(fabs(xmul(T.x, T.u)), fabs(xmul(T.y, T.v)));

  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && !m.all_in) R.dout = 0.0;
    else {
      // phi boundary (a track that travels inside can slide only along a wide segment's
      // plane on its inner side: that plane is then no part of the boundary it can leave by)
      double tphi = GV_INF;
      if (has_phi) {
        if (!wide) {
          if (nds > 0) tphi = dmin(tphi, -f.a / nds);
          if (nde > 0) tphi = dmin(tphi, -f.b / nde);
        } else {  // leave the union of half-planes = enter the excluded wedge
          double tin = -GV_INF, tout = GV_INF;
          bool never = false;
          if (!(sl & kSlPs)) {
            if (nds > 0) tin = dmax(tin, -f.a / nds);
            else if (nds < 0) tout = dmin(tout, -f.a / nds);
            else if (!(f.a > 0)) never = true;
          }
          if (!(sl & kSlPe)) {
            if (nde > 0) tin = dmax(tin, -f.b / nde);
            else if (nde < 0) tout = dmin(tout, -f.b / nde);
            else if (!(f.b > 0)) never = true;
          }
          if (!never && tin < tout && tin > 0) tphi = tin;
        }
      }
      // walk the z-sections
      int k = k0;
      double tlo = 0, t = GV_INF;
      for (int guard = 0; guard < kMaxZ; guard++) {
        double tl = GV_INF;
        const Cross co = line_cross(S.out[k], T, r2, radial, A0, bs0);
        if (co.hp && co.tp > tlo) tl = co.tp;
        if (inner_has(S, k)) {
          const Cross ci = line_cross(S.in[k], T, r2, radial, A0, bs0);
          if (ci.hm && ci.tm > tlo) tl = dmin(tl, ci.tm);
        }
        double tp;
        bool end;
        if (T.w > 0) { tp = (S.z[k + 1] - T.z) / T.w; end = (k + 1 == last); }
        else if (T.w < 0) { tp = (S.z[k] - T.z) / T.w; end = (k == 0); }
        else { tp = GV_INF; end = true; }
        if (tl <= tp) { t = tl; break; }
        if (end) { t = tp; break; }
        k += T.w > 0 ? 1 : -1;
        tlo = tp;
      }
      t = dmin(t, tphi);
      if (R.code == 1 && !(t < GV_INF && pcon_s_wide(S, T.x + 0.5 * t * T.u, T.y + 0.5 * t * T.v,
                                                     T.z + 0.5 * t * T.w, sl) <= 0))
        t = 0.0;
      R.dout = t;
    }
  }

  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.0;
    else if (R.code == 1 && m.all_in) R.din = 0.0;
    else if ((sl & (kSlZ0 | kSlZL)) || (!wide && (sl & (kSlPs | kSlPe))) ||
             ((sl & (kSlPs | kSlPe)) == (kSlPs | kSlPe))) {
      R.din = GV_INF;  // runs along an end plane or a phi plane bounding every point: no entry
    } else {
      const Entry E{T.u, T.v, T.w, nds, nde, sl, k0};
      double best = GV_INF;
      // lateral surfaces of every section the track can reach
      for (int k = 0; k < last; k++) {
        if (T.w > 0 && S.z[k + 1] < T.z) continue;
        if (T.w < 0 && S.z[k] > T.z) continue;
        if (T.w == 0 && (T.z < S.z[k] || T.z > S.z[k + 1])) continue;
        if (!(k == k0 && (sl & kSlOut))) {
          const Cross co = line_cross(S.out[k], T, r2, radial, A0, bs0);
          if (co.hm && co.tm > 0 && co.tm < best) {
            const double qx = T.x + co.tm * T.u, qy = T.y + co.tm * T.v, qz = T.z + co.tm * T.w;
            if (qz >= S.z[k] && qz <= S.z[k + 1] && zends_ok(S, E, qz) &&
                radial_ok(S, E, k, qx, qy, qz, true, false) && phi_ok(S, E, qx, qy))
              best = co.tm;
          }
        }
        if (inner_has(S, k) && !(k == k0 && (sl & kSlIn))) {
          const Cross ci = line_cross(S.in[k], T, r2, radial, A0, bs0);
          if (ci.hp && ci.tp > 0 && ci.tp < best) {
            const double qx = T.x + ci.tp * T.u, qy = T.y + ci.tp * T.v, qz = T.z + ci.tp * T.w;
            if (qz >= S.z[k] && qz <= S.z[k + 1] && zends_ok(S, E, qz) &&
                radial_ok(S, E, k, qx, qy, qz, false, true) && phi_ok(S, E, qx, qy))
              best = ci.tp;
          }
        }
      }
      // end planes
      if (T.w != 0) {
        const int kk = T.w > 0 ? 0 : last - 1;
        const double ze = T.w > 0 ? S.z[0] : S.z[last];
        const double t = (ze - T.z) / T.w;
        if (t > 0 && t < best) {
          const double qx = T.x + t * T.u, qy = T.y + t * T.v;
          if (radial_ok(S, E, kk, qx, qy, ze, false, false) && phi_ok(S, E, qx, qy)) best = t;
        }
      }
      // phi planes
      if (has_phi) {
        for (int j = 0; j < 2; j++) {
          const double a = j == 0 ? f.a : f.b, nd = j == 0 ? nds : nde;
          if ((sl & (j == 0 ? kSlPs : kSlPe)) || !(nd < 0)) continue;
          const double t = -a / nd;
          if (!(t > 0 && t < best)) continue;
          const double qx = T.x + t * T.u, qy = T.y + t * T.v, qz = T.z + t * T.w;
          if (!zends_ok(S, E, qz)) continue;
          const int kq = section_of(S, qz);
          if (!radial_ok(S, E, kq, qx, qy, qz, false, false)) continue;
          if (!wide) {  // inside the other plane
            const double* n2 = j == 0 ? S.ne : S.ns;
            const double nd2 = j == 0 ? nde : nds;
            if (!(xadd(xadd(xmul(n2[0], qx), xmul(n2[1], qy)), kMerge * nd2) < 0)) continue;
          }
          best = t;
        }
      }
      R.din = best;
    }
  }
}

// ------------------------------------------------------------ boolean solids
//
// op(a, c) for two primitives, c placed in a's frame.  Codes and safeties come from the
// components' decision quantities and safeties (union min / max, intersection max / min,
// subtraction as a and not-c).  Distances come from the pieces of the ray inside each
// component - the intervals of t on which the component's s <= 0, found from its surfaces
// in closed form - combined with the set operation; the first piece starting after 0 is
// the entry and the end of the piece holding 0+ (else of the first piece after 0) the exit.
// A component surface the ray slides along holds no piece of that component (the ray is
// on its boundary), except for the subtracted component c, whose complement it bounds:
// there the sliding surface is taken as holding c.  Pieces shorter than kMerge and gaps
// between pieces shorter than kMerge vanish.

constexpr int kMaxPieces = 96;
struct Pieces {
  int n = 0;
  bool over = false;
  double a[kMaxPieces], b[kMaxPieces];
  // pieces arrive in increasing t; a piece touching or overlapping the last is merged
  __device__ __forceinline__ void push(double lo, double hi) {
    if (!(hi - lo > kMerge)) return;
    if (n > 0 && lo - b[n - 1] <= kMerge) {
      if (hi > b[n - 1]) b[n - 1] = hi;
      return;
    }
    if (n < kMaxPieces) { a[n] = lo; b[n] = hi; n++; } else over = true;
  }
};

// constraint g + t gd <= 0 along the ray: clip [lo, hi]; a sliding constraint holds
// nothing (hold = false) or everything (hold = true)
__device__ __forceinline__ void clip_le(double g, double gd, bool hold, double& lo, double& hi) {
  if (slides(g, plane_motion(gd))) {
    if (!hold) { lo = GV_INF; hi = -GV_INF; }
    return;
  }
  if (gd == 0) { if (g > 0) { lo = GV_INF; hi = -GV_INF; } return; }
  const double t = -g / gd;
  if (gd > 0) hi = dmin(hi, t); else lo = dmax(lo, t);
}

__device__ inline void planar_pieces(const Desc& S, const Track& T, bool hold, Pieces& P) {
  double lo = -GV_INF, hi = GV_INF;
  if (S.type == kBox) {
    const double p[3] = {T.x, T.y, T.z}, d[3] = {T.u, T.v, T.w};
    for (int i = 0; i < 3; i++) {
      clip_le(xsub(p[i], S.D[i]), d[i], hold, lo, hi);            //  x - D <= 0
      clip_le(xsub(-p[i], S.D[i]), -d[i], hold, lo, hi);          // -x - D <= 0
    }
  } else {
    for (int i = 0; i < 4; i++) {
      const double* Q = S.pl[i];
      clip_le(xsub(xadd(xadd(xmul(Q[0], T.x), xmul(Q[1], T.y)), xmul(Q[2], T.z)), Q[3]),
              xadd(xadd(xmul(Q[0], T.u), xmul(Q[1], T.v)), xmul(Q[2], T.w)), hold, lo, hi);
    }
    clip_le(xsub(T.z, S.dz), T.w, hold, lo, hi);
    clip_le(xsub(-T.z, S.dz), -T.w, hold, lo, hi);
  }
  P.push(lo, hi);
}

// the region r <= a z + b (one nappe) of a section line along the ray
__device__ __forceinline__ void cone_region(const Line& L, const Track& T, double r2, double radial, double A0,
                                            double bs0, double r, double& lo, double& hi) {
  const Cross c = line_cross(L, T, r2, radial, A0, bs0);
  if (c.hm || c.hp) {
    lo = c.hm ? c.tm : -GV_INF;
    hi = c.hp ? c.tp : GV_INF;
  } else if (xsub(r, xadd(xmul(L.a, T.z), L.b)) <= 0) {  // no crossing: the whole line or nothing
    lo = -GV_INF; hi = GV_INF;
  } else {
    lo = GV_INF; hi = -GV_INF;
  }
}

// [lo, hi] minus (xlo, xhi): up to two pieces, pushed in order
__device__ __forceinline__ int minus(double lo, double hi, double xlo, double xhi, double* oa, double* ob) {
  if (!(xlo < xhi) || xhi <= lo || xlo >= hi) { oa[0] = lo; ob[0] = hi; return 1; }
  int m = 0;
  if (xlo > lo) { oa[m] = lo; ob[m] = xlo; m++; }
  if (xhi < hi) { oa[m] = xhi; ob[m] = hi; m++; }
  return m;
}

// The sliding constraints of a polycone-family primitive at the track's start.
__device__ inline unsigned pcon_slides(const Desc& S, const Track& T, double r, double radial, int k0) {
  unsigned sl = 0;
  const double go = g_out(S.out[k0], r, T.z);
  if (slides(go, wall_motion_near(go, S.out[k0], T, r, radial, true))) sl |= kSlOut;
  if (inner_has(S, k0)) {
    const double gi = g_in(S.in[k0], r, T.z);
    if (slides(gi, wall_motion_near(gi, S.in[k0], T, r, radial, false))) sl |= kSlIn;
  }
  if (slides(xsub(S.z[0], T.z), plane_motion(-T.w))) sl |= kSlZ0;
  if (slides(xsub(T.z, S.z[S.nz - 1]), plane_motion(T.w))) sl |= kSlZL;
  if (S.flags & kHasPhi) {
    const Phi f = phi_eval(S, T.x, T.y);
    if (slides(f.a, plane_motion(xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v))))) sl |= kSlPs;
    if (slides(f.b, plane_motion(xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v))))) sl |= kSlPe;
  }
  return sl;
}

__device__ inline void pcon_pieces(const Desc& S, const Track& T, bool hold, Pieces& P) {
  const int last = S.nz - 1;
  const double r2 = xadd(xmul(T.x, T.x), xmul(T.y, T.y));
  const double r = __dsqrt_rn(r2);
  const double radial = xadd(xmul(T.x, T.u), xmul(T.y, T.v));
  const double A0 = xadd(xmul(T.u, T.u), xmul(T.v, T.v));
  const double bs0 = xadd(fabs(xmul(T.x, T.u)), fabs(xmul(T.y, T.v)));
  const int k0 = section_of(S, T.z);
  const unsigned sl = pcon_slides(S, T, r, radial, k0);
  if (!hold && (sl & (kSlZ0 | kSlZL))) return;  // runs along an end plane: on the boundary
  double plo = -GV_INF, phi_hi = GV_INF, xlo = GV_INF, xhi = -GV_INF;  // narrow phi; wide-phi wedge
  if (S.flags & kHasPhi) {
    const Phi f = phi_eval(S, T.x, T.y);
    const double nds = xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v));
    const double nde = xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v));
    if (!(S.flags & kPhiWide)) {
      clip_le(f.a, nds, hold, plo, phi_hi);
      clip_le(f.b, nde, hold, plo, phi_hi);
    } else {  // the wedge n_s.p > 0 and n_e.p > 0; a sliding plane bounds it (hold: never in it)
      xlo = -GV_INF; xhi = GV_INF;
      if (hold && (sl & (kSlPs | kSlPe))) { xlo = GV_INF; xhi = -GV_INF; }
      if (!(sl & kSlPs)) clip_le(-f.a, -nds, false, xlo, xhi);
      if (!(sl & kSlPe)) clip_le(-f.b, -nde, false, xlo, xhi);
    }
  }
  const int kb = T.w < 0 ? last - 1 : 0, step = T.w < 0 ? -1 : 1;
  for (int i = 0; i < last; i++) {
    const int k = kb + step * i;
    double slo, shi;
    if (T.w > 0) { slo = (S.z[k] - T.z) / T.w; shi = (S.z[k + 1] - T.z) / T.w; }
    else if (T.w < 0) { slo = (S.z[k + 1] - T.z) / T.w; shi = (S.z[k] - T.z) / T.w; }
    else {  // the ray stays in the plane z = const: the section holding it, between the end planes
      if (k != section_of(S, T.z)) continue;
      if (!(T.z >= S.z[0] || (hold && (sl & kSlZ0))) || !(T.z <= S.z[last] || (hold && (sl & kSlZL)))) continue;
      slo = -GV_INF; shi = GV_INF;
    }
    if (hold && T.w != 0) {  // a sliding end plane holds the subtracted component everywhere along it
      if ((sl & kSlZ0) && k == 0) { if (T.w > 0) slo = -GV_INF; else shi = GV_INF; }
      if ((sl & kSlZL) && k == last - 1) { if (T.w > 0) shi = GV_INF; else slo = -GV_INF; }
    }
    double lo, hi;
    if (k == k0 && (sl & kSlOut)) {
      if (hold) { lo = -GV_INF; hi = GV_INF; } else continue;
    } else {
      cone_region(S.out[k], T, r2, radial, A0, bs0, r, lo, hi);
    }
    lo = dmax(dmax(lo, slo), plo);
    hi = dmin(dmin(hi, shi), phi_hi);
    if (!(lo < hi)) continue;
    double ha = GV_INF, hb = -GV_INF;  // the hole
    if (inner_has(S, k)) {
      if (k == k0 && (sl & kSlIn)) {
        if (!hold) continue;  // on the inner wall: never in this section's interior
      } else {
        cone_region(S.in[k], T, r2, radial, A0, bs0, r, ha, hb);
      }
    }
    double a1[2], b1[2];
    const int m1 = minus(lo, hi, ha, hb, a1, b1);
    for (int j = 0; j < m1; j++) {
      double a2[2], b2[2];
      const int m2 = minus(a1[j], b1[j], xlo, xhi, a2, b2);
      for (int q = 0; q < m2; q++) P.push(a2[q], b2[q]);
    }
  }
}

__device__ __forceinline__ void prim_pieces(const Desc& S, const Track& T, bool hold, Pieces& P) {
  if (S.type == kBox || S.type == kTrd || S.type == kTrap) planar_pieces(S, T, hold, P);
  else pcon_pieces(S, T, hold, P);
}

__device__ __forceinline__ double prim_s(const Desc& S, double x, double y, double z) {
  if (S.type == kBox) return box_s(S, x, y, z);
  if (S.type == kTrd || S.type == kTrap) return planar_s(S, x, y, z);
  return pcon_s(S, x, y, z);
}

// The surface start of a primitive within its band: entering (every band constraint
// shrinks) and growing (some band constraint grows: the complement is entered).
struct Start { bool entering, growing; };
__device__ __forceinline__ void start_add(Start& st, double g, int m) {
  if (g >= -H) {
    if (m != -1) st.entering = false;
    if (m == 1) st.growing = true;
  }
}
__device__ inline Start prim_start(const Desc& S, const Track& T) {
  Start st{true, false};
  if (S.type == kBox) {
    const double p[3] = {T.x, T.y, T.z}, d[3] = {T.u, T.v, T.w};
    for (int i = 0; i < 3; i++) start_add(st, xsub(fabs(p[i]), S.D[i]), plane_motion(p[i] < 0 ? -d[i] : d[i]));
  } else if (S.type == kTrd || S.type == kTrap) {
    for (int i = 0; i < 4; i++) {
      const double* P = S.pl[i];
      start_add(st, xsub(xadd(xadd(xmul(P[0], T.x), xmul(P[1], T.y)), xmul(P[2], T.z)), P[3]),
                plane_motion(xadd(xadd(xmul(P[0], T.u), xmul(P[1], T.v)), xmul(P[2], T.w))));
    }
    start_add(st, xsub(fabs(T.z), S.dz), plane_motion(T.z < 0 ? -T.w : T.w));
  } else {
    const int last = S.nz - 1;
    const double r = __dsqrt_rn(xadd(xmul(T.x, T.x), xmul(T.y, T.y)));
    const int k0 = section_of(S, T.z);
    const double radial = xadd(xmul(T.x, T.u), xmul(T.y, T.v));
    const double go = g_out(S.out[k0], r, T.z);
    start_add(st, go, wall_motion_near(go, S.out[k0], T, r, radial, true));
    if (inner_has(S, k0)) {
      const double gi = g_in(S.in[k0], r, T.z);
      start_add(st, gi, wall_motion_near(gi, S.in[k0], T, r, radial, false));
    }
    start_add(st, xsub(S.z[0], T.z), plane_motion(-T.w));
    start_add(st, xsub(T.z, S.z[last]), plane_motion(T.w));
    if (S.flags & kHasPhi) {
      const Phi f = phi_eval(S, T.x, T.y);
      const int ms = plane_motion(xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v)));
      const int me = plane_motion(xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v)));
      if (S.flags & kPhiWide) { if (f.a <= f.b) start_add(st, f.a, ms); else start_add(st, f.b, me); }
      else { start_add(st, f.a, ms); start_add(st, f.b, me); }
    }
  }
  return st;
}

__device__ inline void prim_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  switch (S.type) {
    case kBox: box_query(S, T, want, R); break;
    case kTrd:
    case kTrap: planar_query(S, T, want, R); break;
    default: pcon_query(S, T, want, R); break;
  }
}

static __device__ __noinline__ void bool_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  const Desc& A = S.parts[0];
  const Desc& C = S.parts[1];
  Track Tc;  // c's frame: p_c = R^T (p - t), d_c = R^T d
  {
    const double v0 = xsub(T.x, S.bt[0]), v1 = xsub(T.y, S.bt[1]), v2 = xsub(T.z, S.bt[2]);
    const double* M = S.bR;
    Tc.x = xadd(xadd(xmul(M[0], v0), xmul(M[3], v1)), xmul(M[6], v2));
    Tc.y = xadd(xadd(xmul(M[1], v0), xmul(M[4], v1)), xmul(M[7], v2));
    Tc.z = xadd(xadd(xmul(M[2], v0), xmul(M[5], v1)), xmul(M[8], v2));
    Tc.u = xadd(xadd(xmul(M[0], T.u), xmul(M[3], T.v)), xmul(M[6], T.w));
    Tc.v = xadd(xadd(xmul(M[1], T.u), xmul(M[4], T.v)), xmul(M[7], T.w));
    Tc.w = xadd(xadd(xmul(M[2], T.u), xmul(M[5], T.v)), xmul(M[8], T.w));
  }
  const int op = S.bop;
  const double sa = prim_s(A, T.x, T.y, T.z), sc = prim_s(C, Tc.x, Tc.y, Tc.z);
  const double s = op == kUnion ? dmin(sa, sc) : (op == kIntersection ? dmax(sa, sc) : dmax(sa, -sc));
  R.code = code_of(s);
  if (want & (kWantSin | kWantSout)) {
    Result ra, rc;
    prim_query(A, T, kWantCode | kWantSin | kWantSout, ra);
    prim_query(C, Tc, kWantCode | kWantSin | kWantSout, rc);
    double vin, vout;
    if (op == kUnion) {
      vin = dmin(ra.sin, rc.sin);
      vout = -GV_INF;
      if (ra.code == 0) vout = dmax(vout, ra.sout);
      if (rc.code == 0) vout = dmax(vout, rc.sout);
    } else if (op == kIntersection) {
      vout = dmin(ra.sout, rc.sout);
      vin = -GV_INF;
      if (ra.code == 2) vin = dmax(vin, ra.sin);
      if (rc.code == 2) vin = dmax(vin, rc.sin);
    } else {
      vout = dmin(ra.sout, rc.sin);
      vin = -GV_INF;
      if (ra.code == 2) vin = dmax(vin, ra.sin);
      if (rc.code == 0) vin = dmax(vin, rc.sout);
    }
    finish_safety(R.code, vin, vout, R);
  }
  if (!(want & (kWantDin | kWantDout))) return;
  // surface start from the components within the band: a union is entered when some band
  // component is, an intersection (and a subtraction, a and not-c) when every band component
  // is; not-c is entered where some band constraint of c grows
  bool entering = false;
  if (R.code == 1) {
    const bool ba = fabs(sa) <= H, bc = fabs(sc) <= H;
    bool ea = false, ec = false;
    if (ba) ea = prim_start(A, T).entering;
    if (bc) { const Start st = prim_start(C, Tc); ec = op == kSubtraction ? st.growing : st.entering; }
    if (op == kUnion) entering = (ba && ea) || (bc && ec);
    else entering = (!ba || ea) && (!bc || ec);
  }
  Pieces pa, pc, pr;
  prim_pieces(A, T, false, pa);
  prim_pieces(C, Tc, op == kSubtraction, pc);
  if (op == kUnion) {  // merge in order of start
    int i = 0, j = 0;
    while (i < pa.n || j < pc.n) {
      if (j >= pc.n || (i < pa.n && pa.a[i] <= pc.a[j])) { pr.push(pa.a[i], pa.b[i]); i++; }
      else { pr.push(pc.a[j], pc.b[j]); j++; }
    }
  } else if (op == kIntersection) {
    int i = 0, j = 0;
    while (i < pa.n && j < pc.n) {
      pr.push(dmax(pa.a[i], pc.a[j]), dmin(pa.b[i], pc.b[j]));
      if (pa.b[i] < pc.b[j]) i++; else j++;
    }
  } else {  // a minus every piece of c
    int j = 0;
    for (int i = 0; i < pa.n; i++) {
      double lo = pa.a[i];
      const double hi = pa.b[i];
      while (j < pc.n && pc.b[j] <= lo) j++;
      int q = j;
      while (q < pc.n && pc.a[q] < hi && lo < hi) {
        if (pc.a[q] > lo) pr.push(lo, pc.a[q]);
        lo = dmax(lo, pc.b[q]);
        q++;
      }
      pr.push(lo, hi);
    }
  }
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && !entering) R.dout = 0.0;
    else {
      double t = 0.0;  // a surface point whose ray never gets inside leaves at once
      for (int i = 0; i < pr.n; i++) {
        if (pr.b[i] <= 0) continue;
        t = pr.b[i];  // the piece holding 0+, else the first one after 0
        break;
      }
      R.dout = t;
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.0;
    else if (R.code == 1 && entering) R.din = 0.0;
    else {
      double t = GV_INF;
      for (int i = 0; i < pr.n; i++)
        if (pr.a[i] > 0) { t = pr.a[i]; break; }
      R.din = t;
    }
  }
  if (pa.over || pc.over || pr.over) R.din = R.dout = nan("");
}

__device__ __forceinline__ void query(const Desc& S, const Track& T, unsigned want, Result& R) {
  switch (S.type) {
    case kBox: box_query(S, T, want, R); break;
    case kTrd:
    case kTrap: planar_query(S, T, want, R); break;
    case kBool: bool_query(S, T, want, R); break;
    default: pcon_query(S, T, want, R); break;
  }
}

}  // namespace f64
}  // namespace gv
