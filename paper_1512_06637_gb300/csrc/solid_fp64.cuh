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
// A SURFACE point moving out (some constraint within the band grows along d),
// or whose ray never gets inside (checked halfway to the exit found), has
// DistanceToOut 0; one moving in (every such constraint shrinks) has
// DistanceToIn 0.  Decision quantities use __dadd_rn/__dmul_rn so that no
// multiply-add is fused into them.
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

// Surface motion over the constraints within the band: any growing -> leaving,
// all shrinking -> entering.
struct Motion {
  bool any_out = false, all_in = true;
  __device__ __forceinline__ void add(double g, double gd) {
    if (g >= -H) {
      if (gd > 0) any_out = true;
      if (!(gd < 0)) all_in = false;
    }
  }
};

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
__device__ inline double pcon_s(const Desc& S, double x, double y, double z);

// A surface point that is not leaving: the exit t found is meaningful only if the
// ray is inside (no tolerance) just before it; a ray that never gets inside (a
// tangent ray from a point a hair outside) leaves at once.  Checked at t / 2.
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
  for (int i = 0; i < 3; i++) m.add(g[i], p[i] < 0 ? -d[i] : d[i]);
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && m.any_out) R.dout = 0.0;
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
    else if (R.code == 1) R.din = m.all_in ? 0.0 : GV_INF;
    else {
      double tn = -GV_INF, tf = GV_INF;
      bool miss = false;
      for (int i = 0; i < 3; i++) {
        if (d[i] == 0) { if (g[i] > 0) miss = true; continue; }
        tn = dmax(tn, (-copysign(S.D[i], d[i]) - p[i]) / d[i]);
        tf = dmin(tf, (copysign(S.D[i], d[i]) - p[i]) / d[i]);
      }
      R.din = (!miss && tn < tf && tf > 0) ? tn : GV_INF;
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
  for (int i = 0; i < 5; i++) m.add(g[i], gd[i]);
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && m.any_out) R.dout = 0.0;
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
    else if (R.code == 1) R.din = m.all_in ? 0.0 : GV_INF;
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
      R.din = (!miss && tn < tf && tf > 0) ? tn : GV_INF;
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
// Strict phi membership of an entry point (open region: a touch is not an entry).
__device__ __forceinline__ bool phi_ok(const Desc& S, double x, double y) {
  if (!(S.flags & kHasPhi)) return true;
  const double a = S.ns[0] * x + S.ns[1] * y, b = S.ne[0] * x + S.ne[1] * y;
  return ((S.flags & kPhiWide) ? dmin(a, b) : dmax(a, b)) < 0;
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
// multiply-add) so that tangent rays are decided the same way everywhere.
struct Cross { double tm, tp; bool hm, hp; };
__device__ inline Cross line_cross(const Line& L, const Track& T, double r2, double radial,
                                   double A0) {
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
    if (disc > 0) {
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

// Strict membership (open region, no tolerance) of an entry point in the lateral
// constraints of section k: a ray that only touches the solid does not enter it.
__device__ __forceinline__ bool radial_ok(const Desc& S, int k, double r2, double z, bool skip_out,
                                          bool skip_in) {
  if (!skip_out) {
    const double R = S.out[k].a * z + S.out[k].b;
    if (!(R > 0 && r2 < R * R)) return false;
  }
  if (!skip_in && inner_has(S, k)) {
    const double R = S.in[k].a * z + S.in[k].b;
    if (R >= 0 && !(r2 > R * R)) return false;
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

__device__ inline void pcon_query(const Desc& S, const Track& T, unsigned want, Result& R) {
  const int nz = S.nz, last = nz - 1;
  const double r2 = xadd(xmul(T.x, T.x), xmul(T.y, T.y));
  const double r = __dsqrt_rn(r2);
  const int k0 = section_of(S, T.z);
  const bool has_phi = S.flags & kHasPhi;
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
  m.add(go, xsub(radial, xmul(xmul(S.out[k0].a, T.w), r)));
  if (inner_has(S, k0)) m.add(gi, -xsub(radial, xmul(xmul(S.in[k0].a, T.w), r)));
  m.add(gz0, -T.w);
  m.add(gz1, T.w);
  if (has_phi) {
    nds = xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v));
    nde = xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v));
    if (S.flags & kPhiWide) { if (f.a <= f.b) m.add(f.a, nds); else m.add(f.b, nde); }
    else { m.add(f.a, nds); m.add(f.b, nde); }
  }
  const double A0 = xadd(xmul(T.u, T.u), xmul(T.v, T.v));

  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.0;
    else if (R.code == 1 && m.any_out) R.dout = 0.0;
    else {
      // phi boundary
      double tphi = GV_INF;
      if (has_phi) {
        if (!(S.flags & kPhiWide)) {
          if (nds > 0) tphi = dmin(tphi, -f.a / nds);
          if (nde > 0) tphi = dmin(tphi, -f.b / nde);
        } else {  // leave the union of half-planes = enter the excluded wedge
          double tin = -GV_INF, tout = GV_INF;
          bool never = false;
          if (nds > 0) tin = dmax(tin, -f.a / nds);
          else if (nds < 0) tout = dmin(tout, -f.a / nds);
          else if (!(f.a > 0)) never = true;
          if (nde > 0) tin = dmax(tin, -f.b / nde);
          else if (nde < 0) tout = dmin(tout, -f.b / nde);
          else if (!(f.b > 0)) never = true;
          if (!never && tin < tout && tin > 0) tphi = tin;
        }
      }
      // walk the z-sections
      int k = k0;
      double tlo = 0, t = GV_INF;
      for (int guard = 0; guard < kMaxZ; guard++) {
        double tl = GV_INF;
        const Cross co = line_cross(S.out[k], T, r2, radial, A0);
        if (co.hp && co.tp > tlo) tl = co.tp;
        if (inner_has(S, k)) {
          const Cross ci = line_cross(S.in[k], T, r2, radial, A0);
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
      if (R.code == 1 && !inside_before(S, T, t, pcon_s)) t = 0.0;
      R.dout = t;
    }
  }

  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.0;
    else if (R.code == 1 && m.all_in) R.din = 0.0;
    else {
      double best = GV_INF;
      // lateral surfaces of every section the track can reach
      for (int k = 0; k < last; k++) {
        if (T.w > 0 && S.z[k + 1] < T.z) continue;
        if (T.w < 0 && S.z[k] > T.z) continue;
        if (T.w == 0 && (T.z < S.z[k] || T.z > S.z[k + 1])) continue;
        const Cross co = line_cross(S.out[k], T, r2, radial, A0);
        if (co.hm && co.tm > 0 && co.tm < best) {
          const double qx = T.x + co.tm * T.u, qy = T.y + co.tm * T.v, qz = T.z + co.tm * T.w;
          if (qz >= S.z[k] && qz <= S.z[k + 1] && qz > S.z[0] && qz < S.z[last] &&
              radial_ok(S, k, qx * qx + qy * qy, qz, true, false) && phi_ok(S, qx, qy))
            best = co.tm;
        }
        if (inner_has(S, k)) {
          const Cross ci = line_cross(S.in[k], T, r2, radial, A0);
          if (ci.hp && ci.tp > 0 && ci.tp < best) {
            const double qx = T.x + ci.tp * T.u, qy = T.y + ci.tp * T.v, qz = T.z + ci.tp * T.w;
            if (qz >= S.z[k] && qz <= S.z[k + 1] && qz > S.z[0] && qz < S.z[last] &&
                radial_ok(S, k, qx * qx + qy * qy, qz, false, true) && phi_ok(S, qx, qy))
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
          if (radial_ok(S, kk, qx * qx + qy * qy, ze, false, false) && phi_ok(S, qx, qy)) best = t;
        }
      }
      // phi planes
      if (has_phi) {
        for (int j = 0; j < 2; j++) {
          const double a = j == 0 ? f.a : f.b, nd = j == 0 ? nds : nde;
          if (!(nd < 0)) continue;
          const double t = -a / nd;
          if (!(t > 0 && t < best)) continue;
          const double qx = T.x + t * T.u, qy = T.y + t * T.v, qz = T.z + t * T.w;
          if (!(qz > S.z[0] && qz < S.z[last])) continue;
          const int kq = section_of(S, qz);
          if (!radial_ok(S, kq, qx * qx + qy * qy, qz, false, false)) continue;
          if (!(S.flags & kPhiWide)) {
            const double* n2 = j == 0 ? S.ne : S.ns;
            if (!(n2[0] * qx + n2[1] * qy < 0)) continue;
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

constexpr int kMaxPieces = 96;
struct Pieces {
  int n = 0;
  bool over = false;
  double a[kMaxPieces], b[kMaxPieces];
  // pieces arrive in increasing t; a piece touching or overlapping the last is merged
  __device__ __forceinline__ void push(double lo, double hi) {
    if (!(lo < hi)) return;
    if (n > 0 && lo <= b[n - 1]) {
      if (hi > b[n - 1]) b[n - 1] = hi;
      return;
    }
    if (n < kMaxPieces) { a[n] = lo; b[n] = hi; n++; } else over = true;
  }
};

// constraint g + t gd <= 0 along the ray: clip [lo, hi]
__device__ __forceinline__ void clip_le(double g, double gd, double& lo, double& hi) {
  if (gd == 0) { if (g > 0) { lo = GV_INF; hi = -GV_INF; } return; }
  const double t = -g / gd;
  if (gd > 0) hi = dmin(hi, t); else lo = dmax(lo, t);
}

__device__ inline void planar_pieces(const Desc& S, const Track& T, Pieces& P) {
  double lo = -GV_INF, hi = GV_INF;
  if (S.type == kBox) {
    const double p[3] = {T.x, T.y, T.z}, d[3] = {T.u, T.v, T.w};
    for (int i = 0; i < 3; i++) {
      clip_le(xsub(p[i], S.D[i]), d[i], lo, hi);            //  x - D <= 0
      clip_le(xsub(-p[i], S.D[i]), -d[i], lo, hi);          // -x - D <= 0
    }
  } else {
    for (int i = 0; i < 4; i++) {
      const double* Q = S.pl[i];
      clip_le(xsub(xadd(xadd(xmul(Q[0], T.x), xmul(Q[1], T.y)), xmul(Q[2], T.z)), Q[3]),
              xadd(xadd(xmul(Q[0], T.u), xmul(Q[1], T.v)), xmul(Q[2], T.w)), lo, hi);
    }
    clip_le(xsub(T.z, S.dz), T.w, lo, hi);
    clip_le(xsub(-T.z, S.dz), -T.w, lo, hi);
  }
  P.push(lo, hi);
}

// the region r <= a z + b (one nappe) of a section line along the ray
__device__ __forceinline__ void cone_region(const Line& L, const Track& T, double r2, double radial, double A0,
                                            double r, double& lo, double& hi) {
  const Cross c = line_cross(L, T, r2, radial, A0);
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

__device__ inline void pcon_pieces(const Desc& S, const Track& T, Pieces& P) {
  const int last = S.nz - 1;
  const double r2 = xadd(xmul(T.x, T.x), xmul(T.y, T.y));
  const double r = __dsqrt_rn(r2);
  const double radial = xadd(xmul(T.x, T.u), xmul(T.y, T.v));
  const double A0 = xadd(xmul(T.u, T.u), xmul(T.v, T.v));
  double plo = -GV_INF, phi_hi = GV_INF, xlo = GV_INF, xhi = -GV_INF;  // narrow phi; wide-phi wedge
  if (S.flags & kHasPhi) {
    const Phi f = phi_eval(S, T.x, T.y);
    const double nds = xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v));
    const double nde = xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v));
    if (!(S.flags & kPhiWide)) {
      clip_le(f.a, nds, plo, phi_hi);
      clip_le(f.b, nde, plo, phi_hi);
    } else {  // the wedge n_s.p > 0 and n_e.p > 0
      xlo = -GV_INF; xhi = GV_INF;
      clip_le(-f.a, -nds, xlo, xhi);
      clip_le(-f.b, -nde, xlo, xhi);
    }
  }
  const int kb = T.w < 0 ? last - 1 : 0, step = T.w < 0 ? -1 : 1;
  for (int i = 0; i < last; i++) {
    const int k = kb + step * i;
    double slo, shi;
    if (T.w > 0) { slo = (S.z[k] - T.z) / T.w; shi = (S.z[k + 1] - T.z) / T.w; }
    else if (T.w < 0) { slo = (S.z[k + 1] - T.z) / T.w; shi = (S.z[k] - T.z) / T.w; }
    else if (T.z >= S.z[k] && T.z <= S.z[k + 1]) { slo = -GV_INF; shi = GV_INF; }
    else continue;
    double lo, hi;
    cone_region(S.out[k], T, r2, radial, A0, r, lo, hi);
    lo = dmax(dmax(lo, slo), plo);
    hi = dmin(dmin(hi, shi), phi_hi);
    if (!(lo < hi)) continue;
    double ha = GV_INF, hb = -GV_INF;  // the hole
    if (inner_has(S, k)) cone_region(S.in[k], T, r2, radial, A0, r, ha, hb);
    double a1[2], b1[2];
    const int m1 = minus(lo, hi, ha, hb, a1, b1);
    for (int j = 0; j < m1; j++) {
      double a2[2], b2[2];
      const int m2 = minus(a1[j], b1[j], xlo, xhi, a2, b2);
      for (int q = 0; q < m2; q++) P.push(a2[q], b2[q]);
    }
  }
}

__device__ __forceinline__ void prim_pieces(const Desc& S, const Track& T, Pieces& P) {
  if (S.type == kBox || S.type == kTrd || S.type == kTrap) planar_pieces(S, T, P);
  else pcon_pieces(S, T, P);
}

__device__ __forceinline__ double prim_s(const Desc& S, double x, double y, double z) {
  if (S.type == kBox) return box_s(S, x, y, z);
  if (S.type == kTrd || S.type == kTrap) return planar_s(S, x, y, z);
  return pcon_s(S, x, y, z);
}

// The surface motion of a primitive at its band (the rule its own query applies).
__device__ inline Motion prim_motion(const Desc& S, const Track& T) {
  Motion m;
  if (S.type == kBox) {
    const double p[3] = {T.x, T.y, T.z}, d[3] = {T.u, T.v, T.w};
    for (int i = 0; i < 3; i++) m.add(xsub(fabs(p[i]), S.D[i]), p[i] < 0 ? -d[i] : d[i]);
  } else if (S.type == kTrd || S.type == kTrap) {
    for (int i = 0; i < 4; i++) {
      const double* P = S.pl[i];
      m.add(xsub(xadd(xadd(xmul(P[0], T.x), xmul(P[1], T.y)), xmul(P[2], T.z)), P[3]),
            xadd(xadd(xmul(P[0], T.u), xmul(P[1], T.v)), xmul(P[2], T.w)));
    }
    m.add(xsub(fabs(T.z), S.dz), T.z < 0 ? -T.w : T.w);
  } else {
    const int last = S.nz - 1;
    const double r = __dsqrt_rn(xadd(xmul(T.x, T.x), xmul(T.y, T.y)));
    const int k0 = section_of(S, T.z);
    const double radial = xadd(xmul(T.x, T.u), xmul(T.y, T.v));
    m.add(g_out(S.out[k0], r, T.z), xsub(radial, xmul(xmul(S.out[k0].a, T.w), r)));
    if (inner_has(S, k0)) m.add(g_in(S.in[k0], r, T.z), -xsub(radial, xmul(xmul(S.in[k0].a, T.w), r)));
    m.add(xsub(S.z[0], T.z), -T.w);
    m.add(xsub(T.z, S.z[last]), T.w);
    if (S.flags & kHasPhi) {
      const Phi f = phi_eval(S, T.x, T.y);
      const double nds = xadd(xmul(S.ns[0], T.u), xmul(S.ns[1], T.v));
      const double nde = xadd(xmul(S.ne[0], T.u), xmul(S.ne[1], T.v));
      if (S.flags & kPhiWide) { if (f.a <= f.b) m.add(f.a, nds); else m.add(f.b, nde); }
      else { m.add(f.a, nds); m.add(f.b, nde); }
    }
  }
  return m;
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
  // surface motion from the components within the band
  bool entering = false, leaving = false;
  if (R.code == 1) {
    const bool ba = fabs(sa) <= H, bc = fabs(sc) <= H;
    bool la = false, ea = false, lc = false, ec = false;
    if (ba) { const Motion m = prim_motion(A, T); la = m.any_out; ea = m.all_in; }
    if (bc) { const Motion m = prim_motion(C, Tc); lc = m.any_out; ec = m.all_in; }
    if (op == kSubtraction) { const bool tmp = lc; lc = ec; ec = tmp; }
    if (op == kUnion) {
      entering = (ba && ea) || (bc && ec);
      leaving = (!ba || la) && (!bc || lc);
    } else {
      entering = (!ba || ea) && (!bc || ec);
      leaving = (ba && la) || (bc && lc);
    }
  }
  Pieces pa, pc, pr;
  prim_pieces(A, T, pa);
  prim_pieces(C, Tc, pc);
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
    else if (R.code == 1 && leaving) R.dout = 0.0;
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
