// solid_fp32.cuh -- binary32 bulk evaluation of the five queries with certified
// error bounds; every track whose answer cannot be certified is flagged for the
// binary64 pass.
//
// Arithmetic model.  Each input coordinate (binary64 in memory) is split with
// integer operations only into hi = the double truncated to 24 significant
// bits and lo = the next 23 bits, so x = hi + lo to 2^-46 relative; directions
// keep only hi.  The decision quantities (the constraint values whose maximum
// decides inside / surface / outside, see gv_desc.h) are formed in double-float
// arithmetic (exact products by fmaf, exact sums by two-sum), which gives them
// to about 2^-44 of the coordinates' magnitude.  A code is certified when s is
// farther than its error bound E from both band edges -h and +h; E also covers
// the rounding of the binary64 evaluation it has to agree with.  Distances are
// formed in plain binary32 from those accurate constraint values (so a short
// distance from a near-surface point keeps its relative accuracy) and carry an
// absolute error bound through every operation; a result is certified when its
// bound is below half the stated tolerance (1e-5 relative; 1e-9 mm below 1e-4 mm).
// Near ties (a ray grazing an edge, a tangent root, an entry point on another
// surface) are flagged, as are the surface-start cases of the polycone family
// that need the full set of rules.  So is every track that the binary64 rules for
// grazing rays could decide: a constraint within reach of the band whose derivative
// along d is within reach of the tangent threshold (a ray along or tangent to a
// surface), and two crossings within reach of the merge distance.  No binary64
// instruction is used here.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>
#include "gv_desc.h"

namespace gv {
namespace f32 {

constexpr float U = 5.9604645e-8f;      // 2^-24
constexpr float G42 = 2.2737368e-13f;   // 2^-42
constexpr float HF = 5e-10f;            // h
constexpr float FLOOR = 1e-15f;         // absolute floor of every decision bound
constexpr float TAUF = 2.5e-12f;        // > kTangent: derivatives per unit length this small are flagged
constexpr float MERGEF = 2.5e-12f;      // > kMerge: crossings this close are not told apart
#define F_INF CUDART_INF_F

enum : unsigned { kWantCode = 1, kWantDin = 2, kWantDout = 4, kWantSin = 8, kWantSout = 16 };

struct TrackF {
  float xh, yh, zh, xl, yl, zl;  // point: hi + lo
  float u, v, w;                 // direction: hi
  float ul, vl, wl;              // direction: lo
  long long zkey;                // order key of z (query kernels; keyed = true)
  float fl;                      // absolute error of each point coordinate beyond 2^-46 |x|
  float dfl;                     // absolute error of each direction component (frame tracks)
  bool keyed;                    // zkey holds the binary64 z (false after a frame change)
  bool bad;                      // outside the binary32 range: binary64 only
};

struct R32 {
  int code;
  float din, dout, sin, sout;
  bool flag;
};

struct Val {  // value with an absolute error bound
  float v, e;
};

// "No value" sentinel for interval min/max: finite, so that v - e never forms inf - inf.
constexpr float BIG = 1e37f;
__device__ __forceinline__ float unbig(float v) { return v >= BIG ? F_INF : v; }

__device__ __forceinline__ Val vmin(Val a, Val b) {
  const float v = fminf(a.v, b.v);
  if (isinf(v)) return {v, 0.f};
  const float lo = fminf(a.v - a.e, b.v - b.e), hi = fminf(a.v + a.e, b.v + b.e);
  return {v, fmaxf(v - lo, hi - v)};
}
__device__ __forceinline__ Val vmax(Val a, Val b) {
  const float v = fmaxf(a.v, b.v);
  if (isinf(v)) return {v, 0.f};
  const float lo = fmaxf(a.v - a.e, b.v - b.e), hi = fmaxf(a.v + a.e, b.v + b.e);
  return {v, fmaxf(v - lo, hi - v)};
}
// Certified against the output tolerance (half of it, for margin).
__device__ __forceinline__ bool certified(Val t) {
  if (isinf(t.v) || t.v >= BIG) return true;
  const float tol = t.v < 1e-4f ? 1e-9f : 1e-5f * t.v;
  return t.e <= 0.5f * tol;
}
// a < b decided with certainty (and farther apart than the merge distance)?
__device__ __forceinline__ bool apart(Val a, Val b) { return fabsf(a.v - b.v) > (a.e + b.e) + MERGEF; }

// ------------------------------------------------------------ conversions

// Split a binary64 (as its two 32-bit words) into binary32 hi + lo.
__device__ __forceinline__ void split(uint2 b, float& h, float& l, bool& bad) {
  const uint32_t hi = b.y, lo = b.x;
  const uint32_t e = (hi >> 20) & 0x7FFu, sg = hi & 0x80000000u;
  const uint32_t hb = sg | ((((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29));
  h = __uint_as_float(e >= 897u ? hb : sg);
  const uint32_t M = (lo & 0x1FFFFFFFu) >> 6;
  const uint32_t one = (e - 919u) << 23;
  float v = __uint_as_float(one | M) - __uint_as_float(one);
  v = __uint_as_float(__float_as_uint(v) | sg);
  l = (e >= 920u) ? v : 0.0f;
  bad |= e >= 1151u;
}
// hi part only; a nonzero magnitude below 2^-126 is left to binary64.
__device__ __forceinline__ float trunc_hi(uint2 b, bool& bad) {
  const uint32_t hi = b.y, lo = b.x;
  const uint32_t e = (hi >> 20) & 0x7FFu, sg = hi & 0x80000000u;
  const uint32_t hb = sg | ((((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29));
  bad |= e >= 1151u || (e < 897u && ((hi & 0x7FFFFFFFu) | lo) != 0u);
  return __uint_as_float(e >= 897u ? hb : sg);
}
// Exact binary32 -> binary64 bit pattern.  The conversion instruction runs on the FP64
// pipe, which the binary32 pass otherwise leaves idle, and so frees the integer pipe that
// the input split keeps busy (measured faster than assembling the bits with integer ops).
__device__ __forceinline__ unsigned long long f2d_bits(float f) {
  return (unsigned long long)__double_as_longlong((double)f);
}

// A track from the raw binary64 words of its point and direction.
template <bool DIR_LO = true>
__device__ __forceinline__ TrackF track_from_words(uint2 bx, uint2 by, uint2 bz, uint2 bu, uint2 bv, uint2 bw,
                                                   bool dirs) {
  TrackF T;
  T.bad = false;
  T.fl = FLOOR;
  T.dfl = 0.f;
  T.keyed = true;
  split(bx, T.xh, T.xl, T.bad);
  split(by, T.yh, T.yl, T.bad);
  split(bz, T.zh, T.zl, T.bad);
  T.zkey = order_key((long long)(((unsigned long long)bz.y << 32) | bz.x));
  if (dirs) {
    T.u = trunc_hi(bu, T.bad);
    T.v = trunc_hi(bv, T.bad);
    T.w = trunc_hi(bw, T.bad);
    if (DIR_LO) {
      bool unused = false;
      float h;
      split(bu, h, T.ul, unused);
      split(bv, h, T.vl, unused);
      split(bw, h, T.wl, unused);
    } else {
      T.ul = T.vl = T.wl = 0.f;
    }
  } else {
    T.u = T.v = T.w = 0.f;
    T.ul = T.vl = T.wl = 0.f;
  }
  return T;
}

template <bool DIR_LO = true>
__device__ __forceinline__ TrackF load_track(const uint2* x, const uint2* y, const uint2* z,
                                             const uint2* u, const uint2* v, const uint2* w,
                                             int64_t i, bool dirs) {
  const uint2 zero{0u, 0u};
  return track_from_words<DIR_LO>(__ldg(x + i), __ldg(y + i), __ldg(z + i), dirs ? __ldg(u + i) : zero,
                                  dirs ? __ldg(v + i) : zero, dirs ? __ldg(w + i) : zero, dirs);
}

// ------------------------------------------------- double-float pieces

struct F2 { float h, l; };
__device__ __forceinline__ F2 tprod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ F2 tsum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// The exact s = max_i g_i lies in [lo, hi] = [max_i (g_i - E_i), max_i (g_i + E_i)];
// a code is certified when that interval sits inside one of the three regions.
struct SInt {
  float s, lo, hi;
  __device__ __forceinline__ void add(float g, float E) {
    s = fmaxf(s, g);
    lo = fmaxf(lo, g - E);
    hi = fmaxf(hi, g + E);
  }
  __device__ __forceinline__ void add_int(float g, float glo, float ghi) {
    s = fmaxf(s, g);
    lo = fmaxf(lo, glo);
    hi = fmaxf(hi, ghi);
  }
  __device__ __forceinline__ float err() const { return fmaxf(s - lo, hi - s); }
};
__device__ __forceinline__ SInt sint() { return {-F_INF, -F_INF, -F_INF}; }
__device__ __forceinline__ int decide(const SInt& S, bool& flag) {
  if (S.lo > HF) return 2;
  if (S.hi < -HF) return 0;
  if (S.lo >= -HF && S.hi <= HF) return 1;
  flag = true;
  return 1;
}

// Constraint value with its bound.
struct Gv { float g, E; };

// |p| - D from split values (the low part may have either sign: |p| = |ph| + sign(ph) pl)
__device__ __forceinline__ Gv abs_minus(float ph, float pl, float Dh, float Dl, float fl) {
  const float a = fabsf(ph);
  const float g = (a - Dh) + ((ph < 0 ? -pl : pl) - Dl);
  return {g, fmaf(4.f * U, fabsf(g), fmaf(G42, a + Dh, fl))};
}
// (n.p - c) with n, c split, p split
__device__ __forceinline__ Gv plane_g(const float* nh, const float* nl, float ch, float cl,
                                      const TrackF& T) {
  const F2 p0 = tprod(nh[0], T.xh), p1 = tprod(nh[1], T.yh), p2 = tprod(nh[2], T.zh);
  const F2 s1 = tsum(p0.h, p1.h), s2 = tsum(s1.h, p2.h), s3 = tsum(s2.h, -ch);
  float lo = ((s1.l + s2.l) + s3.l) + ((p0.l + p1.l) + p2.l);
  lo = fmaf(nh[0], T.xl, fmaf(nl[0], T.xh, lo));
  lo = fmaf(nh[1], T.yl, fmaf(nl[1], T.yh, lo));
  lo = fmaf(nh[2], T.zl, fmaf(nl[2], T.zh, lo));
  lo -= cl;
  const float g = s3.h + lo;
  return {g, fmaf(4.f * U, fabsf(g), fmaf(G42, fabsf(T.xh) + fabsf(T.yh) + fabsf(T.zh) + fabsf(ch), 2.f * T.fl))};
}

// ------------------------------------------------------------------- box

// Both distances from one set of slab times, so that inside and outside tracks run
// the same instructions: per axis the crossings are a = (|p| - D)/|d| (accurate,
// the face on the point's side) and b = (D + |p|)/|d| (the far face); moving toward
// the near face the slab is entered at -b and left at -a, otherwise entered at a
// and left at b.  DistanceToOut = min exit, DistanceToIn = max entry when it comes
// before the min exit.
template <bool FRAME = false>
__device__ inline void box32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
  const float ph[3] = {T.xh, T.yh, T.zh}, pl[3] = {T.xl, T.yl, T.zl}, d[3] = {T.u, T.v, T.w};
  Gv g[3];
  SInt si = sint();
  for (int i = 0; i < 3; i++) {
    g[i] = abs_minus(ph[i], pl[i], S.Dh[i], S.Dl[i], T.fl);
    si.add(g[i].g, g[i].E);
  }
  const float s = si.s;
  R.code = decide(si, R.flag);
  R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
  R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
  if (R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
  if (!(want & (kWantDin | kWantDout))) return;
  Val tn{-BIG, 0.f}, tf{BIG, 0.f};
  bool miss = false, any_out = false, all_in = true;
  for (int i = 0; i < 3; i++) {
    const bool toward = (ph[i] < 0) == (d[i] < 0);  // toward the face on the point's side
    if (FRAME && fabsf(d[i]) <= 4.f * T.dfl) R.flag = true;  // sign of d not certain
    if (d[i] == 0) {
      if (fabsf(g[i].g) <= g[i].E) R.flag = true;
      miss |= g[i].g > 0;
    } else {
      const float inv = __frcp_rn(fabsf(d[i]));
      const float a = g[i].g * inv, b = (S.Dh[i] + fabsf(ph[i])) * inv;
      Val A{a, fmaf(g[i].E, inv, 5.f * U * fabsf(a))}, B{b, 9.f * U * b};
      if (FRAME) {  // error of the direction component
        A.e = fmaf(1.01f * fabsf(a) * T.dfl, inv, A.e);
        B.e = fmaf(fmaf(1.01f * b, T.dfl, T.fl), inv, B.e);
      }
      tn = vmax(tn, toward ? Val{-B.v, B.e} : A);
      tf = vmin(tf, toward ? Val{-A.v, A.e} : B);
    }
    // surface start: constraints within the band
    if (g[i].g >= -HF) {
      const float gd = ph[i] < 0 ? -d[i] : d[i];
      any_out |= gd > 0;
      all_in &= gd < 0;
    }
    // along or nearly along the face plane: sliding is decided in binary64
    if (fabsf(d[i]) <= TAUF + (FRAME ? 4.f * T.dfl : 0.f) && fabsf(g[i].g) <= HF + g[i].E) R.flag = true;
    if (R.code == 1 && fabsf(g[i].g + HF) <= g[i].E) R.flag = true;
  }
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.f;
    else if (R.code == 1 && !all_in) R.dout = 0.f;
    else {
      if (!certified(tf)) R.flag = true;
      R.dout = unbig(tf.v);
      if (R.code == 1) {  // an entering surface point: inside (no tolerance) halfway to the exit?
        const float h = 0.5f * tf.v;
        float sm = -BIG, em = 0.f;
        for (int i = 0; i < 3; i++) {
          const float q = fmaf(h, d[i], ph[i]);
          sm = fmaxf(sm, fabsf(q) - S.Dh[i]);
          em = fmaxf(em, 4.f * U * (fabsf(q) + S.Dh[i]) + fabsf(d[i]) * 0.5f * tf.e +
                             (FRAME ? fmaf(h, T.dfl, 2.f * T.fl) : 0.f));
        }
        if (!(tf.v < BIG) || fabsf(sm) <= em + 1e-12f) R.flag = true;
        else if (sm > 0) R.dout = 0.f;
      }
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.f;
    else if (R.code == 1) R.din = all_in ? 0.f : F_INF;
    else if (miss) R.din = F_INF;
    else {
      if (!apart(tn, tf) || fabsf(tf.v) <= tf.e) R.flag = true;
      if (tn.v < tf.v && tf.v > 0) {
        if (!certified(tn)) R.flag = true;
        R.din = tn.v;
      } else R.din = F_INF;
    }
  }
}

// ------------------------------------------------------------ trd / trap

// One uniform path as for the box: every side plane gives one crossing
// t = -g / (n.d), an entry when n.d < 0 and an exit when n.d > 0; the z slab
// gives its two crossings like a box axis.
template <bool FRAME = false>
__device__ inline void planar32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
  Gv g[5];
  float gd[5], egd[5];
  for (int i = 0; i < 4; i++) {
    g[i] = plane_g(S.plh[i], S.pll[i], S.plh[i][3], S.pll[i][3], T);
    const float a = S.plh[i][0] * T.u, b = S.plh[i][1] * T.v, c = S.plh[i][2] * T.w;
    gd[i] = (a + b) + c;
    egd[i] = 8.f * U * (fabsf(a) + fabsf(b) + fabsf(c)) + (FRAME ? 2.f * T.dfl : 0.f) + 1e-30f;
  }
  g[4] = abs_minus(T.zh, T.zl, S.dzh, S.dzl, T.fl);
  gd[4] = T.zh < 0 ? -T.w : T.w;
  egd[4] = FRAME ? T.dfl : 0.f;
  SInt si = sint();
  for (int i = 0; i < 5; i++) si.add(g[i].g, g[i].E);
  const float s = si.s;
  R.code = decide(si, R.flag);
  R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
  R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
  if (R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
  if (!(want & (kWantDin | kWantDout))) return;
  Val tn{-BIG, 0.f}, tf{BIG, 0.f};
  bool miss = false, any_out = false, all_in = true;
  for (int i = 0; i < 4; i++) {
    // along or nearly along the face plane: sliding is decided in binary64
    if (fabsf(gd[i]) <= egd[i] + TAUF && fabsf(g[i].g) <= HF + g[i].E) R.flag = true;
    if (fabsf(gd[i]) <= egd[i]) {  // nearly parallel: which side it stays on must be certain
      if (fabsf(g[i].g) <= g[i].E || R.code == 1) R.flag = true;
      miss |= g[i].g > 0;
      continue;
    }
    const float igd = __frcp_rn(gd[i]);
    const float t = -g[i].g * igd;
    const Val tv{t, fmaf(fmaf(fabsf(t), egd[i], g[i].E), fabsf(igd), 5.f * U * fabsf(t))};
    const bool entry = gd[i] < 0;
    tn = vmax(tn, entry ? tv : Val{-BIG, 0.f});
    tf = vmin(tf, entry ? Val{BIG, 0.f} : tv);
  }
  {  // z slab
    const bool toward = (T.zh < 0) == (T.w < 0);
    if (fabsf(T.w) <= egd[4] + TAUF && fabsf(g[4].g) <= HF + g[4].E) R.flag = true;
    if (FRAME && fabsf(T.w) <= 4.f * T.dfl) R.flag = true;  // sign of w not certain
    if (T.w == 0) {
      if (fabsf(g[4].g) <= g[4].E) R.flag = true;
      miss |= g[4].g > 0;
    } else {
      const float iw = __frcp_rn(fabsf(T.w));
      const float a = g[4].g * iw, b = (S.dzh + fabsf(T.zh)) * iw;
      Val A{a, fmaf(g[4].E, iw, 5.f * U * fabsf(a))}, B{b, 9.f * U * b};
      if (FRAME) {
        A.e = fmaf(1.01f * fabsf(a) * T.dfl, iw, A.e);
        B.e = fmaf(fmaf(1.01f * b, T.dfl, T.fl), iw, B.e);
      }
      tn = vmax(tn, toward ? Val{-B.v, B.e} : A);
      tf = vmin(tf, toward ? Val{-A.v, A.e} : B);
    }
  }
  for (int i = 0; i < 5; i++) {
    if (g[i].g >= -HF) {
      any_out |= gd[i] > 0;
      all_in &= gd[i] < 0;
      if (R.code == 1 && fabsf(gd[i]) <= egd[i] + TAUF) R.flag = true;
    }
    if (R.code == 1 && fabsf(g[i].g + HF) <= g[i].E) R.flag = true;
  }
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.f;
    else if (R.code == 1 && !all_in) R.dout = 0.f;
    else {
      if (!certified(tf)) R.flag = true;
      R.dout = unbig(tf.v);
      if (R.code == 1) {  // an entering surface point: inside (no tolerance) halfway to the exit?
        const float h = 0.5f * tf.v;
        const float qx = fmaf(h, T.u, T.xh), qy = fmaf(h, T.v, T.yh), qz = fmaf(h, T.w, T.zh);
        float sm = fabsf(qz) - S.dzh, em = 4.f * U * (fabsf(qz) + S.dzh);
        for (int i = 0; i < 4; i++) {
          const float* P = S.plh[i];
          const float v = fmaf(P[2], qz, fmaf(P[1], qy, P[0] * qx)) - P[3];
          sm = fmaxf(sm, v);
          em = fmaxf(em, 8.f * U * (fabsf(qx) + fabsf(qy) + fabsf(qz) + fabsf(P[3])));
        }
        em += 0.5f * tf.e + (FRAME ? fmaf(tf.v, T.dfl, 2.f * T.fl) : 0.f) + 1e-12f;
        if (!(tf.v < BIG) || fabsf(sm) <= em) R.flag = true;
        else if (sm > 0) R.dout = 0.f;
      }
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.f;
    else if (R.code == 1) R.din = all_in ? 0.f : F_INF;
    else if (miss) R.din = F_INF;
    else {
      if (!apart(tn, tf) || fabsf(tf.v) <= tf.e) R.flag = true;
      if (tn.v < tf.v && tf.v > 0) {
        if (!certified(tn)) R.flag = true;
        R.din = tn.v;
      } else R.din = F_INF;
    }
  }
}

// ------------------------------------- polycone family (tube, cone, polycone)

struct Lat {   // a lateral constraint evaluated in double-float
  float g, E;  // g = (r - R) k  (outer) or (R - r) k (inner)
  float delta, eDelta;  // r - R and its bound
  float dh, dl;  // r - R in double-float
  float Rh, Rl;  // R = a z + b at the point, double-float
  float scale;   // magnitude of the terms of r - R
  float ed;      // bound of dh + dl
};

template <bool TUBE>
__device__ __forceinline__ Lat lateral(float ah, float al, float bh, float bl, float k, float rh,
                                       float rl, const TrackF& T, bool outer) {
  float Rh, Rl, scale;
  if (TUBE) {
    Rh = bh; Rl = bl; scale = rh + fabsf(bh);
  } else {
    const F2 az = tprod(ah, T.zh);
    const F2 ts = tsum(az.h, bh);
    Rh = ts.h;
    Rl = ((ts.l + az.l) + fmaf(ah, T.zl, al * T.zh)) + bl;
    scale = rh + fabsf(az.h) + fabsf(bh);
  }
  const F2 dd = tsum(rh, -Rh);
  const float dl = dd.l + (rl - Rl);
  const float delta = dd.h + dl;
  // coordinate errors: r moves by up to 1.5 fl, a z + b by |a| fl
  const float ed = fmaf(G42, scale, (2.f + fabsf(ah)) * T.fl);
  const float eDelta = fmaf(4.f * U, fabsf(delta), ed);
  const float g = outer ? delta * k : -delta * k;
  return {g, fmaf(4.f * U, fabsf(g), eDelta * k), delta, eDelta, dd.h, dl, Rh, Rl, scale, ed};
}

// phi plane value n.p in double-float
__device__ __forceinline__ Gv phi_plane(const float* nh, const float* nl, const TrackF& T) {
  const F2 p0 = tprod(nh[0], T.xh), p1 = tprod(nh[1], T.yh);
  const F2 s1 = tsum(p0.h, p1.h);
  float lo = s1.l + (p0.l + p1.l);
  lo = fmaf(nh[0], T.xl, fmaf(nl[0], T.xh, lo));
  lo = fmaf(nh[1], T.yl, fmaf(nl[1], T.yh, lo));
  const float g = s1.h + lo;
  return {g, fmaf(4.f * U, fabsf(g), fmaf(G42, fabsf(T.xh) + fabsf(T.yh), 1.5f * T.fl))};
}

// Crossings of r = a z + b with the track: f(t) = A t^2 + 2 B t + C = r(t)^2 - R(t)^2,
// A = u^2 + v^2 - D^2, B = p.d_xy - P D, C = r^2 - P^2 (P = R at the point, D = a w).
// The discriminant B^2 - A C is formed in double-float from double-float A, B, C: a ray
// grazing a surface (B^2 close to A C) or nearly along a cone's slope keeps its roots
// to about 2^-42 of the terms; the roots themselves are then taken in binary32.
struct Quad {
  Val tm, tp;
  bool hm, hp;
  bool unsure;
};
// A0 = u^2 + v^2 in double-float from the split direction
__device__ __forceinline__ F2 a0_df(const TrackF& T) {
  const F2 uu = tprod(T.u, T.u), vv = tprod(T.v, T.v);
  const F2 s = tsum(uu.h, vv.h);
  const float lo = (s.l + (uu.l + vv.l)) + 2.f * fmaf(T.u, T.ul, T.v * T.vl);
  return {s.h + lo, lo - ((s.h + lo) - s.h)};
}
// p.d_xy = x u + y v in double-float from the split point and direction
__device__ __forceinline__ F2 radial_df(const TrackF& T) {
  const F2 p0 = tprod(T.xh, T.u), p1 = tprod(T.yh, T.v);
  const F2 s = tsum(p0.h, p1.h);
  const float lo = (s.l + (p0.l + p1.l)) + fmaf(T.xh, T.ul, fmaf(T.xl, T.u, fmaf(T.yh, T.vl, T.yl * T.v)));
  return {s.h + lo, lo - ((s.h + lo) - s.h)};
}
__device__ __forceinline__ F2 df_norm(float h, float l) {
  const float s = h + l;
  return {s, l - (s - h)};
}

template <bool TUBE, bool FRAME>
__device__ inline Quad quad32(float a, float al, const Lat& L, const TrackF& T, F2 rad, float erad, F2 A0,
                              float rh, float rl) {
  Quad q;
  q.hm = q.hp = false;
  q.unsure = false;
  q.tm = q.tp = {0.f, 0.f};
  // D = a w, P D, B = rad - P D, A = A0 - D^2, C = (r - P)(r + P): all double-float
  F2 Bd, Ad, D{0.f, 0.f};
  float eB, eA;
  if (TUBE) {
    Bd = rad;
    Ad = A0;
    eB = erad;
    eA = G42 * A0.h + 1e-30f;
    if (FRAME) eA = fmaf(2.02f * T.dfl, fabsf(T.u) + fabsf(T.v), eA);
  } else {
    const F2 dd = tprod(a, T.w);
    D = df_norm(dd.h, dd.l + fmaf(a, T.wl, al * T.w));
    const F2 pd = tprod(L.Rh, D.h);
    const float pdl = pd.l + fmaf(L.Rh, D.l, L.Rl * D.h);
    const F2 bs = tsum(rad.h, -pd.h);
    Bd = df_norm(bs.h, bs.l + (rad.l - pdl));
    const F2 d2 = tprod(D.h, D.h);
    const F2 as = tsum(A0.h, -d2.h);
    Ad = df_norm(as.h, as.l + (A0.l - fmaf(2.f * D.h, D.l, d2.l)));
    eB = fmaf(2.f * G42 * fabsf(D.h), L.scale + fabsf(L.Rh), erad);
    eA = fmaf(G42, A0.h + d2.h, 1e-30f);
    if (FRAME) {  // direction errors: A0 by 2 (|u| + |v|) dfl, D by |a| dfl
      const float eDd = 1.01f * fabsf(a) * T.dfl;
      eB = fmaf(fabsf(L.Rh) + L.ed, eDd, fmaf(fabsf(D.h), fabsf(a) * T.fl, eB));
      eA = fmaf(2.02f * T.dfl, fabsf(T.u) + fabsf(T.v), fmaf(2.f * fabsf(D.h) + eDd, eDd, eA));
    }
  }
  const F2 ps = tsum(rh, L.Rh);
  const F2 Sd = df_norm(ps.h, ps.l + (rl + L.Rl));  // r + P
  const F2 cp = tprod(L.dh, Sd.h);
  const F2 Cd = df_norm(cp.h, cp.l + fmaf(L.dh, Sd.l, L.dl * Sd.h));
  const float eC = fmaf(L.ed, fmaf(2.f, Sd.h, fabsf(L.dh)) + L.ed, 1e-30f);
  const float A = Ad.h, B = Bd.h, C = Cd.h;
  if (A == 0.f && D.h == 0.f && A0.h == 0.f) return q;  // parallel to the axis of a cylinder: no crossing
  const F2 b2 = tprod(Bd.h, Bd.h);
  const F2 ac = tprod(Ad.h, Cd.h);
  const F2 ds = tsum(b2.h, -ac.h);
  const float disc = ds.h + (ds.l + (fmaf(2.f * Bd.h, Bd.l, b2.l) - (ac.l + fmaf(Ad.h, Cd.l, Ad.l * Cd.h))));
  const float eD = fmaf(2.f * fabsf(B), eB, fmaf(fabsf(A), eC, fmaf(fabsf(C), eA, fmaf(eB, eB,
                   fmaf(4.f * U * U, b2.h + fabsf(ac.h), fmaf(2.f * U, fabsf(disc), 1e-30f))))));
  if (disc < -eD) return q;
  if (disc <= eD) { q.unsure = true; return q; }
  const float eB1 = fmaf(U, fabsf(B), eB), eA1 = fmaf(U, fabsf(A), eA), eC1 = fmaf(U, fabsf(C), eC);
  const float rs = rsqrtf(disc);
  const float sq = disc * rs;
  const float esq = fmaf(0.5f * 1.001f * eD, rs, 4.f * U * sq);
  float qq;  // r1 = qq / A, r2 = C / qq
  bool r1_is_plus;
  if (B >= 0) { qq = -(B + sq); r1_is_plus = false; }
  else { qq = sq - B; r1_is_plus = true; }
  const float eq = fmaf(U, fabsf(qq), eB1 + esq);
  const float iA = __frcp_rn(A), iq = __frcp_rn(qq);
  const float r1 = qq * iA;
  const float r2 = C * iq;
  const float relq = eq * fabsf(iq);
  const float rel1 = (fabsf(A) <= eA1) ? F_INF : fmaf(eA1, fabsf(iA), relq + 4.f * U);
  const Val v1{r1, fabsf(r1) * rel1};
  const Val v2{r2, fmaf(fabsf(C), relq + 4.f * U, eC1) * fabsf(iq)};
  const Val vp = r1_is_plus ? v1 : v2, vm = r1_is_plus ? v2 : v1;
  q.tp = vp; q.tm = vm; q.hp = q.hm = true;
  if (!TUBE) {  // keep roots on the nappe a z + b >= 0
    const float P = L.Rh, Dv = D.h;
    for (int j = 0; j < 2; j++) {
      const Val t = j ? q.tp : q.tm;
      const float Rt = fmaf(t.v, Dv, P);
      const float eR = fmaf(4.f * U, fabsf(P) + fabsf(t.v * Dv), fmaf(fabsf(Dv), t.e, fmaf(G42, L.scale, 1e-30f)));
      if (fabsf(Rt) <= eR && isfinite(t.v)) q.unsure = true;
      if (!(Rt >= 0)) { if (j) q.hp = false; else q.hm = false; }
    }
  }
  return q;
}

// ----- interval form of the single-section solids (tube, cone) -----
// Along the track each constraint holds on an interval (convex regions) whose ends
// are its crossings; the solid is C minus X1 minus X2 where C is the intersection
// of the convex constraints (outer surface, z slab, narrow phi) and X1, X2 the
// excluded convex regions (the hole inside rmin, the wedge cut out by a wide phi).
struct Iv {
  Val lo, hi;
  bool empty;
};
__device__ __forceinline__ Iv iv_all() { return {{-BIG, 0.f}, {BIG, 0.f}, false}; }
__device__ __forceinline__ Iv iv_none() { return {{BIG, 0.f}, {-BIG, 0.f}, true}; }
// Interval of a convex cone region from its crossings; no crossing: the whole line or
// nothing, as at the start point (inside if g < 0; |g| within its bound is uncertain).
__device__ __forceinline__ Iv iv_region(const Quad& q, float g, float Eg, bool& unsure) {
  if (q.hm || q.hp) return {q.hm ? q.tm : Val{-BIG, 0.f}, q.hp ? q.tp : Val{BIG, 0.f}, false};
  if (fabsf(g) <= Eg) unsure = true;
  return g < 0 ? iv_all() : iv_none();
}
// Half-space {n.p <= 0} (want_le) or {n.p > 0} crossed at t = -a / nd.
__device__ __forceinline__ Iv iv_half(float a, float Ea, float nd, float end, bool want_le, bool& unsure) {
  if (fabsf(nd) <= end + TAUF && fabsf(a) <= HF + Ea) unsure = true;  // along the plane: binary64
  if (fabsf(nd) <= end) {
    if (fabsf(a) <= Ea) unsure = true;
    return ((a <= 0) == want_le) ? iv_all() : iv_none();
  }
  const float ind = __frcp_rn(nd);
  const float t = -a * ind;
  const Val tv{t, fmaf(fmaf(fabsf(t), end, Ea), fabsf(ind), 5.f * U * fabsf(t))};
  // moving with nd > 0 the value n.p grows: {n.p <= 0} is before t, {n.p > 0} after
  const bool before = (nd > 0) == want_le;
  return before ? Iv{{-BIG, 0.f}, tv, false} : Iv{tv, {BIG, 0.f}, false};
}
__device__ __forceinline__ Iv iv_and(const Iv& x, const Iv& y) {
  if (x.empty || y.empty) return iv_none();
  return {vmax(x.lo, y.lo), vmin(x.hi, y.hi), false};
}
// -1: a < b certainly, +1: a > b certainly, 0: too close to tell
__device__ __forceinline__ int side(Val a, Val b) { return apart(a, b) ? (a.v < b.v ? -1 : 1) : 0; }
// a crossing certainly after 0; one that is not is at 0+ or before it
__device__ __forceinline__ bool after0(Val a) { return a.v > a.e; }
// side(t, b) and side(b, t) where t means "just after" a crossing: 0+ (z), or the crossing
// equal to t itself, count as passed
__device__ __forceinline__ int side_tb(Val t, bool z, Val b) {
  return z ? (after0(b) ? -1 : 1) : (b.v == t.v ? 1 : side(t, b));
}
__device__ __forceinline__ int side_bt(Val b, Val t, bool z) {
  return z ? (after0(b) ? 1 : -1) : (b.v == t.v ? -1 : side(b, t));
}
// Is the point just after t (0+ if z) on the open piece lat \ (X1 u X2)?  +1 certainly,
// -1 certainly not, 0 unsure.
__device__ __forceinline__ int in_piece(const Iv& lat, const Iv& X1, const Iv& X2, Val t, bool z) {
  if (lat.empty) return -1;
  const int a = side_bt(lat.lo, t, z), b = side_tb(t, z, lat.hi);
  if (a > 0 || b > 0) return -1;
  int r = (a < 0 && b < 0) ? 1 : 0;
  const Iv* X[2] = {&X1, &X2};
  for (int j = 0; j < 2; j++) {
    if (X[j]->empty) continue;
    const int c = side_tb(t, z, X[j]->lo), d = side_bt(X[j]->hi, t, z);
    if (c > 0 && d > 0) return -1;      // certainly inside the excluded part
    if (!(c < 0 || d < 0)) r = 0;       // not certainly outside it
  }
  return r;
}
// a <= b certain (false also when too close to tell; the caller flags that)
__device__ __forceinline__ bool lt_sure(Val a, Val b, bool& unsure) {
  if (!apart(a, b)) { unsure = true; }
  return a.v < b.v;
}

// The state of one track's distance walk between two sections (see pcon_begin).
enum : int { kSearch = 0, kStretch = 1, kDone = 2 };
struct Walk {
  F2 rad, A0;        // p.d_xy and u^2 + v^2, double-float
  Iv PH, X2;         // narrow-phi interval, wide-phi excluded wedge
  Val tcur, ans;     // search/stretch position, answer
  float rh, rl, r2h, erad, iw;
  int k, step, st, guard;
  bool zc, answered, u, goal_out, surf, need_in, need_out, in_range, live;
};

template <bool TUBE, bool FRAME = false>
__device__ inline bool pcon_begin(const Desc& S, const TrackF& T, unsigned want, R32& R, Walk& W) {
  W.live = false;
  W.need_in = W.need_out = false;
  const int nz = S.nz, last = nz - 1;
  // r = sqrt(x^2 + y^2) in double-float
  const F2 x2 = tprod(T.xh, T.xh), y2 = tprod(T.yh, T.yh);
  const F2 ss = tsum(x2.h, y2.h);
  const float low = ((ss.l + x2.l) + y2.l) + 2.f * (T.xh * T.xl + T.yh * T.yl);
  const float r2h = ss.h + low, r2l = low - (r2h - ss.h);
  const float rh = sqrtf(r2h);
  float rl = 0.f;
  if (rh > 0.f) {
    const F2 rr = tprod(rh, rh);
    rl = (((r2h - rr.h) - rr.l) + r2l) * __fdividef(0.5f, rh);
  }
  // Section of the point: the first k with z < z[k+1].  In a placed volume's frame the
  // binary64 z is not at hand: a point within rounding of an internal plane goes to binary64.
  int k0 = 0;
  bool near_plane = false;
  if (!FRAME) {
    while (k0 < nz - 2 && T.zkey >= S.zkey[k0 + 1]) k0++;
  } else {
    while (k0 < nz - 2 && (T.zh - S.zh[k0 + 1]) + (T.zl - S.zl[k0 + 1]) >= 0.f) k0++;
    for (int j = k0; j <= k0 + 1; j++) {
      if (j < 1 || j > nz - 2) continue;
      const float gj = (T.zh - S.zh[j]) + (T.zl - S.zl[j]);
      near_plane |= fabsf(gj) <= fmaf(G42, fabsf(T.zh) + fabsf(S.zh[j]), 2.f * T.fl);
    }
  }
  const bool has_phi = S.flags & kHasPhi, wide = S.flags & kPhiWide;
  const bool has_in = (S.inner >> k0) & 1u;
  const Lat lo_ = lateral<TUBE>(S.oah[k0], S.oal[k0], S.obh[k0], S.obl[k0], S.ok_[k0], rh, rl, T, true);
  Lat li_{-F_INF, 0.f, 0.f, 0.f};
  if (has_in) li_ = lateral<TUBE>(S.iah[k0], S.ial[k0], S.ibh[k0], S.ibl[k0], S.ik_[k0], rh, rl, T, false);
  const float gz0 = (S.zh[0] - T.zh) + (S.zl[0] - T.zl);
  const float Ez0 = 4.f * U * fabsf(gz0) + G42 * (fabsf(T.zh) + fabsf(S.zh[0])) + T.fl;
  const float gz1 = (T.zh - S.zh[last]) + (T.zl - S.zl[last]);
  const float Ez1 = 4.f * U * fabsf(gz1) + G42 * (fabsf(T.zh) + fabsf(S.zh[last])) + T.fl;
  Gv pa{-F_INF, 0.f}, pb{-F_INF, 0.f};
  float gphi = -F_INF, phlo = -F_INF, phhi = -F_INF;  // phi value and the interval holding it
  if (has_phi) {
    pa = phi_plane(S.nsh, S.nsl, T);
    pb = phi_plane(S.neh, S.nel, T);
    if (wide) {
      gphi = fminf(pa.g, pb.g);
      phlo = fminf(pa.g - pa.E, pb.g - pb.E);
      phhi = fminf(pa.g + pa.E, pb.g + pb.E);
    } else {
      gphi = fmaxf(pa.g, pb.g);
      phlo = fmaxf(pa.g - pa.E, pb.g - pb.E);
      phhi = fmaxf(pa.g + pa.E, pb.g + pb.E);
    }
  }
  SInt si = sint();
  si.add(lo_.g, lo_.E);
  if (has_in) si.add(li_.g, li_.E);
  si.add(gz0, Ez0);
  si.add(gz1, Ez1);
  if (has_phi) si.add_int(gphi, phlo, phhi);
  const float s = si.s;
  R.code = decide(si, R.flag);
  if (FRAME && near_plane) R.flag = true;

  if (want & (kWantSin | kWantSout)) {
    R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
    R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
    if (nz == 2 && R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
    if (nz > 2 && R.code != 1) {
      // sections as closed pieces (own z-planes included), each a max of constraints
      auto closed_df = [&](int k) -> Val {
        SInt c = sint();
        const Lat lo2 = k == k0 ? lo_ : lateral<TUBE>(S.oah[k], S.oal[k], S.obh[k], S.obl[k], S.ok_[k], rh, rl, T, true);
        c.add(lo2.g, lo2.E);
        if ((S.inner >> k) & 1u) {
          const Lat li2 = k == k0 ? li_ : lateral<TUBE>(S.iah[k], S.ial[k], S.ibh[k], S.ibl[k], S.ik_[k], rh, rl, T, false);
          c.add(li2.g, li2.E);
        }
        const float gk0 = (S.zh[k] - T.zh) + (S.zl[k] - T.zl);
        const float gk1 = (T.zh - S.zh[k + 1]) + (T.zl - S.zl[k + 1]);
        c.add(gk0, 4.f * U * fabsf(gk0) + G42 * (fabsf(T.zh) + fabsf(S.zh[k])) + T.fl);
        c.add(gk1, 4.f * U * fabsf(gk1) + G42 * (fabsf(T.zh) + fabsf(S.zh[k + 1])) + T.fl);
        if (has_phi) c.add_int(gphi, phlo, phhi);
        return {c.s, c.err()};
      };
      if (R.code == 0) {  // SafetyToOut: the containing piece
        const Val c = closed_df(k0);
        R.sout = -c.v;
        if (!certified({fabsf(c.v), c.e})) R.flag = true;
      } else {
        // SafetyToIn = min over pieces.  Plain binary32 values with their bounds give an
        // upper bound umin on the minimum; only pieces whose lower bound is below it can
        // hold it, and only those are evaluated in double-float (each lane loops over its
        // own candidates, one or two as a rule).
        auto closed_f = [&](int k, float& e) -> float {
          float v = fmaxf((rh - fmaf(S.oah[k], T.zh, S.obh[k])) * S.ok_[k], fmaxf(S.zh[k] - T.zh, T.zh - S.zh[k + 1]));
          float m = rh + fabsf(S.oah[k] * T.zh) + fabsf(S.obh[k]) + fabsf(T.zh) + fabsf(S.zh[k]) + fabsf(S.zh[k + 1]);
          if ((S.inner >> k) & 1u) {
            v = fmaxf(v, (fmaf(S.iah[k], T.zh, S.ibh[k]) - rh) * S.ik_[k]);
            m += fabsf(S.iah[k] * T.zh) + fabsf(S.ibh[k]);
          }
          e = fmaf(8.f * U, m, 3.f * T.fl);
          if (has_phi) { v = fmaxf(v, gphi); e += phhi - phlo; }
          return v;
        };
        // Sections are visited outward from k0 in z: a piece's value is at least its z-gap
        // (how far the point lies beyond the piece's z-slab), which grows away from k0, so
        // once a gap minus its rounding bound exceeds umin no farther piece can hold the
        // minimum (its exact value exceeds umin, an upper bound on the minimum).
        auto far_in_z = [&](int k, float u) -> bool {
          const float gap = fmaxf(S.zh[k] - T.zh, T.zh - S.zh[k + 1]);
          return gap - fmaf(4.f * U, fabsf(T.zh) + fabsf(S.zh[k]) + fabsf(S.zh[k + 1]), T.fl) > u;
        };
        float umin;
        {
          float e;
          const float v = closed_f(k0, e);
          umin = v + e;
        }
        int klo = k0, khi = k0;
        for (int k = k0 - 1; k >= 0 && !far_in_z(k, umin); k--) {
          float e;
          const float v = closed_f(k, e);
          umin = fminf(umin, v + e);
          klo = k;
        }
        for (int k = k0 + 1; k < last && !far_in_z(k, umin); k++) {
          float e;
          const float v = closed_f(k, e);
          umin = fminf(umin, v + e);
          khi = k;
        }
        uint32_t cand = 0u;
        for (int k = klo; k <= khi; k++) {
          float e;
          const float v = closed_f(k, e);
          if (!(v - e > umin)) cand |= 1u << k;
        }
        Val best{BIG, 0.f};
        while (cand) {
          const int k = __ffs(cand) - 1;
          cand &= cand - 1u;
          best = vmin(best, closed_df(k));
        }
        R.sin = best.v;
        if (!certified(best)) R.flag = true;
      }
    }
  }
  if (!(want & (kWantDin | kWantDout))) return false;

  const F2 rad = radial_df(T);
  const float radial = rad.h;
  float erad = G42 * (fabsf(T.xh * T.u) + fabsf(T.yh * T.v)) + 1e-30f;  // of rad
  float eRadial = 4.f * U * (fabsf(T.xh * T.u) + fabsf(T.yh * T.v)) + 1e-30f;
  if (FRAME) {  // point and direction errors of a frame track
    const float ef = fmaf(1.01f * T.dfl, fabsf(T.xh) + fabsf(T.yh), 1.01f * T.fl * (fabsf(T.u) + fabsf(T.v)));
    erad += ef;
    eRadial += ef;
  }
  const F2 A0 = a0_df(T);
  float nds = 0.f, nde = 0.f, ends = 0.f, ende = 0.f;
  if (has_phi) {
    nds = S.nsh[0] * T.u + S.nsh[1] * T.v;
    nde = S.neh[0] * T.u + S.neh[1] * T.v;
    ends = 6.f * U * (fabsf(S.nsh[0] * T.u) + fabsf(S.nsh[1] * T.v)) + (FRAME ? 1.5f * T.dfl : 0.f) + 1e-30f;
    ende = 6.f * U * (fabsf(S.neh[0] * T.u) + fabsf(S.neh[1] * T.v)) + (FRAME ? 1.5f * T.dfl : 0.f) + 1e-30f;
  }
  // Derivatives along d and their bounds, widened by the tangent threshold (the lateral
  // ones are r times the derivative per unit length over k).
  const float ao = TUBE ? 0.f : S.oah[k0], ai = TUBE ? 0.f : S.iah[k0];
  const float ew = FRAME ? T.dfl : 0.f;
  const float gdo = radial - ao * T.w * rh, gdi = -(radial - ai * T.w * rh);
  const float egdo = eRadial + 4.f * U * fabsf(ao * T.w * rh) + fabsf(ao) * rh * ew + 2.f * TAUF * rh * (1.f + fabsf(ao));
  const float egdi = eRadial + 4.f * U * fabsf(ai * T.w * rh) + fabsf(ai) * rh * ew + 2.f * TAUF * rh * (1.f + fabsf(ai));
  const float ewz = ew + TAUF, endsT = ends + TAUF, endeT = ende + TAUF;
  // A constraint within reach of the band that the ray may run along (any start): binary64.
  {
    auto slide_chk = [&](float g, float Eg, float gd, float egd) {
      if (fabsf(g) <= HF + Eg && fabsf(gd) <= egd) R.flag = true;
    };
    slide_chk(lo_.g, lo_.E, gdo, egdo);
    if (has_in) slide_chk(li_.g, li_.E, gdi, egdi);
    slide_chk(gz0, Ez0, -T.w, ewz);
    slide_chk(gz1, Ez1, T.w, ewz);
    if (has_phi) {
      slide_chk(pa.g, pa.E, nds, endsT);
      slide_chk(pb.g, pb.E, nde, endeT);
    }
  }
  // surface start: decided here only when some constraint certainly grows (leaving)
  // or every one certainly shrinks (entering); the other surface cases go to binary64.
  bool any_out = false, all_in = true, unsure = false;
  if (R.code == 1) {
    auto add = [&](float g, float Eg, float gd, float egd) {
      if (fabsf(g + HF) <= Eg) { unsure = true; return; }
      if (g >= -HF) {
        if (fabsf(gd) <= egd) { unsure = true; return; }
        if (gd > 0) any_out = true;
        if (!(gd < 0)) all_in = false;
      }
    };
    add(lo_.g, lo_.E, gdo, egdo);
    if (has_in) add(li_.g, li_.E, gdi, egdi);
    add(gz0, Ez0, -T.w, ewz);
    add(gz1, Ez1, T.w, ewz);
    if (has_phi) {
      if (wide) {
        if (fabsf(pa.g - pb.g) <= pa.E + pb.E) unsure = true;
        if (pa.g <= pb.g) add(pa.g, pa.E, nds, endsT); else add(pb.g, pb.E, nde, endeT);
      } else {
        add(pa.g, pa.E, nds, endsT);
        add(pb.g, pb.E, nde, endeT);
      }
    }
  }

  // A surface point that is leaving has DistanceToOut 0 and needs DistanceToIn; one that
  // is entering has DistanceToIn 0 and needs DistanceToOut.  Both searches below start
  // just after 0 (written 0+), where a crossing not certainly after 0 is the surface the
  // point is on.
  const bool surf = R.code == 1;
  const bool leaving = surf && any_out && !unsure, entering = surf && all_in && !unsure;
  if (surf) {
    if (want & kWantDout) R.dout = 0.f;
    if (want & kWantDin) R.din = 0.f;
    if (!leaving && !entering && (want & (kWantDin | kWantDout))) R.flag = true;
  }
  if (R.code == 0 && (want & kWantDin)) R.din = -1.f;
  if (R.code == 2 && (want & kWantDout)) R.dout = -1.f;
  W.need_out = (R.code == 0 || entering) && (want & kWantDout);
  W.need_in = (R.code == 2 || leaving) && (want & kWantDin);
  if (!W.need_out && !W.need_in) return false;

  // Distances in interval form, over the sections the ray meets for t >= 0 in t order.
  // In section k the ray is inside the solid on C \ (X1 u X2): C = outer region of the
  // section's line ∩ the section's z slab ∩ narrow phi, X1 = its hole, X2 = the wedge cut
  // out by a wide phi.  Each track computes one distance with two steps: SEARCH finds the
  // first start of such a piece after tcur; STRETCH follows the piece holding tcur across
  // internal planes (not surfaces: the profile is continuous) to its end.
  //   DistanceToIn, outside point:   SEARCH from 0; the start found is the answer.
  //   DistanceToIn, leaving surface: SEARCH from 0+; if 0+ is itself on a piece (the point
  //     is inside by less than h), STRETCH to its end and SEARCH again from there.
  //   DistanceToOut, inside point:   STRETCH from 0; its end is the answer.
  //   DistanceToOut, entering surface: SEARCH from 0+ (0+ itself, or a start just after 0
  //     when the point is outside by less than h), then STRETCH; none found: 0.
  // A value tcur always means "just after that crossing": a crossing equal to it (the same
  // one) counts as passed.  Inside and outside tracks run the same loop body.
  bool u = false;
  Iv PH = iv_all(), X2 = iv_none();
  if (has_phi) {
    if (!wide) PH = iv_and(iv_half(pa.g, pa.E, nds, ends, true, u), iv_half(pb.g, pb.E, nde, ende, true, u));
    else X2 = iv_and(iv_half(pa.g, pa.E, nds, ends, false, u), iv_half(pb.g, pb.E, nde, ende, false, u));
    if (!X2.empty && !(X2.lo.v < X2.hi.v)) {  // no wedge along the ray, unless too close to tell
      if (!apart(X2.lo, X2.hi)) u = true;
      X2 = iv_none();
    }
  }
  W.iw = T.w != 0 ? __frcp_rn(T.w) : 0.f;
  W.rad = rad;
  W.A0 = A0;
  W.erad = erad;
  W.rh = rh;
  W.rl = rl;
  W.r2h = r2h;
  W.PH = PH;
  W.X2 = X2;
  W.in_range = true;  // for w == 0: the ray's z inside [z0, zN]
  if (FRAME && fabsf(T.w) <= 4.f * T.dfl) u = true;  // the order of the sections is not certain
  // below z0 (above zN) the first section is k0 = 0 (k0 = nz - 2) already
  W.k = k0;
  if (T.w > 0) {
    W.step = 1;
  } else if (T.w < 0) {
    W.step = -1;
  } else {  // the ray stays in the plane z = const: one section or none
    W.step = 0;
    W.in_range = !(gz0 > 0) && !(gz1 > 0);
    for (int j = k0; j <= k0 + 1; j++) {  // on a plane the pieces on both sides meet: binary64
      const float gj = (S.zh[j] - T.zh) + (S.zl[j] - T.zl);
      if (fabsf(gj) <= 4.f * U * fabsf(gj) + G42 * (fabsf(T.zh) + fabsf(S.zh[j])) + T.fl) u = true;
    }
  }
  W.goal_out = W.need_out;
  W.surf = surf;
  W.st = R.code == 0 ? kStretch : kSearch;
  W.tcur = Val{0.f, 0.f};
  W.zc = surf;  // tcur is 0+
  W.ans = Val{BIG, 0.f};
  W.answered = false;
  W.u = u;
  W.guard = 0;
  W.live = true;
  return true;
}

// The binary32 time of z-plane j along the track, with its bound.
template <bool FRAME>
__device__ __forceinline__ Val plane_time(const Desc& S, const TrackF& T, float iw, int j) {
  const float num = (S.zh[j] - T.zh) + (S.zl[j] - T.zl);
  const float t = num * iw;
  float e = fmaf(G42, fabsf(T.zh) + fabsf(S.zh[j]), T.fl);
  if (FRAME) e = fmaf(1.01f * fabsf(t), T.dfl, e);
  return {t, fmaf(5.f * U, fabsf(t), e * fabsf(iw))};
}

// One section of the walk: the section W.k and its intervals, SEARCH and STRETCH in it,
// then the next section.  W.live turns false when the walk is over.
template <bool TUBE, bool FRAME = false>
__device__ inline void pcon_step(const Desc& S, const TrackF& T, Walk& W) {
  const int last = S.nz - 1;
  bool u = W.u;
  // An outside track looks only for an entry: while searching it passes over the sections
  // whose slab the ray crosses (t >= 0) farther from the axis than the section's largest
  // outer radius, by a wide margin; a section not certainly missed is examined in full.
  auto may_enter = [&](int j) -> bool {
    const float t0 = plane_time<FRAME>(S, T, W.iw, j).v, t1 = plane_time<FRAME>(S, T, W.iw, j + 1).v;
    const float m = fmaf(1e-5f, fabsf(t0) + fabsf(t1), 1e-6f);
    const float lo = fmaxf(fminf(t0, t1) - m, 0.f), hi = fmaxf(t0, t1) + m;
    if (hi < lo) return false;  // behind the start
    const float radial = W.rad.h;
    const float tm = fminf(fmaxf(W.A0.h > 0.f ? -radial / W.A0.h : lo, lo), hi);
    const float r2 = fmaf(fmaf(W.A0.h, tm, 2.f * radial), tm, W.r2h);
    const float Rm = fmaxf(fmaf(S.oah[j], S.zh[j], S.obh[j]), fmaf(S.oah[j], S.zh[j + 1], S.obh[j]));
    const float mag = W.r2h + 2.f * fabsf(radial * tm) + W.A0.h * tm * tm + Rm * Rm;
    return !(r2 - Rm * Rm > fmaf(1e-5f, mag, 1e-6f));
  };
  int k = W.k;
  const int step = W.step;
  if (step != 0 && W.st == kSearch && S.nz > 2) {
    while (k >= 0 && k <= last - 1 && !may_enter(k)) k += step;
    if (k < 0 || k > last - 1) {
      W.k = k;
      W.live = false;
      return;
    }
  }
  Iv slab = iv_all();
  if (step != 0) {
    const Val ta = plane_time<FRAME>(S, T, W.iw, k), tb = plane_time<FRAME>(S, T, W.iw, k + 1);
    slab = step > 0 ? Iv{ta, tb, false} : Iv{tb, ta, false};
  } else if (!W.in_range) {
    slab = iv_none();
  }
  const bool beyond = !slab.empty && slab.hi.v < -slab.hi.e;  // this section is behind the ray
  if (!beyond) {
    const float ao = TUBE ? 0.f : S.oah[k];
    const Lat Lo = lateral<TUBE>(S.oah[k], S.oal[k], S.obh[k], S.obl[k], S.ok_[k], W.rh, W.rl, T, true);
    const Quad qo = quad32<TUBE, FRAME>(ao, TUBE ? 0.f : S.oal[k], Lo, T, W.rad, W.erad, W.A0, W.rh, W.rl);
    u |= qo.unsure;
    const Iv lat = iv_and(iv_region(qo, Lo.g, Lo.E, u), W.PH);  // lateral and phi part of C
    Iv X1 = iv_none();
    if ((S.inner >> k) & 1u) {
      const float ai = TUBE ? 0.f : S.iah[k];
      const Lat Li = lateral<TUBE>(S.iah[k], S.ial[k], S.ibh[k], S.ibl[k], S.ik_[k], W.rh, W.rl, T, false);
      const Quad qi = quad32<TUBE, FRAME>(ai, TUBE ? 0.f : S.ial[k], Li, T, W.rad, W.erad, W.A0, W.rh, W.rl);
      u |= qi.unsure;
      X1 = iv_region(qi, -Li.g, Li.E, u);
      if (!X1.empty && !(X1.lo.v < X1.hi.v)) {  // no hole along the ray, unless too close to tell
        if (!apart(X1.lo, X1.hi)) u = true;
        X1 = iv_none();
      }
    }
    const Iv& X2 = W.X2;
    const Iv C = iv_and(lat, slab);
    // v at or before tcur (passed): the same crossing, certainly earlier, or within 0+
    auto passed = [&](Val v) -> bool {
      if (W.zc) return !after0(v);
      if (v.v == W.tcur.v) return true;
      return !lt_sure(W.tcur, v, u);
    };
    // SEARCH: the first point of C \ (X1 u X2) after tcur in this section
    auto search = [&]() {
      if (C.empty || passed(C.hi)) return;
      Val t = W.tcur;
      bool z = W.zc;
      if (!passed(C.lo)) { t = C.lo; z = false; }
      for (int pass = 0; pass < 2; pass++) {
        const Iv* X[2] = {&X1, &X2};
        for (int j = 0; j < 2; j++) {
          if (X[j]->empty || (!z && t.v == X[j]->hi.v)) continue;
          const bool lo_passed = z ? !after0(X[j]->lo) : (X[j]->lo.v == t.v || !lt_sure(t, X[j]->lo, u));
          const bool hi_ahead = z ? after0(X[j]->hi) : lt_sure(t, X[j]->hi, u);
          if (lo_passed && hi_ahead) { t = X[j]->hi; z = false; }
        }
      }
      if (!z && (t.v == C.hi.v || !lt_sure(t, C.hi, u))) return;  // pushed past C
      if (!W.goal_out && !z) {  // an entry: the answer
        if (!W.surf && !(t.v > t.e)) u = true;  // an outside point enters strictly after 0
        W.ans = t;
        W.answered = true;
        W.st = kDone;
        return;
      }
      W.st = kStretch;  // DistanceToOut from the piece's start, or a leaving point inside at 0+
      W.tcur = t;
      W.zc = z;
    };
    if (W.st == kSearch) search();
    if (W.st == kStretch) {
      const int at = in_piece(lat, X1, X2, W.tcur, W.zc);
      Val e = lat.hi;  // end of the inside stretch holding tcur
      if (!X1.empty && (W.zc ? after0(X1.lo) : X1.lo.v > W.tcur.v)) e = vmin(e, X1.lo);
      if (!X2.empty && (W.zc ? after0(X2.lo) : X2.lo.v > W.tcur.v)) e = vmin(e, X2.lo);
      if (at <= 0) {  // the section must hold tcur (the profile is continuous)
        u = true;
        W.st = kDone;
      } else if (step != 0 && lt_sure(slab.hi, e, u)) {  // reaches the far plane first
        const bool end_plane = (step > 0 && k + 1 == last) || (step < 0 && k == 0);
        if (!end_plane) {
          W.tcur = slab.hi;
          W.zc = false;
        } else if (W.goal_out) {
          W.ans = slab.hi;
          W.answered = true;
          W.st = kDone;
        } else {
          W.st = kDone;  // leaves through an end plane: no entry after it
        }
      } else if (W.goal_out) {
        W.ans = e;
        W.answered = true;
        W.st = kDone;
      } else {  // a leaving point's stretch ends: look for the next entry
        W.tcur = e;
        W.zc = false;
        W.st = kSearch;
        search();
      }
    }
  }
  W.u = u;
  W.k = k + step;
  W.guard++;
  if (W.st == kDone || step == 0 || W.k < 0 || W.k > last - 1 || W.guard >= kMaxZ) W.live = false;
}

// The distances from a finished walk (nothing when none was needed).
__device__ inline void pcon_end(const Walk& W, R32& R) {
  bool u = W.u;
  if (W.st == kStretch) u = true;  // a stretch must end at a surface
  if (W.need_out) {
    // entering surface point whose ray never gets inside: 0
    const Val d = W.answered ? W.ans : Val{0.f, 0.f};
    if (u || !certified(d)) R.flag = true;
    R.dout = unbig(d.v);
  }
  if (W.need_in) {
    if (u || !certified(W.ans)) R.flag = true;
    R.din = W.answered ? W.ans.v : F_INF;
  }
}

template <bool TUBE, bool FRAME = false>
__device__ inline void pcon32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
  Walk W;
  if (pcon_begin<TUBE, FRAME>(S, T, want, R, W))
    while (W.live) pcon_step<TUBE, FRAME>(S, T, W);
  pcon_end(W, R);
}

}  // namespace f32
}  // namespace gv
