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
// that need the full set of rules.  No binary64 instruction is used here.
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
#define F_INF CUDART_INF_F

enum : unsigned { kWantCode = 1, kWantDin = 2, kWantDout = 4, kWantSin = 8, kWantSout = 16 };

struct TrackF {
  float xh, yh, zh, xl, yl, zl;  // point: hi + lo
  float u, v, w;                 // direction: hi
  float ul, vl, wl;              // direction: lo
  long long zkey;                // order key of z
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
// a < b decided with certainty?
__device__ __forceinline__ bool apart(Val a, Val b) { return fabsf(a.v - b.v) > a.e + b.e; }

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
// Exact binary32 -> binary64 bit pattern (denormals flushed to zero).
__device__ __forceinline__ unsigned long long f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t s = b & 0x80000000u, a = b & 0x7FFFFFFFu;
  uint32_t hi = s | ((a >> 3) + (896u << 20));
  uint32_t lo = a << 29;
  if (a < 0x00800000u) { hi = s; lo = 0u; }
  if (a >= 0x7F800000u) { hi = s | 0x7FF00000u | (a > 0x7F800000u ? 0x80000u : 0u); lo = 0u; }
  return ((unsigned long long)hi << 32) | lo;
}

template <bool DIR_LO = true>
__device__ __forceinline__ TrackF load_track(const uint2* x, const uint2* y, const uint2* z,
                                             const uint2* u, const uint2* v, const uint2* w,
                                             int64_t i, bool dirs) {
  TrackF T;
  T.bad = false;
  const uint2 bz = __ldg(z + i);
  split(__ldg(x + i), T.xh, T.xl, T.bad);
  split(__ldg(y + i), T.yh, T.yl, T.bad);
  split(bz, T.zh, T.zl, T.bad);
  T.zkey = order_key((long long)(((unsigned long long)bz.y << 32) | bz.x));
  if (dirs) {
    const uint2 bu = __ldg(u + i), bv = __ldg(v + i), bw = __ldg(w + i);
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
__device__ __forceinline__ Gv abs_minus(float ph, float pl, float Dh, float Dl) {
  const float a = fabsf(ph);
  const float g = (a - Dh) + ((ph < 0 ? -pl : pl) - Dl);
  return {g, 4.f * U * fabsf(g) + G42 * (a + Dh) + FLOOR};
}
// (n.p - c) with n, c split, p split
__device__ __forceinline__ Gv plane_g(const float* nh, const float* nl, float ch, float cl,
                                      const TrackF& T) {
  const F2 p0 = tprod(nh[0], T.xh), p1 = tprod(nh[1], T.yh), p2 = tprod(nh[2], T.zh);
  const F2 s1 = tsum(p0.h, p1.h), s2 = tsum(s1.h, p2.h), s3 = tsum(s2.h, -ch);
  float lo = ((s1.l + s2.l) + s3.l) + ((p0.l + p1.l) + p2.l);
  lo += nh[0] * T.xl + nl[0] * T.xh;
  lo += nh[1] * T.yl + nl[1] * T.yh;
  lo += nh[2] * T.zl + nl[2] * T.zh;
  lo -= cl;
  const float g = s3.h + lo;
  return {g, 4.f * U * fabsf(g) + G42 * (fabsf(T.xh) + fabsf(T.yh) + fabsf(T.zh) + fabsf(ch)) + FLOOR};
}

// ------------------------------------------------------------------- box

__device__ inline void box32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
  const float ph[3] = {T.xh, T.yh, T.zh}, pl[3] = {T.xl, T.yl, T.zl}, d[3] = {T.u, T.v, T.w};
  Gv g[3];
  SInt si = sint();
  for (int i = 0; i < 3; i++) {
    g[i] = abs_minus(ph[i], pl[i], S.Dh[i], S.Dl[i]);
    si.add(g[i].g, g[i].E);
  }
  const float s = si.s;
  R.code = decide(si, R.flag);
  R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
  R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
  if (R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
  if (!(want & (kWantDin | kWantDout))) return;
  // surface motion
  bool any_out = false, all_in = true, never = false;
  if (R.code == 1) {
    for (int i = 0; i < 3; i++) {
      if (fabsf(g[i].g + HF) <= g[i].E) R.flag = true;
      if (g[i].g >= -HF) {
        const float gd = ph[i] < 0 ? -d[i] : d[i];
        if (gd > 0) any_out = true;
        if (!(gd < 0)) all_in = false;
      }
      if (d[i] == 0) {
        if (fabsf(g[i].g) <= g[i].E) R.flag = true;
        never |= g[i].g > 0;
      }
    }
  }
  // 1 / |d_i| once per axis (rounded to within 2 ulp); d_i == 0 gives a huge sentinel
  float inv[3];
  for (int i = 0; i < 3; i++) inv[i] = d[i] != 0 ? __frcp_rn(fabsf(d[i])) : 0.f;
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.f;
    else if (R.code == 1 && any_out) R.dout = 0.f;
    else if (R.code == 1) { R.flag = true; R.dout = 0.f; }  // surface, not leaving: binary64
    else {
      Val acc{BIG, 0.f};
      for (int i = 0; i < 3; i++) {
        if (d[i] == 0) continue;
        float num, en;
        if ((ph[i] < 0) == (d[i] < 0)) { num = -g[i].g; en = g[i].E; }
        else { num = S.Dh[i] + fabsf(ph[i]); en = 4.f * U * num; }
        const float t = num * inv[i];
        acc = vmin(acc, {t, fmaf(en, inv[i], 5.f * U * t)});
      }
      if (!certified(acc)) R.flag = true;
      R.dout = unbig(acc.v);
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.f;
    else if (R.code == 1) R.din = all_in ? 0.f : F_INF;
    else {
      Val tn{-BIG, 0.f}, tf{BIG, 0.f};
      bool miss = false;
      for (int i = 0; i < 3; i++) {
        if (d[i] == 0) {
          if (fabsf(g[i].g) <= g[i].E) R.flag = true;
          if (g[i].g > 0) miss = true;
          continue;
        }
        const float far = S.Dh[i] + fabsf(ph[i]);
        const float tnear = g[i].g * inv[i];
        const Val acc_near{tnear, fmaf(g[i].E, inv[i], 5.f * U * fabsf(tnear))};
        const float tfar = far * inv[i];
        const Val plain{tfar, 9.f * U * tfar};
        if ((ph[i] < 0) != (d[i] < 0)) {  // toward the face on the point's side
          tn = vmax(tn, acc_near);
          tf = vmin(tf, plain);
        } else {
          tn = vmax(tn, {-plain.v, plain.e});
          tf = vmin(tf, {-acc_near.v, acc_near.e});
        }
      }
      if (!miss) {
        if (!apart(tn, tf) || fabsf(tf.v) <= tf.e) R.flag = true;
        if (tn.v < tf.v && tf.v > 0) {
          if (!certified(tn)) R.flag = true;
          R.din = tn.v;
        } else R.din = F_INF;
      } else R.din = F_INF;
    }
  }
}

// ------------------------------------------------------------ trd / trap

__device__ inline void planar32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
  Gv g[5];
  float gd[5], egd[5];
  for (int i = 0; i < 4; i++) {
    g[i] = plane_g(S.plh[i], S.pll[i], S.plh[i][3], S.pll[i][3], T);
    const float a = S.plh[i][0] * T.u, b = S.plh[i][1] * T.v, c = S.plh[i][2] * T.w;
    gd[i] = (a + b) + c;
    egd[i] = 8.f * U * (fabsf(a) + fabsf(b) + fabsf(c)) + 1e-30f;
  }
  g[4] = abs_minus(T.zh, T.zl, S.dzh, S.dzl);
  gd[4] = T.zh < 0 ? -T.w : T.w;
  egd[4] = 0.f;
  SInt si = sint();
  for (int i = 0; i < 5; i++) si.add(g[i].g, g[i].E);
  const float s = si.s;
  R.code = decide(si, R.flag);
  R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
  R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
  if (R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
  if (!(want & (kWantDin | kWantDout))) return;
  bool any_out = false, all_in = true, never = false;
  if (R.code == 1) {
    for (int i = 0; i < 5; i++) {
      if (fabsf(g[i].g + HF) <= g[i].E) R.flag = true;
      const bool tangent = (i < 4) ? fabsf(gd[i]) <= egd[i] : gd[i] == 0;
      if (g[i].g >= -HF) {
        if (tangent && i < 4) R.flag = true;
        if (gd[i] > 0) any_out = true;
        if (!(gd[i] < 0)) all_in = false;
      }
      if (tangent) {
        if (fabsf(g[i].g) <= g[i].E || i < 4) { if (g[i].g > -HF) R.flag = true; }
        never |= g[i].g > 0;
      }
    }
  }
  float igd[4];
  for (int i = 0; i < 4; i++) igd[i] = __frcp_rn(gd[i]);
  const float iw = T.w != 0 ? __frcp_rn(fabsf(T.w)) : 0.f;
  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.f;
    else if (R.code == 1 && any_out) R.dout = 0.f;
    else if (R.code == 1) { R.flag = true; R.dout = 0.f; }  // surface, not leaving: binary64
    else {
      Val acc{BIG, 0.f};
      for (int i = 0; i < 4; i++) {
        if (fabsf(gd[i]) <= egd[i]) { R.flag = true; continue; }
        if (gd[i] > 0) {
          const float t = -g[i].g * igd[i];
          acc = vmin(acc, {t, fmaf(fmaf(fabsf(t), egd[i], g[i].E), igd[i], 5.f * U * fabsf(t))});
        }
      }
      if (T.w != 0) {
        float num, en;
        if ((T.zh < 0) == (T.w < 0)) { num = -g[4].g; en = g[4].E; }
        else { num = S.dzh + fabsf(T.zh); en = 4.f * U * num; }
        const float t = num * iw;
        acc = vmin(acc, {t, fmaf(en, iw, 5.f * U * t)});
      }
      if (!certified(acc)) R.flag = true;
      R.dout = unbig(acc.v);
    }
  }
  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.f;
    else if (R.code == 1) R.din = all_in ? 0.f : F_INF;
    else {
      Val tn{-BIG, 0.f}, tf{BIG, 0.f};
      bool miss = false;
      for (int i = 0; i < 4; i++) {
        if (fabsf(gd[i]) <= egd[i]) {
          // nearly parallel: entering never or much later; only certain if clearly outside
          if (g[i].g > g[i].E) { miss = true; continue; }
          R.flag = true;
          continue;
        }
        const float t = -g[i].g * igd[i];
        const Val tv{t, fmaf(fmaf(fabsf(t), egd[i], g[i].E), fabsf(igd[i]), 5.f * U * fabsf(t))};
        if (gd[i] < 0) tn = vmax(tn, tv); else tf = vmin(tf, tv);
      }
      if (T.w == 0) {
        if (fabsf(g[4].g) <= g[4].E) R.flag = true;
        if (g[4].g > 0) miss = true;
      } else {
        const float far = S.dzh + fabsf(T.zh);
        const float tnear = g[4].g * iw;
        const Val accn{tnear, fmaf(g[4].E, iw, 5.f * U * fabsf(tnear))};
        const Val plain{far * iw, far * iw * 9.f * U};
        if ((T.zh < 0) != (T.w < 0)) { tn = vmax(tn, accn); tf = vmin(tf, plain); }
        else { tn = vmax(tn, {-plain.v, plain.e}); tf = vmin(tf, {-accn.v, accn.e}); }
      }
      if (!miss) {
        if (!apart(tn, tf) || fabsf(tf.v) <= tf.e) R.flag = true;
        if (tn.v < tf.v && tf.v > 0) {
          if (!certified(tn)) R.flag = true;
          R.din = tn.v;
        } else R.din = F_INF;
      } else R.din = F_INF;
    }
  }
}

// ------------------------------------- polycone family (tube, cone, polycone)

struct Lat {   // a lateral constraint evaluated in double-float
  float g, E;  // g = (r - R) k  (outer) or (R - r) k (inner)
  float delta, eDelta;  // r - R and its bound
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
    Rl = ((ts.l + az.l) + (ah * T.zl + al * T.zh)) + bl;
    scale = rh + fabsf(az.h) + fabsf(bh);
  }
  const F2 dd = tsum(rh, -Rh);
  const float delta = dd.h + (dd.l + (rl - Rl));
  const float eDelta = 4.f * U * fabsf(delta) + G42 * scale + FLOOR;
  const float g = outer ? delta * k : -delta * k;
  return {g, 4.f * U * fabsf(g) + eDelta * k, delta, eDelta};
}

// phi plane value n.p in double-float
__device__ __forceinline__ Gv phi_plane(const float* nh, const float* nl, const TrackF& T) {
  const F2 p0 = tprod(nh[0], T.xh), p1 = tprod(nh[1], T.yh);
  const F2 s1 = tsum(p0.h, p1.h);
  float lo = s1.l + (p0.l + p1.l);
  lo += nh[0] * T.xl + nl[0] * T.xh;
  lo += nh[1] * T.yl + nl[1] * T.yh;
  const float g = s1.h + lo;
  return {g, 4.f * U * fabsf(g) + G42 * (fabsf(T.xh) + fabsf(T.yh)) + FLOOR};
}

// Crossings of r = a z + b with the track in binary32 with error bounds.
struct Quad {
  Val tm, tp;
  bool hm, hp;
  bool unsure;
};
// A0 = u^2 + v^2 in double-float from the split direction
__device__ __forceinline__ F2 a0_df(const TrackF& T) {
  const F2 uu = tprod(T.u, T.u), vv = tprod(T.v, T.v);
  const F2 s = tsum(uu.h, vv.h);
  const float lo = (s.l + (uu.l + vv.l)) + 2.f * (T.u * T.ul + T.v * T.vl);
  return {s.h + lo, lo - ((s.h + lo) - s.h)};
}

template <bool TUBE>
__device__ inline Quad quad32(float a, float al, float b, const TrackF& T, float radial, float eRadial, F2 A0,
                              float C, float eC) {
  Quad q;
  q.hm = q.hp = false;
  q.unsure = false;
  q.tm = q.tp = {0.f, 0.f};
  const float P = TUBE ? b : fmaf(a, T.zh, b);
  float D, A, eA;
  if (TUBE) {
    D = 0.f;
    A = A0.h + A0.l;
    eA = 2.f * U * A + 1e-30f;
  } else {  // A = A0 - (a w)^2 in double-float: rays nearly along the cone's slope keep their roots
    const F2 dd = tprod(a, T.w);
    const float dl = dd.l + (a * T.wl + al * T.w);
    D = dd.h + dl;
    const F2 d2 = tprod(dd.h, dd.h);
    const float d2l = d2.l + 2.f * dd.h * dl;
    const F2 s = tsum(A0.h, -d2.h);
    A = s.h + ((s.l + A0.l) - d2l);
    eA = 4.f * U * fabsf(A) + 2.3e-13f * (A0.h + d2.h) + 1e-30f;
  }
  const float B = radial - P * D;
  const float eB = eRadial + 6.f * U * fabsf(P * D) + 4.f * U * fabsf(a) * fabsf(T.zh) * fabsf(D);
  if (A == 0.f && D == 0.f && A0.h == 0.f) return q;  // parallel to the axis of a cylinder: no crossing
  const float disc = B * B - A * C;
  const float eD = 2.f * fabsf(B) * eB + fabsf(A) * eC + fabsf(C) * eA + 4.f * U * (B * B + fabsf(A * C));
  if (disc < -eD) return q;
  if (disc <= eD) { q.unsure = true; return q; }
  const float rs = rsqrtf(disc);
  const float sq = disc * rs;
  const float esq = 0.5f * eD * rs + 4.f * U * sq;
  float qq, r1, r2;  // r1 = qq / A, r2 = C / qq
  bool r1_is_plus;
  if (B >= 0) { qq = -(B + sq); r1_is_plus = false; }
  else { qq = sq - B; r1_is_plus = true; }
  const float eq = eB + esq + U * fabsf(qq);
  const float iA = __frcp_rn(A), iq = __frcp_rn(qq);
  r1 = qq * iA;
  r2 = C * iq;
  const float relq = eq * fabsf(iq);
  const float rel1 = (fabsf(A) <= eA) ? F_INF : relq + eA * fabsf(iA) + 4.f * U;
  const Val v1{r1, fabsf(r1) * rel1};
  const Val v2{r2, fmaf(fabsf(C), relq + 4.f * U, eC) * fabsf(iq)};
  Val vp = r1_is_plus ? v1 : v2, vm = r1_is_plus ? v2 : v1;
  q.tp = vp; q.tm = vm; q.hp = q.hm = true;
  if (!TUBE) {  // keep roots on the nappe a z + b >= 0
    for (int j = 0; j < 2; j++) {
      const Val t = j ? q.tp : q.tm;
      const float Rt = fmaf(t.v, D, P);
      const float eR = 4.f * U * (fabsf(P) + fabsf(t.v * D)) + fabsf(D) * t.e + 1e-30f;
      if (fabsf(Rt) <= eR && isfinite(t.v)) q.unsure = true;
      if (!(Rt >= 0)) { if (j) q.hp = false; else q.hm = false; }
    }
  }
  return q;
}

// strict-margin checks of an entry point q = p + t d (error of q: eq per coordinate)
struct Pt { float x, y, z, e; };
__device__ __forceinline__ Pt advance(const TrackF& T, Val t) {
  const float x = fmaf(t.v, T.u, T.xh), y = fmaf(t.v, T.v, T.yh), z = fmaf(t.v, T.w, T.zh);
  const float e = t.e + 4.f * U * (fabsf(T.xh) + fabsf(T.yh) + fabsf(T.zh) + fabsf(t.v));
  return {x, y, z, e};
}
// Returns +1 if certainly inside the open lateral region of section k, -1 if certainly
// not, 0 if too close to decide.
__device__ __forceinline__ int radial_in(const Desc& S, int k, const Pt& q, bool skip_out, bool skip_in) {
  const float r = sqrtf(q.x * q.x + q.y * q.y);
  const float er = q.e * 1.5f + 4.f * U * r;
  int res = 1;
  if (!skip_out) {
    const float R = fmaf(S.oah[k], q.z, S.obh[k]);
    const float m = R - r;
    const float e = er + fabsf(S.oah[k]) * q.e + 4.f * U * (fabsf(R) + fabsf(S.oah[k] * q.z)) + 1e-30f;
    if (fabsf(m) <= e) res = 0;
    else if (m < 0) return -1;
  }
  if (!skip_in && ((S.inner >> k) & 1u)) {
    const float R = fmaf(S.iah[k], q.z, S.ibh[k]);
    const float m = r - R;
    const float e = er + fabsf(S.iah[k]) * q.e + 4.f * U * (fabsf(R) + fabsf(S.iah[k] * q.z)) + 1e-30f;
    if (fabsf(m) <= e) res = 0;
    else if (m < 0) return -1;
  }
  return res;
}
__device__ __forceinline__ int phi_in(const Desc& S, const Pt& q) {
  if (!(S.flags & kHasPhi)) return 1;
  const float a = S.nsh[0] * q.x + S.nsh[1] * q.y, b = S.neh[0] * q.x + S.neh[1] * q.y;
  const float e = 1.5f * q.e + 4.f * U * (fabsf(q.x) + fabsf(q.y)) + 1e-30f;
  const float g = (S.flags & kPhiWide) ? fminf(a, b) : fmaxf(a, b);
  if (fabsf(g) <= e) return 0;
  return g < 0 ? 1 : -1;
}
// +1 if z0 < q.z < zN and zk <= q.z <= zk1 certainly, -1 if certainly not, 0 otherwise
__device__ __forceinline__ int zrange_in(float lo, float hi, float z0, float zN, const Pt& q) {
  const float e = q.e + 4.f * U * fabsf(q.z);
  if (fabsf(q.z - lo) <= e || fabsf(q.z - hi) <= e || fabsf(q.z - z0) <= e || fabsf(q.z - zN) <= e) return 0;
  return (q.z >= lo && q.z <= hi && q.z > z0 && q.z < zN) ? 1 : -1;
}

template <bool TUBE>
__device__ inline void pcon32(const Desc& S, const TrackF& T, unsigned want, R32& R) {
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
  int k0 = 0;
  while (k0 < nz - 2 && T.zkey >= S.zkey[k0 + 1]) k0++;
  const bool has_phi = S.flags & kHasPhi, wide = S.flags & kPhiWide;
  const bool has_in = (S.inner >> k0) & 1u;
  const Lat lo_ = lateral<TUBE>(S.oah[k0], S.oal[k0], S.obh[k0], S.obl[k0], S.ok_[k0], rh, rl, T, true);
  Lat li_{-F_INF, 0.f, 0.f, 0.f};
  if (has_in) li_ = lateral<TUBE>(S.iah[k0], S.ial[k0], S.ibh[k0], S.ibl[k0], S.ik_[k0], rh, rl, T, false);
  const float gz0 = (S.zh[0] - T.zh) + (S.zl[0] - T.zl);
  const float Ez0 = 4.f * U * fabsf(gz0) + G42 * (fabsf(T.zh) + fabsf(S.zh[0])) + FLOOR;
  const float gz1 = (T.zh - S.zh[last]) + (T.zl - S.zl[last]);
  const float Ez1 = 4.f * U * fabsf(gz1) + G42 * (fabsf(T.zh) + fabsf(S.zh[last])) + FLOOR;
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

  if (want & (kWantSin | kWantSout)) {
    R.sin = R.code == 0 ? -1.f : (R.code == 1 ? 0.f : s);
    R.sout = R.code == 2 ? -1.f : (R.code == 1 ? 0.f : -s);
    if (nz == 2 && R.code != 1 && !certified({fabsf(s), si.err()})) R.flag = true;
    if (nz > 2 && R.code != 1) {
      // sections as closed pieces: the containing one and its neighbours in
      // double-float, the others in plain binary32 with their bounds
      Val best{F_INF, 0.f};
      const int kb = R.code == 0 ? k0 : 0, ke = R.code == 0 ? k0 + 1 : last;
      for (int k = kb; k < ke; k++) {
        SInt c = sint();
        if (k >= k0 - 1 && k <= k0 + 1) {
          const Lat lo2 = k == k0 ? lo_ : lateral<TUBE>(S.oah[k], S.oal[k], S.obh[k], S.obl[k], S.ok_[k], rh, rl, T, true);
          c.add(lo2.g, lo2.E);
          if ((S.inner >> k) & 1u) {
            const Lat li2 = k == k0 ? li_ : lateral<TUBE>(S.iah[k], S.ial[k], S.ibh[k], S.ibl[k], S.ik_[k], rh, rl, T, false);
            c.add(li2.g, li2.E);
          }
          const float gk0 = (S.zh[k] - T.zh) + (S.zl[k] - T.zl);
          const float gk1 = (T.zh - S.zh[k + 1]) + (T.zl - S.zl[k + 1]);
          c.add(gk0, 4.f * U * fabsf(gk0) + G42 * (fabsf(T.zh) + fabsf(S.zh[k])) + FLOOR);
          c.add(gk1, 4.f * U * fabsf(gk1) + G42 * (fabsf(T.zh) + fabsf(S.zh[k + 1])) + FLOOR);
        } else {
          const float go = (rh - fmaf(S.oah[k], T.zh, S.obh[k])) * S.ok_[k];
          c.add(go, 8.f * U * (rh + fabsf(S.oah[k] * T.zh) + fabsf(S.obh[k])));
          if ((S.inner >> k) & 1u) {
            const float gi2 = (fmaf(S.iah[k], T.zh, S.ibh[k]) - rh) * S.ik_[k];
            c.add(gi2, 8.f * U * (rh + fabsf(S.iah[k] * T.zh) + fabsf(S.ibh[k])));
          }
          c.add(S.zh[k] - T.zh, 4.f * U * (fabsf(T.zh) + fabsf(S.zh[k])));
          c.add(T.zh - S.zh[k + 1], 4.f * U * (fabsf(T.zh) + fabsf(S.zh[k + 1])));
        }
        if (has_phi) c.add_int(gphi, phlo, phhi);
        if (R.code == 0 && k == k0) {
          R.sout = -c.s;
          if (!certified({c.s < 0 ? -c.s : c.s, c.err()})) R.flag = true;
          break;
        }
        best = vmin(best, {c.s, c.err()});
      }
      if (R.code == 2) {
        R.sin = best.v;
        if (!certified(best)) R.flag = true;
      }
    }
  }
  if (!(want & (kWantDin | kWantDout))) return;

  const float radial = fmaf(T.xh, T.u, fmaf(T.yh, T.v, (T.xh * T.ul + T.xl * T.u) + (T.yh * T.vl + T.yl * T.v)));
  const float eRadial = 4.f * U * (fabsf(T.xh * T.u) + fabsf(T.yh * T.v)) + 1e-30f;
  const F2 A0 = a0_df(T);
  float nds = 0.f, nde = 0.f, ends = 0.f, ende = 0.f;
  if (has_phi) {
    nds = S.nsh[0] * T.u + S.nsh[1] * T.v;
    nde = S.neh[0] * T.u + S.neh[1] * T.v;
    ends = 6.f * U * (fabsf(S.nsh[0] * T.u) + fabsf(S.nsh[1] * T.v)) + 1e-30f;
    ende = 6.f * U * (fabsf(S.neh[0] * T.u) + fabsf(S.neh[1] * T.v)) + 1e-30f;
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
    const float ao = TUBE ? 0.f : S.oah[k0], ai = TUBE ? 0.f : S.iah[k0];
    add(lo_.g, lo_.E, radial - ao * T.w * rh, eRadial + 4.f * U * fabsf(ao * T.w * rh));
    if (has_in) add(li_.g, li_.E, -(radial - ai * T.w * rh), eRadial + 4.f * U * fabsf(ai * T.w * rh));
    add(gz0, Ez0, -T.w, 0.f);
    add(gz1, Ez1, T.w, 0.f);
    if (has_phi) {
      if (wide) {
        if (fabsf(pa.g - pb.g) <= pa.E + pb.E) unsure = true;
        if (pa.g <= pb.g) add(pa.g, pa.E, nds, ends); else add(pb.g, pb.E, nde, ende);
      } else {
        add(pa.g, pa.E, nds, ends);
        add(pb.g, pb.E, nde, ende);
      }
    }
  }

  if (want & kWantDout) {
    if (R.code == 2) R.dout = -1.f;
    else if (R.code == 1 && any_out && !unsure) R.dout = 0.f;
    else if (R.code == 1) { R.flag = true; R.dout = 0.f; }
    else {
      // phi boundary
      Val tphi{F_INF, 0.f};
      if (has_phi) {
        if (!wide) {
          if (fabsf(nds) <= ends || fabsf(nde) <= ende) R.flag = true;
          if (nds > 0) { const float t = -pa.g / nds; tphi = vmin(tphi, {t, fabsf(t) * (pa.E / fabsf(pa.g) + ends / nds + 2.f * U)}); }
          if (nde > 0) { const float t = -pb.g / nde; tphi = vmin(tphi, {t, fabsf(t) * (pb.E / fabsf(pb.g) + ende / nde + 2.f * U)}); }
        } else {
          Val tin{-F_INF, 0.f}, tout{F_INF, 0.f};
          bool never = false;
          const Gv gg[2] = {pa, pb};
          const float nd[2] = {nds, nde}, en[2] = {ends, ende};
          for (int j = 0; j < 2; j++) {
            if (fabsf(nd[j]) <= en[j]) {
              if (gg[j].g > gg[j].E) continue;     // already and always beyond this plane
              if (gg[j].g < -gg[j].E) { never = true; continue; }
              R.flag = true;
              continue;
            }
            const float t = -gg[j].g / nd[j];
            const Val tv{t, fabsf(t) * (gg[j].E / fabsf(gg[j].g) + en[j] / fabsf(nd[j]) + 2.f * U)};
            if (nd[j] > 0) tin = vmax(tin, tv); else tout = vmin(tout, tv);
          }
          if (!never) {
            if (!apart(tin, tout) || fabsf(tin.v) <= tin.e) R.flag = true;
            if (tin.v < tout.v && tin.v > 0) tphi = tin;
          }
        }
      }
      // walk the z-sections
      int k = k0;
      Val tlo{0.f, 0.f}, t{F_INF, 0.f};
      for (int guard = 0; guard < kMaxZ; guard++) {
        Val tl{F_INF, 0.f};
        {
          const float ao = TUBE ? 0.f : S.oah[k];
          float C, eC;
          if (k == k0) {
            const float Rp = TUBE ? S.obh[k] : fmaf(ao, T.zh, S.obh[k]);
            C = lo_.delta * (rh + Rp);
            eC = lo_.eDelta * (rh + fabsf(Rp)) + 4.f * U * fabsf(C);
          } else {
            const float P = TUBE ? S.obh[k] : fmaf(ao, T.zh, S.obh[k]);
            C = r2h - P * P;
            eC = 8.f * U * (r2h + P * P) + 1e-30f;
          }
          const Quad q = quad32<TUBE>(ao, TUBE ? 0.f : S.oal[k], S.obh[k], T, radial, eRadial, A0, C, eC);
          if (q.unsure) R.flag = true;
          if (q.hp) {
            if (!apart(q.tp, tlo)) R.flag = true;
            if (q.tp.v > tlo.v) tl = q.tp;
          }
        }
        if ((S.inner >> k) & 1u) {
          const float ai = TUBE ? 0.f : S.iah[k];
          float C, eC;
          if (k == k0) {
            const float Rp = TUBE ? S.ibh[k] : fmaf(ai, T.zh, S.ibh[k]);
            C = li_.delta * (rh + Rp);
            eC = li_.eDelta * (rh + fabsf(Rp)) + 4.f * U * fabsf(C);
          } else {
            const float P = TUBE ? S.ibh[k] : fmaf(ai, T.zh, S.ibh[k]);
            C = r2h - P * P;
            eC = 8.f * U * (r2h + P * P) + 1e-30f;
          }
          const Quad q = quad32<TUBE>(ai, TUBE ? 0.f : S.ial[k], S.ibh[k], T, radial, eRadial, A0, C, eC);
          if (q.unsure) R.flag = true;
          if (q.hm) {
            if (!apart(q.tm, tlo)) R.flag = true;
            if (q.tm.v > tlo.v) tl = vmin(tl, q.tm);
          }
        }
        Val tp{F_INF, 0.f};
        bool end;
        if (T.w > 0) {
          const float num = (S.zh[k + 1] - T.zh) + (S.zl[k + 1] - T.zl);
          tp = {num / T.w, fabsf(num / T.w) * 4.f * U + (G42 * (fabsf(T.zh) + fabsf(S.zh[k + 1])) + FLOOR) / T.w};
          end = (k + 1 == last);
        } else if (T.w < 0) {
          const float num = (S.zh[k] - T.zh) + (S.zl[k] - T.zl);
          tp = {num / T.w, fabsf(num / T.w) * 4.f * U + (G42 * (fabsf(T.zh) + fabsf(S.zh[k])) + FLOOR) / -T.w};
          end = (k == 0);
        } else {
          end = true;
        }
        if (isfinite(tl.v) && isfinite(tp.v) && !apart(tl, tp)) R.flag = true;
        if (tl.v <= tp.v) { t = tl; break; }
        if (end) { t = tp; break; }
        k += T.w > 0 ? 1 : -1;
        tlo = tp;
      }
      const Val res = vmin(t, tphi);
      if (!certified(res)) R.flag = true;
      R.dout = res.v;
    }
  }

  if (want & kWantDin) {
    if (R.code == 0) R.din = -1.f;
    else if (R.code == 1 && all_in && !unsure) R.din = 0.f;
    else if (R.code == 1) { R.flag = true; R.din = 0.f; }
    else {
      Val best{F_INF, 0.f};
      const float z0 = S.zh[0], zN = S.zh[last];
      for (int k = 0; k < last; k++) {
        if (T.w > 0 && S.zh[k + 1] < T.zh - 1e-3f * fabsf(T.zh)) continue;
        if (T.w < 0 && S.zh[k] > T.zh + 1e-3f * fabsf(T.zh)) continue;
        if (T.w == 0 && (T.zh < S.zh[k] - 1e-3f * fabsf(T.zh) - 1e-6f || T.zh > S.zh[k + 1] + 1e-3f * fabsf(T.zh) + 1e-6f)) continue;
        for (int side = 0; side < 2; side++) {
          if (side == 1 && !((S.inner >> k) & 1u)) continue;
          const float a = TUBE ? 0.f : (side ? S.iah[k] : S.oah[k]);
          const float b = side ? S.ibh[k] : S.obh[k];
          float C, eC;
          if (k == k0) {
            const Lat& L = side ? li_ : lo_;
            const float Rp = TUBE ? b : fmaf(a, T.zh, b);
            C = L.delta * (rh + Rp);
            eC = L.eDelta * (rh + fabsf(Rp)) + 4.f * U * fabsf(C);
          } else {
            const float P = TUBE ? b : fmaf(a, T.zh, b);
            C = r2h - P * P;
            eC = 8.f * U * (r2h + P * P) + 1e-30f;
          }
          const Quad q = quad32<TUBE>(a, TUBE ? 0.f : (side ? S.ial[k] : S.oal[k]), b, T, radial, eRadial, A0, C, eC);
          if (q.unsure) R.flag = true;
          const bool has = side ? q.hp : q.hm;
          const Val tc = side ? q.tp : q.tm;
          if (!has || !(tc.v > -tc.e) || tc.v - tc.e > best.v + best.e) continue;
          if (fabsf(tc.v) <= tc.e) { R.flag = true; continue; }
          const Pt p = advance(T, tc);
          const int zr = zrange_in(S.zh[k], S.zh[k + 1], z0, zN, p);
          if (zr == 0) { R.flag = true; continue; }
          if (zr < 0) continue;
          const int rr = radial_in(S, k, p, side == 0, side == 1);
          const int pr = phi_in(S, p);
          if (rr == 0 || pr == 0) { R.flag = true; continue; }
          if (rr > 0 && pr > 0) best = vmin(best, tc);
        }
      }
      if (T.w != 0) {
        const int kk = T.w > 0 ? 0 : last - 1;
        const int ze = T.w > 0 ? 0 : last;
        const float num = (S.zh[ze] - T.zh) + (S.zl[ze] - T.zl);
        const float tv = num / T.w;
        const Val tc{tv, fabsf(tv) * 4.f * U + (G42 * (fabsf(T.zh) + fabsf(S.zh[ze])) + FLOOR) / fabsf(T.w)};
        if (tc.v > tc.e && tc.v - tc.e <= best.v + best.e) {
          Pt p = advance(T, tc);
          p.z = S.zh[ze];
          const int rr = radial_in(S, kk, p, false, false);
          const int pr = phi_in(S, p);
          if (rr == 0 || pr == 0) R.flag = true;
          else if (rr > 0 && pr > 0) best = vmin(best, tc);
        } else if (fabsf(tc.v) <= tc.e) R.flag = true;
      }
      if (has_phi) {
        const Gv gg[2] = {pa, pb};
        const float nd[2] = {nds, nde}, en[2] = {ends, ende};
        for (int j = 0; j < 2; j++) {
          if (fabsf(nd[j]) <= en[j]) { if (fabsf(gg[j].g) <= gg[j].E * 4.f + 1e-6f) R.flag = true; continue; }
          if (!(nd[j] < 0)) continue;
          const float tv = -gg[j].g / nd[j];
          const Val tc{tv, fabsf(tv) * (gg[j].E / fmaxf(fabsf(gg[j].g), 1e-30f) + en[j] / fabsf(nd[j]) + 2.f * U)};
          if (!(tc.v > -tc.e) || tc.v - tc.e > best.v + best.e) continue;
          if (fabsf(tc.v) <= tc.e) { R.flag = true; continue; }
          const Pt p = advance(T, tc);
          const float ez = p.e + 4.f * U * fabsf(p.z);
          if (fabsf(p.z - z0) <= ez || fabsf(p.z - zN) <= ez) { R.flag = true; continue; }
          if (!(p.z > z0 && p.z < zN)) continue;
          int kq = 0;
          while (kq < nz - 2 && p.z >= S.zh[kq + 1]) kq++;
          if (nz > 2) {  // near an internal plane either section may apply
            const float ek = p.e + 4.f * U * fabsf(p.z);
            if ((kq + 1 <= nz - 2 && fabsf(p.z - S.zh[kq + 1]) <= ek) || (kq >= 1 && fabsf(p.z - S.zh[kq]) <= ek)) {
              R.flag = true;
              continue;
            }
          }
          const int rr = radial_in(S, kq, p, false, false);
          if (rr == 0) { R.flag = true; continue; }
          if (rr < 0) continue;
          if (!wide) {
            const float* n2 = j == 0 ? S.neh : S.nsh;
            const float o = n2[0] * p.x + n2[1] * p.y;
            const float eo = 1.5f * p.e + 4.f * U * (fabsf(p.x) + fabsf(p.y)) + 1e-30f;
            if (fabsf(o) <= eo) { R.flag = true; continue; }
            if (o > 0) continue;
          }
          best = vmin(best, tc);
        }
      }
      if (!certified(best)) R.flag = true;
      R.din = best.v;
    }
  }
}

}  // namespace f32
}  // namespace gv
