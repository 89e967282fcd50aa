// work_class.cuh -- the work class of a track against a primitive solid, from the high parts
// of its binary64 words: the key by which the binary64 pass orders a basket (k_sort_classes).
#pragma once
#include "solid_fp32.cuh"

namespace gv {
namespace f32 {

// ------------------------------------------------------------- work classes
// The work class of a track against a primitive solid, for grouping tracks that take the same
// path through a pass (a plain binary32 estimate from the high parts: no result depends on
// it).  In the order the passes take them: outside points whose rays reach the solid's
// bounding volume (the box itself, the axis-aligned box around a trd or trap, the cylinder
// around the polycone family), inside points, points near a surface, outside points whose rays
// miss the bounding volume.  Without directions an outside point counts as missing.
enum : uint32_t { kClsHit = 0, kClsInside = 1, kClsNear = 2, kClsMiss = 3, kClasses = 4 };
__device__ __forceinline__ uint32_t track_class(const Desc& S, float x, float y, float z, float u, float v,
                                                float w, bool dirs) {
  float s;
  const bool pcon = S.type == kTube || S.type == kCone || S.type == kPcon;
  if (S.type == kBox) {
    s = fmaxf(fmaxf(fabsf(x) - S.Dh[0], fabsf(y) - S.Dh[1]), fabsf(z) - S.Dh[2]);
  } else if (!pcon) {  // trd, trap: four side planes and the z slab
    s = fabsf(z) - S.dzh;
    for (int i = 0; i < 4; i++) s = fmaxf(s, S.plh[i][0] * x + S.plh[i][1] * y + S.plh[i][2] * z - S.plh[i][3]);
  } else {
    const int last = S.nz - 1;
    const float r = sqrtf(x * x + y * y);
    int k = 0;
    while (k < last - 1 && z >= S.zh[k + 1]) k++;
    s = fmaxf(S.zh[0] - z, z - S.zh[last]);
    s = fmaxf(s, (r - fmaf(S.oah[k], z, S.obh[k])) * S.ok_[k]);
    if ((S.inner >> k) & 1u) s = fmaxf(s, (fmaf(S.iah[k], z, S.ibh[k]) - r) * S.ik_[k]);
    if (S.flags & kHasPhi) {
      const float pa = S.nsh[0] * x + S.nsh[1] * y, pb = S.neh[0] * x + S.neh[1] * y;
      s = fmaxf(s, (S.flags & kPhiWide) ? fminf(pa, pb) : fmaxf(pa, pb));
    }
  }
  if (fabsf(s) <= fmaf(1e-5f, S.size, 1e-6f)) return kClsNear;
  if (s < 0.f) return kClsInside;
  if (!dirs) return kClsMiss;
  if (!pcon) {  // slab test against the box [-ext, ext]
    const float p[3] = {x, y, z}, d[3] = {u, v, w};
    float lo = 0.f, hi = BIG;
    for (int i = 0; i < 3; i++) {
      const float e = (float)S.ext[i];
      if (d[i] == 0.f) {
        if (fabsf(p[i]) > e) return kClsMiss;
        continue;
      }
      const float ta = (-e - p[i]) / d[i], tb = (e - p[i]) / d[i];
      lo = fmaxf(lo, fminf(ta, tb));
      hi = fminf(hi, fmaxf(ta, tb));
    }
    return hi < lo ? kClsMiss : kClsHit;
  }
  const int last = S.nz - 1;
  float lo = 0.f, hi = BIG;
  if (w != 0.f) {
    const float ta = (S.zh[0] - z) / w, tb = (S.zh[last] - z) / w;
    lo = fmaxf(fminf(ta, tb), 0.f);
    hi = fmaxf(ta, tb);
    if (hi < lo) return kClsMiss;
  } else if (z < S.zh[0] || z > S.zh[last]) {
    return kClsMiss;
  }
  const float radial = x * u + y * v, A0 = u * u + v * v;
  const float tm = fminf(fmaxf(A0 > 0.f ? -radial / A0 : lo, lo), hi);
  const float Rb = (float)S.ext[0];
  return fmaf(fmaf(A0, tm, 2.f * radial), tm, x * x + y * y) > Rb * Rb ? kClsMiss : kClsHit;
}

}  // namespace f32
}  // namespace gv
