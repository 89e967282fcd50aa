// gv_desc.h -- solid descriptor shared by the host constructors and the kernels.
//
// One plain-old-data record per solid, uploaded once to device memory and staged
// in shared memory by every block that evaluates it.  The decision quantities
// (the constraint values whose maximum s decides inside / surface / outside) are
// formed from these fields with round-to-nearest binary64 operations in a fixed
// order and with no fused multiply-add, so that a code never depends on how the
// compiler schedules the arithmetic:
//
//   box        |x| - dx, |y| - dy, |z| - dz
//   trd, trap  ((nx*x + ny*y) + nz*z) - c for the four side planes, |z| - dz
//   tube       r - rmax, rmin - r (rmin > 0), |z| - dz, phi
//   cone/pcon  (r - (a*z + b))*k, ((a*z + b) - r)*k per section, z0 - z, z - zN, phi
//   phi        ns.p = ns0*x + ns1*y, ne.p likewise; max of the two for dphi <= pi,
//              min of the two for dphi > pi
//   r          sqrt(x*x + y*y)
#pragma once
#include <stdint.h>

namespace gv {

enum SolidType : int32_t { kBox = 0, kTrd = 1, kTrap = 2, kTube = 3, kCone = 4, kPcon = 5, kBool = 6 };
enum BoolOp : int32_t { kUnion = 0, kSubtraction = 1, kIntersection = 2 };

constexpr int kMaxZ = 32;            // polycone z-planes (GV_MAX_ZPLANES)
constexpr double kHalfTol = 0.5e-9;  // h = kTolerance / 2 (mm)
// Grazing rays: a derivative per unit length within kTangent of zero is tangent; crossings
// closer than kMerge (mm) are one crossing; a quadratic's discriminant within kDisc times its
// rounding scale is a double root (a touch).
constexpr double kTangent = 1e-12;
constexpr double kMerge = 1e-12;
constexpr double kDisc = 16 * 1.1102230246251565e-16;

// kFp64Only: the solid has a feature finer than 2^-16 of its size (a wall, a z-section, a phi
// wedge or the sliver a phi segment leaves out), which the binary32 passes cannot order reliably
// against its neighbours: every pass evaluates it in binary64 (as booleans).
enum : int32_t { kHasPhi = 1, kPhiWide = 2, kFp64Only = 4 };

struct Line {   // R(z) = a*z + b, k = 1 / sqrt(1 + a*a)
  double a, b, k;
};

struct alignas(16) Desc {
  int32_t type;
  int32_t nz;          // z-planes of the polycone family (2 for tube and cone)
  int32_t flags;       // kHasPhi | kPhiWide
  uint32_t inner;      // bit k: section k has an inner surface
  double D[3];         // box half-lengths
  double pl[4][4];     // trd/trap side planes (nx, ny, nz, c), outward unit normals
  double dz;           // half-length in z (box/trd/trap/tube/cone)
  double ns[2], ne[2]; // outward normals of the phi = sphi and phi = sphi + dphi planes
  double z[kMaxZ];     // polycone family z-planes
  Line out[kMaxZ - 1]; // outer surface of each section
  Line in[kMaxZ - 1];  // inner surface of each section (valid where `inner` has the bit)

  // Split constants for the binary32 pass: every binary64 constant v above is
  // also stored as hi = float(v) (round to nearest) and lo = float(v - hi), so
  // that v = hi + lo to about 2^-48 relative.
  float Dh[3], Dl[3];            // box half-lengths
  float plh[4][4], pll[4][4];    // side planes
  float dzh, dzl;
  float nsh[2], nsl[2], neh[2], nel[2];
  float zh[kMaxZ], zl[kMaxZ];
  long long zkey[kMaxZ];         // z-planes as order-preserving integers (exact comparisons)
  float oah[kMaxZ - 1], oal[kMaxZ - 1], obh[kMaxZ - 1], obl[kMaxZ - 1], ok_[kMaxZ - 1];
  float iah[kMaxZ - 1], ial[kMaxZ - 1], ibh[kMaxZ - 1], ibl[kMaxZ - 1], ik_[kMaxZ - 1];
  float size;                    // largest |coordinate| of the solid's extent (mm)

  // Boolean solids (type kBool): op(a, c) with c placed in a's frame by
  // p_a = bR p_c + bt (row-major); parts points to the two component records
  // (device memory owned by the boolean's handle).
  int32_t bop;
  int32_t bpad;
  double bR[9], bt[3];
  const Desc* parts;
  double ext[3];  // half-extents of an axis-aligned box around the origin holding the solid
};

// Order-preserving integer key of a binary64 bit pattern: for non-NaN a, b,
// a < b iff key(a) < key(b) and a == b iff key(a) == key(b) (-0 and +0 both map to 0).
__host__ __device__ inline long long order_key(long long bits) {
  return bits < 0 ? -(bits & 0x7FFFFFFFFFFFFFFFll) : bits;
}

}  // namespace gv
