/*
 * gv.h -- C ABI of the GB300 track-versus-solid geometry library.
 *
 * The paper (arXiv:1512.06637, VecGeom section) names three questions that the
 * geometry answers for every particle at every step:
 *   (1) is the particle inside or outside the solid?           -> Inside
 *   (2) what is its minimal distance to the border of the solid? -> SafetyToIn / SafetyToOut
 *   (3) how far may it move along its direction?              -> DistanceToIn / DistanceToOut
 * and evaluates them for whole "baskets" of particles that sit in the same kind
 * of volume at once (Project goals, item 1; VecGeom section).  This header is the
 * boundary of that hot path: a solid description and a structure-of-arrays
 * basket of points and directions go in; codes, distances and safeties come out.
 *
 * Conventions (they hold for every call below):
 *  - Units are mm and radians.  All track and result arrays are DEVICE pointers
 *    owned by the caller, FP64 (codes int8), one element per track, 8-byte
 *    aligned; directions are unit vectors (the library does not renormalise).
 *  - Inside codes: GV_INSIDE = 0, GV_SURFACE = 1, GV_OUTSIDE = 2.  The surface
 *    band is |s| <= h with h = 0.5e-9 mm (kTolerance = 1e-9 mm), where s is the
 *    largest of the solid's signed constraint distances.
 *  - A distance or safety asked from the wrong side is -1 (DistanceToIn and
 *    SafetyToIn of an INSIDE point; DistanceToOut and SafetyToOut of an OUTSIDE
 *    point).  A ray that never enters returns +inf.  A SURFACE point moving into
 *    the solid has DistanceToIn 0; one moving out has DistanceToOut 0.
 *  - Safeties are the largest signed constraint distance (a lower bound on the
 *    Euclidean distance to the border).
 *  - Every call returns a gv_status; GV_OK means the work was enqueued on the
 *    given CUDA stream (cudaStream_t passed as void*, NULL = legacy default
 *    stream).  Calls never synchronise the stream unless stated.  On failure
 *    gv_last_error() returns a message for the calling thread.  The library
 *    never aborts and never traps on the device.
 *  - Handles (solids, workspaces) are created and destroyed by the library.
 *    Solids are immutable after creation and may be shared between threads.
 */
#ifndef GV_H
#define GV_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GV_OK = 0,
  GV_ERR_INVALID_ARG = 1,   /* bad pointer, size or solid parameters           */
  GV_ERR_UNSUPPORTED = 2,   /* e.g. a polycone with more z-planes than allowed */
  GV_ERR_OUT_OF_MEMORY = 3, /* device or host allocation failed, or a workspace
                               too small for the request                        */
  GV_ERR_CUDA = 4,          /* a CUDA runtime call failed                        */
  GV_ERR_TIMEOUT = 5,
  GV_ERR_BUSY = 6
} gv_status;

enum { GV_INSIDE = 0, GV_SURFACE = 1, GV_OUTSIDE = 2 };

/* Arithmetic of a query pass.  GV_FP64: every quantity in binary64.
 * GV_FP32_REFINE: a binary32 bulk pass that flags every track whose result it
 * cannot certify (codes near the surface band, ill-conditioned roots, short
 * distances) and recomputes exactly those tracks in binary64.  Codes are
 * identical to GV_FP64; distances and safeties agree to 1e-5 relative
 * (1e-9 mm absolute below 1e-4 mm). */
typedef enum { GV_FP64 = 0, GV_FP32_REFINE = 1 } gv_precision;

#define GV_MAX_ZPLANES 32 /* largest polycone z-plane count */

typedef struct gv_solid gv_solid;         /* opaque, immutable */
typedef struct gv_workspace gv_workspace; /* opaque device scratch */

/* --- solids (Detector geometry subsection: rectangular solids, tubes and their
 *     relatives; parameters are half-lengths).  Each constructor validates its
 *     arguments (finite, positive sizes, ordered radii, 0 < dphi) and derives
 *     the host-side constants; *out receives a new handle. ----------------- */

/* Box: |x| <= dx, |y| <= dy, |z| <= dz. */
gv_status gv_solid_box(double dx, double dy, double dz, gv_solid** out);
/* Trd: x half-width dx1 at z = -dz growing linearly to dx2 at z = +dz; same for y. */
gv_status gv_solid_trd(double dx1, double dx2, double dy1, double dy2, double dz, gv_solid** out);
/* General trapezoid p[11] = (dz, theta, phi, dy1, dx1, dx2, alpha1, dy2, dx3, dx4, alpha2):
 * faces at z = -/+dz are trapezoids centred on the line of polar angle theta and
 * azimuth phi; dy1 is the y half-length at -dz, dx1 / dx2 the x half-lengths at
 * y = -dy1 / +dy1, alpha1 the shear (x offset y tan alpha1); dy2, dx3, dx4,
 * alpha2 the same at +dz.  Side faces must be planar (within 1e-9 mm). */
gv_status gv_solid_trap(const double p[11], gv_solid** out);
/* Tube segment: rmin <= r <= rmax, |z| <= dz, sphi <= phi <= sphi + dphi
 * (dphi >= 2 pi means a full tube; 0 <= rmin < rmax). */
gv_status gv_solid_tube(double rmin, double rmax, double dz, double sphi, double dphi,
                        gv_solid** out);
/* Cone segment: radii interpolate linearly from (rmin1, rmax1) at z = -dz to
 * (rmin2, rmax2) at z = +dz; phi as for the tube. */
gv_status gv_solid_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz,
                        double sphi, double dphi, gv_solid** out);
/* Polycone: nz z-planes (2 <= nz <= GV_MAX_ZPLANES, strictly increasing) with
 * 0 <= rmin[k] < rmax[k]; radii interpolate linearly between planes.  The
 * arrays are host memory and are copied. */
gv_status gv_solid_polycone(int nz, const double* z, const double* rmin, const double* rmax,
                            double sphi, double dphi, gv_solid** out);
void gv_solid_destroy(gv_solid* s);

/* --- baskets ------------------------------------------------------------ */

typedef struct {
  const double *x, *y, *z;    /* points                (device, n each) */
  const double *dx, *dy, *dz; /* unit directions       (device, n each) */
  int64_t n;                  /* number of tracks, >= 0                 */
} gv_tracks;

/* Any pointer may be NULL to skip that query. */
typedef struct {
  int8_t* inside;
  double *dist_in, *dist_out, *safety_in, *safety_out;
} gv_results;

/* --- device scratch for the FP32 + refinement pass ---------------------- */

/* Allocates (cudaMalloc, on the current device) scratch for baskets of up to
 * max_tracks tracks: the refinement worklist (4 bytes per track) and a counter. */
gv_status gv_workspace_create(int64_t max_tracks, gv_workspace** out);
void gv_workspace_destroy(gv_workspace* ws);
/* Number of tracks the last GV_FP32_REFINE query on this workspace sent to the
 * binary64 refinement (reads a device counter: synchronises `stream`). */
gv_status gv_workspace_refined(gv_workspace* ws, void* stream, int64_t* n_refined);

/* --- the queries --------------------------------------------------------- */

/* All requested queries for one basket against one solid (VecGeom section, the
 * three questions).  ws may be NULL for GV_FP64 and must hold >= tracks->n for
 * GV_FP32_REFINE.  Asynchronous on `stream`. */
gv_status gv_query(const gv_solid* s, const gv_tracks* tracks, gv_precision prec,
                   const gv_results* res, gv_workspace* ws, void* stream);

/* Thread-local description of the last error on this thread ("" if none). */
const char* gv_last_error(void);
/* Library version string. */
const char* gv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GV_H */
