/*
 * gv_oracle.c -- CPU oracle for the geometry queries and the navigation step.
 *
 * TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the CUDA library.  It shares no code with
 * the library.  Every quantity is IEEE binary64; the file is compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * What it computes (the three questions of the VecGeom section, the navigation step
 * of the Physics / Detector geometry subsections, and the transport loop of the
 * Physics subsection, see or_transport):
 *
 *   Each solid is a set of constraints g_i(p) (in mm, negative = satisfied).
 *   s(p) = max_i g_i(p) is the decision quantity.  The point is INSIDE if
 *   s < -h, OUTSIDE if s > h, SURFACE otherwise, with h = 0.5e-9 mm.
 *
 *   Safety:   SafetyToIn  = s  (OUTSIDE), 0 (SURFACE), -1 (INSIDE, wrong side)
 *             SafetyToOut = -s (INSIDE),  0 (SURFACE), -1 (OUTSIDE)
 *             (polycone: per-section closed constraint sets, see below).
 *
 *   Distance: every root t > 0 of every constraint surface along p + t d is a
 *   candidate (roots closer than 1e-12 mm merged); the gaps between consecutive
 *   candidates are classified inside or outside by the sign of s at their
 *   midpoint (no tolerance).
 *   DistanceToIn:  INSIDE -> -1; SURFACE and entering -> 0; otherwise the first
 *                  candidate where an outside gap is followed by an inside one;
 *                  none -> +inf.
 *   DistanceToOut: OUTSIDE -> -1; SURFACE and not entering -> 0; otherwise the
 *                  first candidate where an inside gap is followed by an outside
 *                  one; none (a surface point whose ray never gets inside) -> 0.
 *   A SURFACE point is "entering" when every constraint within the band
 *   (g_i >= -h) shrinks along d.  Rays that graze or run along a surface follow
 *   the readings stated above the surface-start code below (tangent, sliding,
 *   touch).
 */
#include "gv_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define H OR_HALF_TOL
#define MAXROOTS 1024  /* two polycones of OR_MAXZ planes at most (booleans) */

int or_solid_size(void) { return (int)sizeof(or_solid); }
int or_bool_size(void) { return (int)sizeof(or_bool); }

/* ------------------------------------------------------------ boolean solids */

int or_setup_bool(int op, const or_solid* a, const or_solid* c, const double R[9], const double t[3],
                  or_bool* b, or_solid* s) {
  if (op < OR_UNION || op > OR_INTERSECTION || !a || !c) return -1;
  if (a->type == OR_BOOL || c->type == OR_BOOL) return -1;  /* components are primitives */
  for (int i = 0; i < 9; i++) if (!isfinite(R[i])) return -1;
  for (int i = 0; i < 3; i++) if (!isfinite(t[i])) return -1;
  memset(b, 0, sizeof(*b));
  b->op = op;
  b->a = *a;
  b->c = *c;
  memcpy(b->R, R, sizeof(b->R));
  memcpy(b->t, t, sizeof(b->t));
  memset(s, 0, sizeof(*s));
  s->type = OR_BOOL;
  s->family = 2;
  s->bl = b;
  return 0;
}

/* a's frame -> c's frame: p_c = R^T (p - t), d_c = R^T d */
static void bool_to_c(const or_bool* b, const double p[3], const double d[3], double pc[3], double dc[3]) {
  const double v[3] = {p[0] - b->t[0], p[1] - b->t[1], p[2] - b->t[2]};
  for (int i = 0; i < 3; i++) {
    pc[i] = (b->R[0 * 3 + i] * v[0] + b->R[1 * 3 + i] * v[1]) + b->R[2 * 3 + i] * v[2];
    if (d) dc[i] = (b->R[0 * 3 + i] * d[0] + b->R[1 * 3 + i] * d[1]) + b->R[2 * 3 + i] * d[2];
  }
}

/* The decision quantity of op(a, c) from those of its components: union min, intersection
 * max, subtraction max(s_a, -s_c) (inside a and outside c). */
static double bool_combine(int op, double sa, double sc) {
  if (op == OR_UNION) return sa < sc ? sa : sc;
  if (op == OR_INTERSECTION) return sa > sc ? sa : sc;
  return sa > -sc ? sa : -sc;
}

/* ------------------------------------------------------------------ setup */

static void set_plane(or_plane* P, double nx, double ny, double nz, double c) {
  P->n[0] = nx; P->n[1] = ny; P->n[2] = nz; P->c = c;
}

static double dot3(const double a[3], const double b[3]) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

int or_setup_box(double dx, double dy, double dz, or_solid* s) {
  if (!(dx > 0 && dy > 0 && dz > 0) || !isfinite(dx + dy + dz)) return -1;
  memset(s, 0, sizeof(*s));
  s->type = OR_BOX; s->family = 0; s->nplanes = 6;
  set_plane(&s->pl[0], 0, 0, -1, dz);
  set_plane(&s->pl[1], 0, 0, 1, dz);
  set_plane(&s->pl[2], 0, -1, 0, dy);
  set_plane(&s->pl[3], 0, 1, 0, dy);
  set_plane(&s->pl[4], -1, 0, 0, dx);
  set_plane(&s->pl[5], 1, 0, 0, dx);
  return 0;
}

/* A side face through the quad (A, B, C, D): normal from the cross product of
 * the diagonals, oriented away from the solid's vertex centroid, normalised;
 * the offset is the mean of n.V over the four vertices. */
static int face_plane(const double A[3], const double B[3], const double C[3],
                      const double D[3], const double cs[3], or_plane* P) {
  double u[3], w[3], n[3], cf[3], e[3];
  for (int i = 0; i < 3; i++) { u[i] = C[i] - A[i]; w[i] = D[i] - B[i]; }
  n[0] = u[1] * w[2] - u[2] * w[1];
  n[1] = u[2] * w[0] - u[0] * w[2];
  n[2] = u[0] * w[1] - u[1] * w[0];
  for (int i = 0; i < 3; i++) { cf[i] = ((A[i] + B[i]) + (C[i] + D[i])) * 0.25; e[i] = cf[i] - cs[i]; }
  if (dot3(n, e) < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  double len = sqrt(dot3(n, n));
  if (!(len > 0)) return -1;
  for (int i = 0; i < 3; i++) n[i] = n[i] / len;
  double c = ((dot3(n, A) + dot3(n, B)) + (dot3(n, C) + dot3(n, D))) * 0.25;
  const double* V[4] = {A, B, C, D};
  for (int i = 0; i < 4; i++)
    if (fabs(dot3(n, V[i]) - c) > 1e-9) return -1; /* not planar */
  set_plane(P, n[0], n[1], n[2], c);
  return 0;
}

/* General trapezoid, parameters (dz, theta, phi, dy1, dx1, dx2, alpha1,
 * dy2, dx3, dx4, alpha2): the faces at z = -dz and z = +dz are trapezoids
 * whose centres lie on the line of polar angle theta and azimuth phi through
 * the origin; on the face at -dz the half-length in y is dy1, the half-lengths
 * in x at y = -dy1 and y = +dy1 are dx1 and dx2, and the face is sheared by
 * alpha1 (x offset y tan alpha1); likewise dy2, dx3, dx4, alpha2 at +dz. */
int or_setup_trap(const double p[11], or_solid* s) {
  const double dz = p[0], th = p[1], ph = p[2];
  for (int i = 0; i < 11; i++) if (!isfinite(p[i])) return -1;
  if (!(dz > 0 && p[3] > 0 && p[4] > 0 && p[5] > 0 && p[7] > 0 && p[8] > 0 && p[9] > 0)) return -1;
  if (!(fabs(th) < 1.5707963267948966 && fabs(p[6]) < 1.5707963267948966 &&
        fabs(p[10]) < 1.5707963267948966)) return -1;
  memset(s, 0, sizeof(*s));
  s->type = OR_TRAP; s->family = 0; s->nplanes = 6;
  const double tthc = tan(th) * cos(ph), tths = tan(th) * sin(ph);
  double v[8][3];
  for (int j = 0; j < 2; j++) {
    const double zf = j == 0 ? -dz : dz;
    const double dy = j == 0 ? p[3] : p[7];
    const double dxa = j == 0 ? p[4] : p[8];
    const double dxb = j == 0 ? p[5] : p[9];
    const double ta = tan(j == 0 ? p[6] : p[10]);
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
  set_plane(&s->pl[0], 0, 0, -1, dz);
  set_plane(&s->pl[1], 0, 0, 1, dz);
  if (face_plane(v[0], v[1], v[5], v[4], cs, &s->pl[2])) return -1; /* -y */
  if (face_plane(v[2], v[6], v[7], v[3], cs, &s->pl[3])) return -1; /* +y */
  if (face_plane(v[0], v[4], v[6], v[2], cs, &s->pl[4])) return -1; /* -x */
  if (face_plane(v[1], v[3], v[7], v[5], cs, &s->pl[5])) return -1; /* +x */
  return 0;
}

int or_setup_trd(double dx1, double dx2, double dy1, double dy2, double dz, or_solid* s) {
  const double p[11] = {dz, 0, 0, dy1, dx1, dx1, 0, dy2, dx2, dx2, 0};
  int rc = or_setup_trap(p, s);
  if (rc == 0) s->type = OR_TRD;
  return rc;
}

static void set_line(or_line* L, double r0, double r1, double z0, double z1) {
  L->a = (r1 - r0) / (z1 - z0);
  L->b = r0 - L->a * z0;
  L->k = 1.0 / sqrt(1.0 + L->a * L->a);
}

int or_setup_pcon(int nz, const double* z, const double* rmin, const double* rmax,
                  double sphi, double dphi, or_solid* s) {
  if (nz < 2 || nz > OR_MAXZ) return -1;
  if (!isfinite(sphi) || !isfinite(dphi) || !(dphi > 0)) return -1;
  for (int k = 0; k < nz; k++) {
    if (!isfinite(z[k]) || !isfinite(rmin[k]) || !isfinite(rmax[k])) return -1;
    if (!(rmin[k] >= 0 && rmin[k] < rmax[k])) return -1;
    if (k > 0 && !(z[k] > z[k - 1])) return -1;
  }
  memset(s, 0, sizeof(*s));
  s->type = OR_PCON; s->family = 1; s->nz = nz;
  for (int k = 0; k < nz; k++) s->z[k] = z[k];
  for (int k = 0; k + 1 < nz; k++) {
    set_line(&s->out[k], rmax[k], rmax[k + 1], z[k], z[k + 1]);
    s->out[k].present = 1;
    set_line(&s->in[k], rmin[k], rmin[k + 1], z[k], z[k + 1]);
    s->in[k].present = (rmin[k] > 0 || rmin[k + 1] > 0);
  }
  const double twopi = 6.283185307179586, pi = 3.141592653589793;
  s->has_phi = dphi < twopi;
  s->phi_wide = dphi > pi;
  const double ephi = sphi + dphi;
  s->ns[0] = sin(sphi);  s->ns[1] = -cos(sphi);
  s->ne[0] = -sin(ephi); s->ne[1] = cos(ephi);
  return 0;
}

int or_setup_tube(double rmin, double rmax, double dz, double sphi, double dphi, or_solid* s) {
  if (!(dz > 0)) return -1;
  const double z[2] = {-dz, dz}, rn[2] = {rmin, rmin}, rx[2] = {rmax, rmax};
  int rc = or_setup_pcon(2, z, rn, rx, sphi, dphi, s);
  if (rc == 0) s->type = OR_TUBE;
  return rc;
}

int or_setup_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz,
                  double sphi, double dphi, or_solid* s) {
  if (!(dz > 0)) return -1;
  const double z[2] = {-dz, dz}, rn[2] = {rmin1, rmin2}, rx[2] = {rmax1, rmax2};
  int rc = or_setup_pcon(2, z, rn, rx, sphi, dphi, s);
  if (rc == 0) s->type = OR_CONE;
  return rc;
}

/* ------------------------------------------------------ constraint values */

static double plane_g(const or_plane* P, const double p[3]) {
  return ((P->n[0] * p[0] + P->n[1] * p[1]) + P->n[2] * p[2]) - P->c;
}
static double line_out_g(const or_line* L, double r, double z) { return (r - (L->a * z + L->b)) * L->k; }
static double line_in_g(const or_line* L, double r, double z) { return ((L->a * z + L->b) - r) * L->k; }
static double rho(const double p[3]) { return sqrt(p[0] * p[0] + p[1] * p[1]); }
static double phi_plane(const double n[2], const double p[3]) { return n[0] * p[0] + n[1] * p[1]; }

static double phi_g(const or_solid* s, const double p[3]) {
  const double a = phi_plane(s->ns, p), b = phi_plane(s->ne, p);
  return s->phi_wide ? (a < b ? a : b) : (a > b ? a : b);
}

static int section_of(const or_solid* s, double z) {
  int k = 0;
  while (k < s->nz - 2 && z >= s->z[k + 1]) k++;
  return k;
}

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

double or_s_code(const or_solid* s, const double p[3]) {
  if (s->type == OR_BOOL) {
    double pc[3];
    bool_to_c(s->bl, p, NULL, pc, NULL);
    return bool_combine(s->bl->op, or_s_code(&s->bl->a, p), or_s_code(&s->bl->c, pc));
  }
  if (s->family == 0) {
    double v = plane_g(&s->pl[0], p);
    for (int i = 1; i < s->nplanes; i++) v = dmax(v, plane_g(&s->pl[i], p));
    return v;
  }
  const double r = rho(p), z = p[2];
  const int k = section_of(s, z);
  double v = line_out_g(&s->out[k], r, z);
  v = dmax(v, s->z[0] - z);
  v = dmax(v, z - s->z[s->nz - 1]);
  if (s->in[k].present) v = dmax(v, line_in_g(&s->in[k], r, z));
  if (s->has_phi) v = dmax(v, phi_g(s, p));
  return v;
}

/* Polycone section k as a closed piece, its own z-planes included. */
static double s_closed(const or_solid* s, int k, const double p[3]) {
  const double r = rho(p), z = p[2];
  double v = line_out_g(&s->out[k], r, z);
  v = dmax(v, s->z[k] - z);
  v = dmax(v, z - s->z[k + 1]);
  if (s->in[k].present) v = dmax(v, line_in_g(&s->in[k], r, z));
  if (s->has_phi) v = dmax(v, phi_g(s, p));
  return v;
}

static int code_of(double v) { return v < -H ? OR_INSIDE : (v > H ? OR_OUTSIDE : OR_SURFACE); }

int or_inside(const or_solid* s, const double p[3]) { return code_of(or_s_code(s, p)); }

/* Safeties of op(a, c) from the components' own safeties (lower bounds on their
 * distances): leaving a union means leaving every component the point is in, entering an
 * intersection means entering every component it is outside of, a subtraction is a and
 * not-c (SafetyToIn of not-c is SafetyToOut of c, and the reverse). */
static double bool_safety(const or_bool* b, const double p[3], int to_in) {
  double pc[3];
  bool_to_c(b, p, NULL, pc, NULL);
  const int ca = or_inside(&b->a, p), cc = or_inside(&b->c, pc);
  const double sia = or_safety_in(&b->a, p), soa = or_safety_out(&b->a, p);
  const double sic = or_safety_in(&b->c, pc), soc = or_safety_out(&b->c, pc);
  double v = -INFINITY;
  if (b->op == OR_UNION) {
    if (to_in) return dmin(sia, sic);
    if (ca == OR_INSIDE) v = dmax(v, soa);
    if (cc == OR_INSIDE) v = dmax(v, soc);
  } else if (b->op == OR_INTERSECTION) {
    if (!to_in) return dmin(soa, soc);
    if (ca == OR_OUTSIDE) v = dmax(v, sia);
    if (cc == OR_OUTSIDE) v = dmax(v, sic);
  } else {
    if (!to_in) return dmin(soa, sic);
    if (ca == OR_OUTSIDE) v = dmax(v, sia);
    if (cc == OR_INSIDE) v = dmax(v, soc);
  }
  return v;
}

double or_safety_in(const or_solid* s, const double p[3]) {
  const double v = or_s_code(s, p);
  const int c = code_of(v);
  if (c == OR_INSIDE) return -1.0;
  if (c == OR_SURFACE) return 0.0;
  if (s->type == OR_BOOL) return bool_safety(s->bl, p, 1);
  if (s->family == 0) return v;
  double best = s_closed(s, 0, p);
  for (int k = 1; k + 1 < s->nz; k++) best = dmin(best, s_closed(s, k, p));
  return best;
}

double or_safety_out(const or_solid* s, const double p[3]) {
  const double v = or_s_code(s, p);
  const int c = code_of(v);
  if (c == OR_OUTSIDE) return -1.0;
  if (c == OR_SURFACE) return 0.0;
  if (s->type == OR_BOOL) return bool_safety(s->bl, p, 0);
  if (s->family == 0) return -v;
  return -s_closed(s, section_of(s, p[2]), p);
}

/* ------------------------------------------- rays along and across surfaces */

/* Readings for rays that meet a surface at a grazing angle (the paper gives none):
 *
 * Tangent.  The derivative along d of a constraint that holds the start point within the
 * band is taken per unit length (plane and phi normals are unit vectors, a lateral wall
 * r = a z + b gives (d r/dt - a d_z) k).  Within OR_TAU of zero it is tangent: a tangent
 * plane is one the ray runs along; a tangent wall curves away from the ray unless the ray
 * lies in the meridian plane of the point (|p_xy x d_xy| <= OR_TAU r), where it runs along
 * a straight generator of the wall.  A convex (outer) wall that curves away is left, a
 * concave (inner) one is entered.
 *
 * Sliding.  A constraint within the band whose surface the ray runs along (a tangent
 * plane, or a wall along its generator) slides: along the ray the point stays on that
 * surface, which is the boundary and not the interior.  It has no crossing of its own,
 * and its value along the ray is taken as violated (+inf; -inf for the subtracted solid
 * of a boolean subtraction, whose complement it bounds).
 *
 * Surface start.  A point on the surface enters when every constraint within the band
 * shrinks along d (tangent concave walls included); otherwise the ray does not get into
 * the interior at 0+, and DistanceToOut is 0.
 *
 * Touch.  A wall crossed where the quadratic's discriminant is within its rounding bound
 * of zero is touched (a double root): no crossing.  Crossings closer
 * than OR_MERGE mm are one crossing: a chord shorter than that is a touch. */
#define OR_TAU 1e-12
#define OR_MERGE 1e-12
#define OR_DISC (16 * 1.1102230246251565e-16)

enum { SL_OUT = 1, SL_IN = 2, SL_Z0 = 4, SL_ZL = 8, SL_PS = 16, SL_PE = 32 };

/* The sliding constraints of one primitive along one ray. */
typedef struct {
  unsigned bits;  /* planar: bit i = plane i; polycone family: SL_* */
  int k0;         /* polycone family: the start point's section (its walls slide) */
  double forced;  /* the value a sliding constraint takes along the ray */
} slide1;

typedef struct { slide1 a, c; } or_slide;  /* a primitive uses a; a boolean a and c */

/* One constraint at the start point: value, derivative per unit length along d, motion
 * (+1 grows, -1 shrinks, 0 runs along its surface), sliding bit, and whether it takes
 * part in the surface-start rule (a wide phi uses the plane holding the smaller value). */
typedef struct { double g, gd; int m; unsigned bit; int motion; } cons;

static int plane_motion(double gd) { return gd > OR_TAU ? 1 : (gd < -OR_TAU ? -1 : 0); }

static double wall_gd(const or_line* L, const double p[3], const double d[3], double r) {
  const double rd = r > 0 ? (p[0] * d[0] + p[1] * d[1]) / r : sqrt(d[0] * d[0] + d[1] * d[1]);
  return (rd - L->a * d[2]) * L->k;
}

static int wall_motion(double gd, const double p[3], const double d[3], double r, int outer) {
  if (gd > OR_TAU) return 1;
  if (gd < -OR_TAU) return -1;
  if (r > 0 && fabs(p[0] * d[1] - p[1] * d[0]) > OR_TAU * r) return outer ? 1 : -1;
  return 0;
}

/* The constraints of a primitive at its start point p along d. */
static int start_constraints(const or_solid* s, const double p[3], const double d[3], cons* c, int* k0) {
  int m = 0;
  *k0 = 0;
  if (s->family == 0) {
    for (int i = 0; i < s->nplanes; i++) {
      c[m].g = plane_g(&s->pl[i], p);
      c[m].gd = dot3(s->pl[i].n, d);
      c[m].m = plane_motion(c[m].gd);
      c[m].bit = 1u << i;
      c[m].motion = 1;
      m++;
    }
    return m;
  }
  const double r = rho(p), z = p[2];
  const int k = section_of(s, z);
  *k0 = k;
  c[m].g = line_out_g(&s->out[k], r, z);
  c[m].gd = wall_gd(&s->out[k], p, d, r);
  c[m].m = wall_motion(c[m].gd, p, d, r, 1);
  c[m].bit = SL_OUT; c[m].motion = 1; m++;
  if (s->in[k].present) {
    c[m].g = line_in_g(&s->in[k], r, z);
    c[m].gd = -wall_gd(&s->in[k], p, d, r);
    c[m].m = wall_motion(c[m].gd, p, d, r, 0);
    c[m].bit = SL_IN; c[m].motion = 1; m++;
  }
  c[m].g = s->z[0] - z; c[m].gd = -d[2]; c[m].m = plane_motion(c[m].gd); c[m].bit = SL_Z0; c[m].motion = 1; m++;
  c[m].g = z - s->z[s->nz - 1]; c[m].gd = d[2]; c[m].m = plane_motion(c[m].gd); c[m].bit = SL_ZL; c[m].motion = 1; m++;
  if (s->has_phi) {
    const double a = phi_plane(s->ns, p), b = phi_plane(s->ne, p);
    c[m].g = a; c[m].gd = phi_plane(s->ns, d); c[m].m = plane_motion(c[m].gd); c[m].bit = SL_PS;
    c[m].motion = !s->phi_wide || a <= b; m++;
    c[m].g = b; c[m].gd = phi_plane(s->ne, d); c[m].m = plane_motion(c[m].gd); c[m].bit = SL_PE;
    c[m].motion = !s->phi_wide || !(a <= b); m++;
  }
  return m;
}

static void slide_setup1(const or_solid* s, const double p[3], const double d[3], double forced, slide1* sl) {
  cons c[8];
  int k0;
  const int m = start_constraints(s, p, d, c, &k0);
  sl->bits = 0;
  sl->k0 = k0;
  sl->forced = forced;
  for (int i = 0; i < m; i++)
    if (fabs(c[i].g) <= H && c[i].m == 0) sl->bits |= c[i].bit;
}

static void slide_setup(const or_solid* s, const double p[3], const double d[3], or_slide* sl) {
  if (s->type == OR_BOOL) {
    double pc[3], dc[3];
    bool_to_c(s->bl, p, d, pc, dc);
    slide_setup1(&s->bl->a, p, d, INFINITY, &sl->a);
    slide_setup1(&s->bl->c, pc, dc, s->bl->op == OR_SUBTRACTION ? -INFINITY : INFINITY, &sl->c);
  } else {
    slide_setup1(s, p, d, INFINITY, &sl->a);
  }
}

/* The decision quantity at q along a ray, sliding constraints at their forced value. */
static double s_ray1(const or_solid* s, const double q[3], const slide1* sl) {
  if (s->family == 0) {
    double v = -INFINITY;
    for (int i = 0; i < s->nplanes; i++)
      v = dmax(v, (sl->bits >> i) & 1u ? sl->forced : plane_g(&s->pl[i], q));
    return v;
  }
  const double r = rho(q), z = q[2];
  const int k = section_of(s, z);
  const int own = k == sl->k0;
  double v = own && (sl->bits & SL_OUT) ? sl->forced : line_out_g(&s->out[k], r, z);
  v = dmax(v, sl->bits & SL_Z0 ? sl->forced : s->z[0] - z);
  v = dmax(v, sl->bits & SL_ZL ? sl->forced : z - s->z[s->nz - 1]);
  if (s->in[k].present) v = dmax(v, own && (sl->bits & SL_IN) ? sl->forced : line_in_g(&s->in[k], r, z));
  if (s->has_phi) {
    const double a = sl->bits & SL_PS ? sl->forced : phi_plane(s->ns, q);
    const double b = sl->bits & SL_PE ? sl->forced : phi_plane(s->ne, q);
    v = dmax(v, s->phi_wide ? dmin(a, b) : dmax(a, b));
  }
  return v;
}

static double s_ray(const or_solid* s, const double q[3], const or_slide* sl) {
  if (s->type != OR_BOOL) return s_ray1(s, q, &sl->a);
  double qc[3];
  bool_to_c(s->bl, q, NULL, qc, NULL);
  return bool_combine(s->bl->op, s_ray1(&s->bl->a, q, &sl->a), s_ray1(&s->bl->c, qc, &sl->c));
}

/* ------------------------------------------- surface start: does the ray enter? */

static int entering_of(const or_solid* s, const double p[3], const double d[3]);

/* A boolean surface point: over the components within the band |s_x| <= h, each with its
 * own rule (the complement of c, for a subtraction, is entered where c is certainly left:
 * some constraint of c within the band grows): a union is entered when some band component
 * is entered; an intersection (and a subtraction, a n not-c) when every band component is. */
static int bool_entering(const or_bool* b, const double p[3], const double d[3]) {
  double pc[3], dc[3];
  bool_to_c(b, p, d, pc, dc);
  const double sa = or_s_code(&b->a, p), sc = or_s_code(&b->c, pc);
  const int ba = fabs(sa) <= H, bc = fabs(sc) <= H;
  const int ea = ba && entering_of(&b->a, p, d);
  int ec = 0;
  if (bc) {
    if (b->op == OR_SUBTRACTION) {
      cons c[8];
      int k0;
      const int m = start_constraints(&b->c, pc, dc, c, &k0);
      for (int i = 0; i < m; i++)
        if (c[i].motion && c[i].g >= -H && c[i].m == 1) ec = 1;
    } else {
      ec = entering_of(&b->c, pc, dc);
    }
  }
  if (b->op == OR_UNION) return (ba && ea) || (bc && ec);
  return (!ba || ea) && (!bc || ec);
}

static int entering_of(const or_solid* s, const double p[3], const double d[3]) {
  if (s->type == OR_BOOL) return bool_entering(s->bl, p, d);
  cons c[8];
  int k0;
  const int m = start_constraints(s, p, d, c, &k0);
  for (int i = 0; i < m; i++)
    if (c[i].motion && c[i].g >= -H && c[i].m != -1) return 0;
  return 1;
}

/* ------------------------------------------------- candidate crossings */

static void add_root(double* t, int* m, double v) {
  if (v > 0 && isfinite(v) && *m < MAXROOTS) t[(*m)++] = v;
}

/* Crossings of the surface r = a z + b (a z + b >= 0) by p + t d: the roots of
 * A t^2 + 2 B t + C = 0, by the cancellation-free pair q/A, C/q.  A discriminant within
 * its rounding bound, OR_DISC (|B| Bs + |A| Cs + |C| As) with As, Bs, Cs the magnitudes of
 * the terms A, B, C are formed from, is a double root (a touch, no crossing). */
static void cone_roots(const or_line* L, const double p[3], const double d[3], double* t, int* m) {
  const double P = L->a * p[2] + L->b, D = L->a * d[2];
  const double A0 = d[0] * d[0] + d[1] * d[1], R2 = p[0] * p[0] + p[1] * p[1];
  const double A = A0 - D * D;
  const double B = (p[0] * d[0] + p[1] * d[1]) - P * D;
  const double C = R2 - P * P;
  double r[2]; int nr = 0;
  if (A == 0) {
    if (B != 0) r[nr++] = -C / (2 * B);
  } else {
    const double disc = B * B - A * C;
    const double As = A0 + D * D, Cs = R2 + P * P;
    const double Bs = (fabs(p[0] * d[0]) + fabs(p[1] * d[1])) + fabs(P * D);
    if (disc > OR_DISC * ((fabs(B) * Bs + fabs(A) * Cs) + fabs(C) * As)) {
      const double sq = sqrt(disc);
      const double q = -(B + (B >= 0 ? sq : -sq));
      r[nr++] = q / A;
      if (q != 0) r[nr++] = C / q;
    }
  }
  for (int i = 0; i < nr; i++) {
    const double zr = p[2] + r[i] * d[2];
    if (L->a * zr + L->b >= 0) add_root(t, m, r[i]);
  }
}

static void plane_root(const double n[3], double c, const double p[3], const double d[3],
                       double* t, int* m) {
  const double nd = dot3(n, d);
  if (nd != 0) add_root(t, m, (c - dot3(n, p)) / nd);
}

static int cmp_double(const void* a, const void* b) {
  const double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Every crossing of a primitive's constraint surfaces except those of its sliding ones. */
static int prim_roots(const or_solid* s, const double p[3], const double d[3], const slide1* sl, double* t) {
  int m = 0;
  if (s->family == 0) {
    for (int i = 0; i < s->nplanes; i++)
      if (!((sl->bits >> i) & 1u)) plane_root(s->pl[i].n, s->pl[i].c, p, d, t, &m);
    return m;
  }
  for (int k = 0; k + 1 < s->nz; k++) {
    const int own = k == sl->k0;
    if (!(own && (sl->bits & SL_OUT))) cone_roots(&s->out[k], p, d, t, &m);
    if (s->in[k].present && !(own && (sl->bits & SL_IN))) cone_roots(&s->in[k], p, d, t, &m);
  }
  const double ez[3] = {0, 0, 1};
  for (int k = 0; k < s->nz; k++) {
    if (k == 0 && (sl->bits & SL_Z0)) continue;
    if (k == s->nz - 1 && (sl->bits & SL_ZL)) continue;
    plane_root(ez, s->z[k], p, d, t, &m);
  }
  if (s->has_phi) {
    const double n1[3] = {s->ns[0], s->ns[1], 0}, n2[3] = {s->ne[0], s->ne[1], 0};
    if (!(sl->bits & SL_PS)) plane_root(n1, 0, p, d, t, &m);
    if (!(sl->bits & SL_PE)) plane_root(n2, 0, p, d, t, &m);
  }
  return m;
}

/* The crossings along the ray, sorted; crossings closer than OR_MERGE to the last one
 * kept are merged into it. */
static int candidates(const or_solid* s, const double p[3], const double d[3], const or_slide* sl, double* t) {
  int m;
  if (s->type == OR_BOOL) {  /* every crossing of either component's surfaces */
    double pc[3], dc[3];
    bool_to_c(s->bl, p, d, pc, dc);
    m = prim_roots(&s->bl->a, p, d, &sl->a, t);
    m += prim_roots(&s->bl->c, pc, dc, &sl->c, t + m);
  } else {
    m = prim_roots(s, p, d, &sl->a, t);
  }
  qsort(t, (size_t)m, sizeof(double), cmp_double);
  int u = 0;
  for (int i = 0; i < m; i++)
    if (u == 0 || t[i] - t[u - 1] > OR_MERGE) t[u++] = t[i];
  return u;
}

/* Inside (no tolerance) on the gap that follows candidate j-1 (gap 0 starts at t = 0). */
static int gap_inside(const or_solid* s, const double p[3], const double d[3], const or_slide* sl,
                      const double* t, int m, int j) {
  const double lo = j == 0 ? 0.0 : t[j - 1];
  const double mid = j < m ? 0.5 * (lo + t[j]) : 2.0 * lo + 1.0;
  const double q[3] = {p[0] + mid * d[0], p[1] + mid * d[1], p[2] + mid * d[2]};
  return s_ray(s, q, sl) <= 0;
}

double or_dist_in(const or_solid* s, const double p[3], const double d[3]) {
  const int c = or_inside(s, p);
  if (c == OR_INSIDE) return -1.0;
  if (c == OR_SURFACE && entering_of(s, p, d)) return 0.0;
  or_slide sl;
  slide_setup(s, p, d, &sl);
  double t[MAXROOTS];
  const int m = candidates(s, p, d, &sl, t);
  int prev = gap_inside(s, p, d, &sl, t, m, 0);
  for (int j = 1; j <= m; j++) {
    const int cur = gap_inside(s, p, d, &sl, t, m, j);
    if (cur && !prev) return t[j - 1];
    prev = cur;
  }
  return INFINITY;
}

double or_dist_out(const or_solid* s, const double p[3], const double d[3]) {
  const int c = or_inside(s, p);
  if (c == OR_OUTSIDE) return -1.0;
  if (c == OR_SURFACE && !entering_of(s, p, d)) return 0.0;
  or_slide sl;
  slide_setup(s, p, d, &sl);
  double t[MAXROOTS];
  const int m = candidates(s, p, d, &sl, t);
  int prev = gap_inside(s, p, d, &sl, t, m, 0);
  for (int j = 1; j <= m; j++) {
    const int cur = gap_inside(s, p, d, &sl, t, m, j);
    if (!cur && prev) return t[j - 1];
    prev = cur;
  }
  /* never inside: a surface point whose ray stays out leaves at once */
  return 0.0;
}

void or_query(const or_solid* s, int64_t n,
              const double* x, const double* y, const double* z,
              const double* dx, const double* dy, const double* dz,
              int8_t* inside, double* dist_in, double* dist_out,
              double* safety_in, double* safety_out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (int64_t i = 0; i < n; i++) {
    const double p[3] = {x[i], y[i], z[i]};
    if (inside) inside[i] = (int8_t)or_inside(s, p);
    if (safety_in) safety_in[i] = or_safety_in(s, p);
    if (safety_out) safety_out[i] = or_safety_out(s, p);
    if (dist_in || dist_out) {
      const double d[3] = {dx[i], dy[i], dz[i]};
      if (dist_in) dist_in[i] = or_dist_in(s, p, d);
      if (dist_out) dist_out[i] = or_dist_out(s, p, d);
    }
  }
}

void or_s_code_n(const or_solid* s, int64_t n, const double* x, const double* y,
                 const double* z, double* out) {
  for (int64_t i = 0; i < n; i++) {
    const double p[3] = {x[i], y[i], z[i]};
    out[i] = or_s_code(s, p);
  }
}

/* -------------------------------------------------------------- navigation */

void or_compose(int nnodes, const int32_t* parent, const double* RL, const double* tl,
                double* RG, double* tg) {
  for (int v = 0; v < nnodes; v++) {
    const double* L = RL + 9 * v;
    double* G = RG + 9 * v;
    if (parent[v] < 0) {
      for (int i = 0; i < 9; i++) G[i] = L[i];
      for (int i = 0; i < 3; i++) tg[3 * v + i] = tl[3 * v + i];
      continue;
    }
    const double* P = RG + 9 * parent[v];
    const double* tp = tg + 3 * parent[v];
    for (int i = 0; i < 3; i++) {
      for (int j = 0; j < 3; j++)
        G[3 * i + j] = (P[3 * i + 0] * L[0 * 3 + j] + P[3 * i + 1] * L[1 * 3 + j]) + P[3 * i + 2] * L[2 * 3 + j];
      tg[3 * v + i] = ((P[3 * i + 0] * tl[3 * v + 0] + P[3 * i + 1] * tl[3 * v + 1]) +
                       P[3 * i + 2] * tl[3 * v + 2]) + tp[i];
    }
  }
}

/* World to the frame of a node: p_local = R^T (p - t), d_local = R^T d. */
static void to_local(const double* R, const double* t, const double p[3], const double d[3],
                     double pl[3], double dl[3]) {
  const double v[3] = {p[0] - t[0], p[1] - t[1], p[2] - t[2]};
  for (int i = 0; i < 3; i++) {
    pl[i] = (R[0 * 3 + i] * v[0] + R[1 * 3 + i] * v[1]) + R[2 * 3 + i] * v[2];
    if (d) dl[i] = (R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1]) + R[2 * 3 + i] * d[2];
  }
}

/* Locate one point: -1 outside the world, else the deepest node reached by descending
 * into the first daughter (in index order) that does not classify it as outside.
 * *surface (may be NULL) is set when a classification on the way was SURFACE. */
static int locate_one(const or_solid* solids, int nnodes, const int32_t* node_solid, const int32_t* parent,
                      const double* RG, const double* tg, const double p[3], int* surface) {
  double pl[3];
  to_local(RG, tg, p, NULL, pl, NULL);
  int c0 = or_inside(&solids[node_solid[0]], pl);
  if (surface && c0 == OR_SURFACE) *surface = 1;
  if (c0 == OR_OUTSIDE) return -1;
  int v = 0, moved = 1;
  while (moved) {
    moved = 0;
    for (int c = 0; c < nnodes; c++) {
      if (parent[c] != v) continue;
      to_local(RG + 9 * c, tg + 3 * c, p, NULL, pl, NULL);
      const int code = or_inside(&solids[node_solid[c]], pl);
      if (surface && code == OR_SURFACE) *surface = 1;
      if (code != OR_OUTSIDE) { v = c; moved = 1; break; }
    }
  }
  return v;
}

void or_locate(const or_solid* solids, int nnodes, const int32_t* node_solid,
               const int32_t* parent, const double* RG, const double* tg,
               int64_t n, const double* x, const double* y, const double* z,
               int32_t* node, int nthreads) {
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (int64_t i = 0; i < n; i++) {
    const double p[3] = {x[i], y[i], z[i]};
    node[i] = locate_one(solids, nnodes, node_solid, parent, RG, tg, p, NULL);
  }
}

/* The geometry half of a step for one track in node v: the distance to the next
 * boundary (mother exit or first daughter entry), the safety, and the daughter entered
 * (-1: the track leaves v).  *second (may be NULL) is the next smaller candidate. */
static void nav_one(const or_solid* solids, int nnodes, const int32_t* node_solid, const int32_t* parent,
                    const double* RG, const double* tg, const double p[3], const double d[3], int v,
                    double* step, double* safety, int* next, double* second) {
  double pl[3], dl[3];
  to_local(RG + 9 * v, tg + 3 * v, p, d, pl, dl);
  const or_solid* m = &solids[node_solid[v]];
  double best = or_dist_out(m, pl, dl), runner = INFINITY;
  int who = -1, have = best >= 0;
  double saf = or_safety_out(m, pl);
  int have_s = saf >= 0;
  for (int c = 0; c < nnodes; c++) {
    if (parent[c] != v) continue;
    to_local(RG + 9 * c, tg + 3 * c, p, d, pl, dl);
    const or_solid* ds = &solids[node_solid[c]];
    const double t = or_dist_in(ds, pl, dl);
    if (t >= 0 && (!have || t < best || (t == best && who == -1))) {
      if (have && best < runner) runner = best;
      best = t; who = c; have = 1;
    } else if (t >= 0 && t < runner) {
      runner = t;
    }
    const double sd = or_safety_in(ds, pl);
    if (sd >= 0 && (!have_s || sd < saf)) { saf = sd; have_s = 1; }
  }
  *step = have ? best : -1.0;
  if (safety) *safety = have_s ? saf : -1.0;
  *next = have ? who : -1;
  if (second) *second = runner;
}

void or_nav_step(const or_solid* solids, int nnodes, const int32_t* node_solid,
                 const int32_t* parent, const double* RG, const double* tg,
                 int64_t n, const double* x, const double* y, const double* z,
                 const double* dx, const double* dy, const double* dz, const int32_t* node,
                 double* step, double* safety, int32_t* next, int nthreads) {
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (int64_t i = 0; i < n; i++) {
    const double p[3] = {x[i], y[i], z[i]}, d[3] = {dx[i], dy[i], dz[i]};
    const int v = node[i];
    if (v < 0 || v >= nnodes) { step[i] = -1.0; safety[i] = -1.0; next[i] = -1; continue; }
    int who;
    nav_one(solids, nnodes, node_solid, parent, RG, tg, p, d, v, &step[i], &safety[i], &who, NULL);
    next[i] = who;
  }
}

/* ---------------------------------------------------------- transport loop */

/* The transport of one track until it leaves the world, is absorbed, or has taken kmax
 * steps (Physics subsection).  Per step, in the volume v the track is in:
 *   - the geometry gives the distance dgeo to the next boundary (nav_one);
 *   - for each of the two processes of v's material (0 scatter, 1 absorb) a step
 *     s_i = -ln(xi_i) lambda_i is sampled, lambda_i = 1 / (n sigma_i) the mean free path
 *     (Eq. 1; sigma_n[2 m + i] = n sigma_i of material m, 0 = process absent), and the
 *     shortest is the candidate (ties: process 0);
 *   - if it is shorter than dgeo the track moves by it and the process acts: scatter
 *     turns the direction to (sin a cos b, sin a sin b, cos a) with cos a = 2 xi_2 - 1,
 *     b = 2 pi xi_3; absorb ends the track;
 *   - otherwise the track moves to the boundary and is located again from the world at
 *     the probe point p + kPush d (the boundary itself belongs to both sides); outside
 *     the world it has escaped.
 * The random numbers are inputs: xi[(i kmax + k) 4 + j] in (0, 1] for step k.  A step
 * whose outcome hangs on a near tie (physics against geometry, the two nearest
 * boundaries, or a probe on a surface) marks the track in tie[i] (results stay valid). */
#define OR_PUSH 1e-6
void or_transport(const or_solid* solids, int nnodes, const int32_t* node_solid,
                  const int32_t* parent, const double* RG, const double* tg,
                  const int32_t* node_material, const double* sigma_n,
                  int64_t n, const double* x, const double* y, const double* z,
                  const double* dx, const double* dy, const double* dz, const int32_t* node0,
                  const double* xi, int kmax, int8_t* reason, int32_t* nsteps, double* xo,
                  double* yo, double* zo, double* path, int32_t* last, int8_t* tie, int nthreads) {
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t i = 0; i < n; i++) {
    double p[3] = {x[i], y[i], z[i]}, d[3] = {dx[i], dy[i], dz[i]};
    int v = node0[i], k = 0, why = OR_TRUNCATED, near = 0;
    double len = 0.0;
    if (v < 0) why = OR_ESCAPED;
    while (v >= 0 && k < kmax) {
      const double* r = xi + ((size_t)i * (size_t)kmax + (size_t)k) * 4;
      double dgeo, second;
      int next;
      nav_one(solids, nnodes, node_solid, parent, RG, tg, p, d, v, &dgeo, NULL, &next, &second);
      if (dgeo < 0) { why = OR_LOST; break; }
      const int m = node_material[v];
      const double s0 = sigma_n[2 * m] > 0 ? -log(r[0]) / sigma_n[2 * m] : INFINITY;
      const double s1 = sigma_n[2 * m + 1] > 0 ? -log(r[1]) / sigma_n[2 * m + 1] : INFINITY;
      const int proc = s1 < s0 ? 1 : 0;
      const double sp = proc ? s1 : s0;
      const double scale = 1.0 + dgeo;
      if (fabs(sp - dgeo) <= 1e-9 * scale || fabs(second - dgeo) <= 1e-9 * scale) near = 1;
      k++;
      if (sp < dgeo) {
        for (int j = 0; j < 3; j++) p[j] = p[j] + sp * d[j];
        len += sp;
        if (proc == 1) { why = OR_ABSORBED; break; }
        const double ca = 2.0 * r[2] - 1.0, b = 6.283185307179586 * r[3];  /* 2 pi */
        const double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
        d[0] = sa * cos(b); d[1] = sa * sin(b); d[2] = ca;
      } else {
        for (int j = 0; j < 3; j++) p[j] = p[j] + dgeo * d[j];
        len += dgeo;
        const double q[3] = {p[0] + OR_PUSH * d[0], p[1] + OR_PUSH * d[1], p[2] + OR_PUSH * d[2]};
        int surf = 0;
        v = locate_one(solids, nnodes, node_solid, parent, RG, tg, q, &surf);
        if (surf) near = 1;
        if (v < 0) { why = OR_ESCAPED; break; }
      }
    }
    reason[i] = (int8_t)why;
    nsteps[i] = k;
    xo[i] = p[0]; yo[i] = p[1]; zo[i] = p[2];
    path[i] = len;
    last[i] = why == OR_ESCAPED ? -1 : v;
    tie[i] = (int8_t)near;
  }
}
