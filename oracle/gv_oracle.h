/*
 * gv_oracle.h -- the CPU oracle for the track-versus-solid geometry queries.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, scalar FP64 restatement of
 * what the three geometry questions of the VecGeom section (is the particle
 * inside the solid, its minimal distance to the border, the maximal step along
 * its direction) compute for box, trd, trapezoid, tube segment, cone segment and
 * polycone solids, plus the navigation step of the Physics / Detector geometry
 * subsections (step = distance to the boundary of the current volume, the
 * hierarchy of placed daughters).  Only the tests, the smoke check and the CPU
 * baseline of the benchmark use it; the CUDA library never links or calls it.
 * It shares no code, header or table with the library.
 *
 * Distances are found by enumerating every crossing of every constraint surface
 * along the ray and classifying the gaps between crossings by their midpoint.
 * That is deliberately unlike the closed-form solid code of the library.
 *
 * All arithmetic is IEEE binary64, compiled with -ffp-contract=off.
 */
#ifndef GV_ORACLE_H
#define GV_ORACLE_H
#include <stdint.h>

#define OR_MAXZ 64          /* largest polycone z-plane count */
#define OR_HALF_TOL 0.5e-9  /* h = kTolerance / 2, kTolerance = 1e-9 mm */

enum { OR_BOX = 0, OR_TRD = 1, OR_TRAP = 2, OR_TUBE = 3, OR_CONE = 4, OR_PCON = 5, OR_BOOL = 6 };
enum { OR_UNION = 0, OR_SUBTRACTION = 1, OR_INTERSECTION = 2 };
enum { OR_INSIDE = 0, OR_SURFACE = 1, OR_OUTSIDE = 2 };

typedef struct { double n[3]; double c; } or_plane;             /* g = n.p - c       */
typedef struct { double a, b, k; int present; } or_line;        /* R(z) = a z + b    */

struct or_bool_s;

typedef struct {
  int type;
  int family;                 /* 0 = planar (box/trd/trap), 1 = phi-segmented polycone */
  const struct or_bool_s* bl; /* OR_BOOL: the two components and the placement */
  int nplanes; or_plane pl[6];
  int nz; double z[OR_MAXZ];
  or_line out[OR_MAXZ - 1], in[OR_MAXZ - 1];
  int has_phi, phi_wide;
  double ns[2], ne[2];        /* outward normals of the phi = sphi and phi = sphi+dphi planes */
} or_solid;

/* A boolean solid: op(a, c), c placed in a's frame by p_a = R p_c + t (row-major R);
 * components are primitive solids (copied). */
typedef struct or_bool_s {
  int op;
  or_solid a, c;
  double R[9], t[3];
} or_bool;

/* Setup.  Return 0 on success, -1 on an invalid description. */
int or_setup_box(double dx, double dy, double dz, or_solid* s);
int or_setup_trap(const double p[11], or_solid* s);
int or_setup_trd(double dx1, double dx2, double dy1, double dy2, double dz, or_solid* s);
int or_setup_tube(double rmin, double rmax, double dz, double sphi, double dphi, or_solid* s);
int or_setup_cone(double rmin1, double rmax1, double rmin2, double rmax2, double dz,
                  double sphi, double dphi, or_solid* s);
int or_setup_pcon(int nz, const double* z, const double* rmin, const double* rmax,
                  double sphi, double dphi, or_solid* s);
int or_solid_size(void);
/* b must outlive s (s points to it). */
int or_setup_bool(int op, const or_solid* a, const or_solid* c, const double R[9], const double t[3],
                  or_bool* b, or_solid* s);
int or_bool_size(void);

/* Per-point queries (single track). */
double or_s_code(const or_solid* s, const double p[3]);
int    or_inside(const or_solid* s, const double p[3]);
double or_safety_in(const or_solid* s, const double p[3]);
double or_safety_out(const or_solid* s, const double p[3]);
double or_dist_in(const or_solid* s, const double p[3], const double d[3]);
double or_dist_out(const or_solid* s, const double p[3], const double d[3]);

/* The decision quantity s for n points (no tolerance applied). */
void or_s_code_n(const or_solid* s, int64_t n, const double* x, const double* y,
                 const double* z, double* out);

/* Batched over a structure-of-arrays basket; any output pointer may be NULL. */
void or_query(const or_solid* s, int64_t n,
              const double* x, const double* y, const double* z,
              const double* dx, const double* dy, const double* dz,
              int8_t* inside, double* dist_in, double* dist_out,
              double* safety_in, double* safety_out, int nthreads);

/* Navigation over a tree of placed volumes ("nodes"); node 0 is the world.
 * node_parent[0] = -1, parents precede children, the daughters of a node are
 * its children in increasing node index.  R_local/t_local place a node in its
 * parent: p_parent = R p_local + t (row-major R). */
void or_compose(int nnodes, const int32_t* node_parent, const double* R_local,
                const double* t_local, double* R_global, double* t_global);
void or_locate(const or_solid* solids, int nnodes, const int32_t* node_solid,
               const int32_t* node_parent, const double* R_global, const double* t_global,
               int64_t n, const double* x, const double* y, const double* z,
               int32_t* node, int nthreads);
void or_nav_step(const or_solid* solids, int nnodes, const int32_t* node_solid,
                 const int32_t* node_parent, const double* R_global, const double* t_global,
                 int64_t n, const double* x, const double* y, const double* z,
                 const double* dx, const double* dy, const double* dz, const int32_t* node,
                 double* step, double* safety, int32_t* next, int nthreads);
/* Transport loop: see gv_oracle.c.  End reasons: */
enum { OR_ESCAPED = 0, OR_ABSORBED = 1, OR_TRUNCATED = 2, OR_LOST = 3 };
void or_transport(const or_solid* solids, int nnodes, const int32_t* node_solid,
                  const int32_t* node_parent, const double* R_global, const double* t_global,
                  const int32_t* node_material, const double* sigma_n,
                  int64_t n, const double* x, const double* y, const double* z,
                  const double* dx, const double* dy, const double* dz, const int32_t* node0,
                  const double* xi, int kmax, int8_t* reason, int32_t* nsteps, double* xo,
                  double* yo, double* zo, double* path, int32_t* last, int8_t* tie, int nthreads);
#endif
