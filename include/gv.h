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
 * (1e-9 mm absolute below 1e-4 mm).  Booleans, and solids with a feature finer
 * than 2^-16 of their size (a wall, a z-section, a phi wedge, or the sliver a
 * phi segment leaves out), are evaluated in binary64 under both. */
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
/* Boolean solid op(a, c) (Detector geometry subsection: composite elements built with
 * boolean operations): c placed in a's frame by p_a = R p_c + t (R row-major, a rotation:
 * orthonormal to 1e-9, determinant +1).  The components must be primitive solids; the
 * boolean keeps its own copies, so a and c may be destroyed afterwards.  Semantics: the
 * decision quantity is min(s_a, s_c) (union), max(s_a, s_c) (intersection) or
 * max(s_a, -s_c) (subtraction, a without c); safeties combine the components' safeties
 * (lower bounds); distances are the first crossing from outside to inside (inside to
 * outside) of the combined set along the ray, a surface point entering (leaving) the
 * boolean by its components' own motion having DistanceToIn (DistanceToOut) 0.
 * Booleans are evaluated in binary64 only: GV_FP32_REFINE runs the binary64 pass on them
 * and sends nothing to the worklist.  At most 96 pieces of the ray inside a component
 * are kept (far more than any solid here can produce). */
enum { GV_UNION = 0, GV_SUBTRACTION = 1, GV_INTERSECTION = 2 };
gv_status gv_solid_boolean(int32_t op, const gv_solid* a, const gv_solid* c, const double R[9], const double t[3],
                           gv_solid** out);
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
 * GV_FP32_REFINE.  With GV_FP32_REFINE, a basket of at most 65536 tracks of a
 * primitive solid is one launch (uncertain tracks are evaluated in binary64 at
 * once, with the same bits as the refinement pass).  With GV_FP64, a basket of a primitive solid with at least 2048
 * tracks per SM is evaluated in tiles ordered by work class (inside, outside, near
 * a surface): the results are the same bits as in index order, the pass is faster.
 * Asynchronous on `stream`. */
gv_status gv_query(const gv_solid* s, const gv_tracks* tracks, gv_precision prec,
                   const gv_results* res, gv_workspace* ws, void* stream);

/* --- baskets in host memory ---------------------------------------------------
 * The same queries for track and result arrays in HOST memory (the exception to
 * the device-pointer convention above).  A pipeline owns device staging slots
 * (81 bytes per track of chunk, per slot: the six inputs, the code, four results,
 * and the refinement worklist) and three CUDA streams of its own; a basket is cut
 * into chunks and, slot by slot, chunk c+1 is copied in while chunk c is evaluated
 * and chunk c-1 copied out, so the host link carries both directions at once and
 * the kernels run under the copies.  Host arrays should be pinned
 * (cudaHostAlloc/cudaHostRegister); pageable memory gives the same results, with
 * copies staged through the CUDA runtime that do not overlap.  The paper's baskets are
 * filled on the host by the scheduler (Project goals, item 1); this is how they
 * reach the device. */
typedef struct gv_pipeline gv_pipeline;
/* chunk_tracks >= 1 tracks per chunk, 2 <= slots <= 8 staging slots; allocates
 * slots * chunk_tracks * 85 bytes (cudaMalloc) on the current device. */
gv_status gv_pipeline_create(int64_t chunk_tracks, int32_t slots, gv_pipeline** out);
void gv_pipeline_destroy(gv_pipeline* p);
/* Enqueues gv_query for host arrays (tracks->x..dz and res->* are HOST pointers,
 * 8-byte aligned, NULL result pointers skip that query).  The work starts after
 * everything enqueued on `stream` so far; `stream` itself does not wait for it.
 * Consecutive calls on one pipeline overlap (the last chunks of one with the first
 * of the next).  A pipeline must not be used from two threads at once.  Results
 * are bit-identical to gv_query on the same tracks. */
gv_status gv_query_host(const gv_solid* s, const gv_tracks* host_tracks, gv_precision prec,
                        const gv_results* host_results, gv_pipeline* p, void* stream);
/* Makes `stream` wait for every gv_query_host call made on the pipeline so far: their
 * results are in the host arrays once `stream` has passed this point, and their host
 * arrays must stay valid and unchanged until then. */
gv_status gv_pipeline_join(gv_pipeline* p, void* stream);

/* --- mixed baskets in one launch --------------------------------------------
 * The scheduler of the paper (Project goals, item 1) collects particles that sit
 * in the same kind of volume into baskets and hands them to the geometry.  A
 * batch holds many such baskets, each against its own solid, over one shared
 * structure-of-arrays track set, and evaluates all of them with persistent
 * kernels replayed from a CUDA graph: GV_FP64 one kernel over all tiles;
 * GV_FP32_REFINE one kernel per solid family present (box; trd/trap; tube;
 * one-section cone; multi-section polycone, with lane refill; boolean, in
 * binary64) on parallel graph branches, then the binary64 worklist pass. */
typedef struct {
  int64_t offset;   /* first track of the basket in the shared arrays */
  int64_t n;        /* tracks in the basket (>= 0)                    */
  int32_t solid;    /* index into the batch's solid list              */
  int32_t reserved; /* must be 0                                       */
} gv_basket;

/* Launch shape: threads per CTA (128, 256 or 512), tracks per thread in a tile
 * (1..16; a tile is threads * items tracks of one basket), resident CTAs per SM
 * (1..32, 0 = as many as fit).  GV_FP32_REFINE: each family kernel has its own
 * block size (set by its registers); threads * items is the tile length and
 * ctas_per_sm caps the resident CTAs of every family kernel. */
typedef struct {
  int32_t threads, items, ctas_per_sm, reserved;
} gv_batch_config;

typedef struct gv_batch gv_batch;

/* Copies the solids' descriptors into a device table (the solid handles may be
 * destroyed afterwards), builds the tile list, and allocates the tile counter
 * and a worklist as long as the largest offset + n (cudaMalloc). */
gv_status gv_batch_create(const gv_solid* const* solids, int32_t nsolids, const gv_basket* baskets,
                          int32_t nbaskets, gv_batch** out);
gv_status gv_batch_set_config(gv_batch* b, const gv_batch_config* cfg);
gv_status gv_batch_get_config(const gv_batch* b, gv_batch_config* cfg);
/* All requested queries for every basket; tracks->n must cover every basket.
 * The first call with a given set of pointers, precision and configuration
 * captures a CUDA graph (on a private stream); later calls replay it on
 * `stream`.  Calls on one batch must not overlap on the GPU. */
gv_status gv_batch_run(gv_batch* b, const gv_tracks* tracks, gv_precision prec, const gv_results* res,
                       void* stream);
/* Times graph replays of every launch shape (128/256/512 threads x 1/2/4 items x
 * 1..max resident CTAs per SM) on these inputs, keeps the fastest and returns it
 * in *best (may be NULL).  If the environment variable GV_AUTOTUNE_CACHE names
 * a file, a stored result for the same workload is reused and new ones are
 * appended.  Synchronises `stream`. */
gv_status gv_batch_autotune(gv_batch* b, const gv_tracks* tracks, gv_precision prec, const gv_results* res,
                            void* stream, gv_batch_config* best);
/* Tracks of the last GV_FP32_REFINE run sent to binary64 (synchronises `stream`). */
gv_status gv_batch_refined(gv_batch* b, void* stream, int64_t* n_refined);
void gv_batch_destroy(gv_batch* b);

/* --- navigation (Physics and Detector geometry subsections: the detector is a
 *     hierarchy of placed solids; a step ends at the nearest boundary) -------
 * A geometry is a flat table of placed volumes ("nodes"): node 0 is the world
 * (parent -1), every other node's parent precedes it, and the daughters of a
 * node are its children in increasing index.  R (row-major 3x3, nine doubles per
 * node) and t (three per node) place a node in its parent: p_parent = R p_local
 * + t.  Host arrays, copied; the solids' descriptors are copied too. */
typedef struct gv_geom gv_geom;
gv_status gv_geom_create(int32_t nnodes, const gv_solid* const* node_solid, const int32_t* parent,
                         const double* R, const double* t, gv_geom** out);
void gv_geom_destroy(gv_geom* g);
int32_t gv_geom_node_count(const gv_geom* g);
/* Voxelised navigation (Detector geometry subsection: a volume with many daughters).
 * gv_geom_create gives every node with at least 16 daughters a uniform grid in the
 * node's frame over the daughters' bounding boxes (each padded by 1e-6 (1 + |centre|
 * + half-extent) mm), about one cell per daughter, at most 64 cells per axis; a cell
 * lists the daughters whose padded box meets it.  With grids on, locate tests only the
 * daughters listed in the point's cell (a point outside the grid is in none of them),
 * and a navigation step in such a node walks the cells along the ray in order of
 * entry (3-D DDA), evaluating DistanceToIn of the listed daughters and stopping once
 * the best distance so far lies more than 4e-9 (1 + best) mm before the next cell.
 * SafetyToIn is still taken over every daughter (the step's safety is a minimum over
 * all of them; pass safety = NULL to leave it out).  Binary64 results (locate, step,
 * safety, next, transport) are bit-identical with grids on or off: the walk sees every
 * daughter that could give the minimum or tie with it, and ties are broken by the
 * same rule.  GV_FP32_REFINE steps in a node with at least 128 daughters walk the
 * grid in binary32 with certified bounds (below that, 8 lanes per track scan them all):
 * next is the same with grids on or off, step and safety within that precision's
 * tolerance (a track certain on the walk may be refined without it, or the reverse).
 * enable != 0 turns the grids on (the default), 0 off;
 * takes effect for launches made after the call.  gv_geom_voxel_count returns the
 * number of nodes that have a grid. */
gv_status gv_geom_set_voxels(gv_geom* g, int32_t enable);
int32_t gv_geom_voxel_count(const gv_geom* g);
/* node[i] = the deepest node containing point i: start at the world and enter
 * the first daughter (lowest index) that does not classify the point OUTSIDE;
 * -1 if the point is outside the world.  Binary64 decisions. */
gv_status gv_nav_locate(const gv_geom* g, const gv_tracks* tracks, int32_t* node, void* stream);
/* One navigation step for tracks located in node[i] (world coordinates):
 * step = min(DistanceToOut of the node's solid, DistanceToIn of every daughter in
 * its own frame), safety = min(SafetyToOut, SafetyToIn of every daughter),
 * next = the daughter node giving the step or -1 (the track leaves its node);
 * values of -1 are left out, ties go to the lowest daughter index and a
 * daughter wins over the mother; no candidate -> step = safety = -1.
 * GV_FP32_REFINE needs a workspace of >= tracks->n (a binary32 pass; tracks
 * with an uncertain minimum go to binary64).  safety may be NULL: the safeties are
 * then not evaluated at all (with voxel grids the step no longer scans every
 * daughter).  Device arrays; async. */
gv_status gv_nav_step(const gv_geom* g, const gv_tracks* tracks, const int32_t* node, gv_precision prec,
                      double* step, double* safety, int32_t* next, gv_workspace* ws, void* stream);

/* --- transport loop (Physics subsection) -------------------------------------
 * Each track is followed from its start point until it leaves the world, is absorbed
 * or has taken kmax steps.  Per step, in the volume v it is in: the geometry gives the
 * distance dgeo to the next boundary (the navigation step above, binary64); for each of
 * the two processes of v's material (0 scatter, 1 absorb) a physics step
 * s_i = -ln(xi_i) lambda_i is sampled with lambda_i = 1 / (n sigma_i), the mean free
 * path of Eq. 1 (sigma_n[2 m + i] = n sigma_i of material m in 1/mm; 0 = the process
 * is absent), and the shortest is taken (ties: process 0), as the paper's step
 * selection does.  If it is shorter than dgeo the track moves by it and the process
 * acts: scatter turns the direction to (sin a cos b, sin a sin b, cos a) with
 * cos a = 2 xi_2 - 1, b = 2 pi xi_3; absorb ends the track.  Otherwise the track moves
 * to the boundary and is located again from the world at the probe point p + 1e-6 d
 * (a boundary belongs to both sides); outside the world it has escaped.
 * The random numbers are inputs: xi[(i kmax + k) 4 + j] in (0, 1] for step k of track
 * i (the library draws none).  Outputs per track: end reason, steps taken, end point,
 * path length (the sum of the steps), the node of the last step (-1 escaped), and tie = 1
 * when some step's outcome hung on a near tie (physics step within 1e-9 (1 + dgeo) of
 * dgeo, the two nearest boundaries as close, or a relocation probe on a surface) - such
 * a track may legitimately differ from another evaluation of the same loop.
 * All arrays are device arrays; node_material has one entry per node (a material index
 * outside [0, nmat) ends the track as GV_LOST); async on `stream`.
 * prec: GV_FP64 evaluates every candidate boundary and every code of the relocation in
 * binary64; GV_FP32_REFINE ranks them in binary32 first and evaluates in binary64 only the
 * nearest boundary when the binary32 pass certifies it (else every candidate), and takes the
 * relocation's codes in binary32 when all are certified (else binary64).  The results are
 * the same bits either way. */
enum { GV_ESCAPED = 0, GV_ABSORBED = 1, GV_TRUNCATED = 2, GV_LOST = 3 };
typedef struct {
  int8_t* reason;
  int32_t* steps;
  double *x, *y, *z;  /* end point */
  double* path;
  int32_t* last;
  int8_t* tie;
} gv_transport_out;
gv_status gv_transport(const gv_geom* g, const gv_tracks* tracks, const int32_t* node0,
                       const int32_t* node_material, const double* sigma_n, int32_t nmat,
                       const double* xi, int32_t kmax, gv_precision prec,
                       const gv_transport_out* out, void* stream);

/* --- serving: continuous batching of navigation requests (Project goals, item 1:
 *     the scheduler keeps handing baskets to the geometry) --------------------
 * A request is n tracks in world coordinates; the service locates them and takes
 * one navigation step.  A worker thread admits queued requests in arrival order
 * while a slot is free and the device arena has room, launches everything
 * admitted together as one group (one H2D copy per request, one launch per
 * kernel for the group, one D2H copy per request), spreads groups over several
 * streams so that their copies and kernels overlap, and records each request's
 * latency from submit to the moment the host sees it complete.  Buffers are host
 * memory (pinned for speed) that must stay valid until the request is waited:
 * input 6 n doubles (blocks of n: x, y, z, dx, dy, dz), output 24 n bytes
 * (blocks of n: step and safety as doubles, next and located node as int32). */
typedef struct {
  int64_t arena_bytes; /* device memory for admitted requests (about 192 bytes per track) */
  int32_t max_slots;   /* requests on the device at once (1..65536)                      */
  int32_t streams;     /* groups in flight (1..8)                                          */
  int32_t precision;   /* gv_precision of the navigation step                              */
  int32_t reserved;    /* 0                                                                */
} gv_server_config;
typedef struct {
  int64_t completed, tracks, launches, queued;
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit-to-completion latency */
} gv_server_stats;
typedef struct gv_server gv_server;
/* Allocates the arena, per-stream workspaces and streams (cudaMalloc) on the
 * current device and starts the worker thread.  The geometry must outlive it. */
gv_status gv_server_create(const gv_geom* g, const gv_server_config* cfg, gv_server** out);
/* Queues a request and returns its ticket; never blocks.  A request that can
 * never fit the arena returns GV_ERR_OUT_OF_MEMORY. */
gv_status gv_server_submit(gv_server* s, int64_t n, const double* host_in, void* host_out, int64_t* ticket);
/* *done = 1 once the request's results are in host_out. */
gv_status gv_server_poll(gv_server* s, int64_t ticket, int32_t* done);
/* Blocks until the request completes (GV_OK, its latency in *latency_ms, may be
 * NULL, and the ticket is released) or timeout_s passes (GV_ERR_TIMEOUT, the
 * ticket stays valid).  Every ticket must eventually be waited. */
gv_status gv_server_wait(gv_server* s, int64_t ticket, double timeout_s, double* latency_ms);
gv_status gv_server_get_stats(gv_server* s, gv_server_stats* out);
gv_status gv_server_reset_stats(gv_server* s);
/* Drains the queue, stops the worker and frees everything. */
void gv_server_destroy(gv_server* s);

/* The GV_FP32_REFINE query pass without a workspace, for callers that cannot
 * allocate device memory at call time: a framework that owns all device memory
 * through its own pool, a serving loop that cannot take cudaMalloc's implicit
 * device synchronisation, a plug-in with no allocator.  (The paper has no
 * counterpart; this is an interface convenience of this library.)
 * Its scratch (refinement worklist and counter) is a fixed device array owned by
 * the library: every GPU that loads the library holds 4 MiB for it until the
 * process exits.  At most 1048576 (2^20) tracks per call; larger baskets return
 * GV_ERR_INVALID_ARG.  The call allocates nothing (no cudaMalloc, no cudaFree).
 * All calls share the one array: the counter is cleared on `stream` at the start
 * of each call and the worklist keeps the last call's contents, so calls that
 * overlap on the GPU race and must be serialised by the caller.  The first call
 * on a device with a non-empty basket looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it; make that call before any stream capture.
 * The kept address belongs to the device's primary context: it does not survive
 * cudaDeviceReset, and callers in another (driver-API) context must not use this
 * entry point.  An empty basket returns GV_OK and enqueues nothing.  Results,
 * arguments and errors otherwise as for gv_query with GV_FP32_REFINE. */
gv_status gv_query_fp32_static(const gv_solid* s, const gv_tracks* tracks, const gv_results* res,
                               void* stream);

/* Device-side checks of a GV_DEBUG build (the paper has no counterpart: a development aid).
 * A library built with GV_DEBUG=1 (libgvgeo_debug.so) checks on the device, in the query passes,
 * that directions are unit vectors (| |d|^2 - 1 | <= 1e-6), that a refinement worklist holds no
 * more entries than its basket and that every track it names exists; a failed check records its
 * code and the smallest offending track index, and the pass goes on.  gv_debug_status
 * synchronises the device and returns the OR of the codes seen (*codes) and that index
 * (*first_index, -1 if none) since the last clear; clear != 0 resets them.  A release build
 * returns GV_ERR_UNSUPPORTED (codes 0, index -1). */
enum { GV_DEBUG_DIRECTION = 1, GV_DEBUG_WORKLIST = 2, GV_DEBUG_INDEX = 4 };
gv_status gv_debug_status(uint32_t* codes, int64_t* first_index, int32_t clear);

/* Thread-local description of the last error on this thread ("" if none). */
const char* gv_last_error(void);
/* Library version string. */
const char* gv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GV_H */
