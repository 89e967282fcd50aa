// nav.cu -- the navigation step over a tree of placed volumes.
//
// The detector is an ordered hierarchy of placed solids (Detector geometry
// subsection); in a step the particle moves by the smaller of the physics length
// and the distance to the next boundary (Physics subsection).  The geometry half
// of the step, per track located in node v:
//   step   = min( DistanceToOut of v's solid, DistanceToIn of every daughter c of v
//                 in c's frame p_c = R_c^T (p - t_c), d_c = R_c^T d ),
//   safety = min( SafetyToOut of v, SafetyToIn of every daughter ),
//   next   = the daughter that gives the step, or -1 (the track leaves v);
// -1 values (a point on the wrong side) are left out; among equal distances the
// lowest daughter index wins and a daughter wins over the mother.
// Locate descends from the world into the first daughter (in index order) that
// does not classify the point as outside.
//
// Kernels: binary64, one thread per track; binary32 with kLanes lanes per track
// (daughters dealt round-robin to the lanes, results combined with warp
// shuffles), whose tracks with an ambiguous minimum, an uncertain daughter or a
// polycone are recomputed by the binary64 kernel from a worklist.  World-to-node
// transforms are composed on the host (binary64, no fused multiply-add) and
// applied on the device with round-to-nearest operations in a fixed order, so the
// binary64 results and codes agree with any evaluation that uses the same order.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>
#include <array>
#include "gv_internal.h"
#include "solid_fp32.cuh"
#include "solid_fp64.cuh"

namespace gv {

struct alignas(16) NodeD {
  double R[9];      // global rotation (row-major), p_world = R p_local + t
  double t[3];
  float Rh[9], Rl[9], th[3], tl[3];  // binary32 splits of R and t
  int32_t desc;     // index into the solid table
  int32_t parent;
  int32_t first;    // daughters: children[first .. first + count)
  int32_t count;
  int32_t grid;     // voxel grid over the daughters (-1: none)
  int32_t pad;
};

// A uniform grid over the daughters of a node, in the node's frame: cell (i, j, k) lists
// (in increasing node index) the daughters whose bounding box, padded, meets the cell.
struct GridD {
  double lo[3], cell[3], inv[3];  // origin, cell edges, their inverses
  int32_t n[3];                   // cells per axis
  int32_t start;                  // first cell's entry in the geometry's cell table
};

// Device pointers of a geometry's grids (grids == nullptr: no grid is used).
struct Vox {
  const GridD* grids;
  const int32_t* cells;  // per cell: [begin, end) into list
  const int32_t* list;
};

// Nodes with at least this many daughters get a grid.
constexpr int kVoxelMin = 16;
// The binary32 pass walks a node's grid only from this many daughters on: its walk (a
// binary64 DDA per lane, a group merge per cell) costs more than 8 lanes scanning a few
// dozen daughters.
constexpr int kWalk32Min = 128;

constexpr int kLanes = 8;  // lanes per track in the binary32 kernel

}  // namespace gv

struct gv_geom {
  int device;
  int nnodes, nsolids;
  gv::NodeD* d_nodes = nullptr;
  int32_t* d_children = nullptr;
  gv::Desc* d_solids = nullptr;
  gv::GridD* d_grids = nullptr;
  int32_t* d_cells = nullptr;
  int32_t* d_list = nullptr;
  bool use_vox = true;
  bool walk32 = false;  // some node with a grid has at least kWalk32Min daughters
  std::vector<gv::NodeD> nodes;
  std::vector<int32_t> children;
  std::vector<gv::Desc> solids;
  std::vector<gv::GridD> grids;
  std::vector<int32_t> cells, list;
};

namespace gv {

using f64::xadd;
using f64::xmul;
using f64::xsub;

// binary64 world -> node frame
__device__ __forceinline__ void to_local64(const NodeD& N, double x, double y, double z, double& lx, double& ly,
                                           double& lz) {
  const double v0 = xsub(x, N.t[0]), v1 = xsub(y, N.t[1]), v2 = xsub(z, N.t[2]);
  lx = xadd(xadd(xmul(N.R[0], v0), xmul(N.R[3], v1)), xmul(N.R[6], v2));
  ly = xadd(xadd(xmul(N.R[1], v0), xmul(N.R[4], v1)), xmul(N.R[7], v2));
  lz = xadd(xadd(xmul(N.R[2], v0), xmul(N.R[5], v1)), xmul(N.R[8], v2));
}
__device__ __forceinline__ void rot_local64(const NodeD& N, double u, double v, double w, double& lu, double& lv,
                                            double& lw) {
  lu = xadd(xadd(xmul(N.R[0], u), xmul(N.R[3], v)), xmul(N.R[6], w));
  lv = xadd(xadd(xmul(N.R[1], u), xmul(N.R[4], v)), xmul(N.R[7], w));
  lw = xadd(xadd(xmul(N.R[2], u), xmul(N.R[5], v)), xmul(N.R[8], w));
}

__device__ __forceinline__ void query64(const Desc& S, const f64::Track& T, unsigned want, f64::Result& R) {
  if (S.type == kBox) f64::box_query(S, T, want, R);
  else if (S.type == kTrd || S.type == kTrap) f64::planar_query(S, T, want, R);
  else if (S.type == kBool) f64::bool_query(S, T, want, R);
  else f64::pcon_query(S, T, want, R);
}

// The cell of a point given in the grid's node frame; false outside the grid (where no
// daughter is).
__device__ __forceinline__ bool grid_cell(const GridD& G, const double q[3], int c[3]) {
  for (int a = 0; a < 3; a++) {
    const double f = (q[a] - G.lo[a]) * G.inv[a];
    if (!(f >= 0.0 && f <= (double)G.n[a])) return false;
    c[a] = min((int)f, G.n[a] - 1);
  }
  return true;
}

// The daughters of node N to look at for a point (x, y, z) in world coordinates: all of
// them, or those listed in the point's cell when N has a grid.
__device__ __forceinline__ void candidates64(const NodeD& N, const int32_t* __restrict__ children, const Vox& vox,
                                             double x, double y, double z, const int32_t*& ids, int& count) {
  ids = children + N.first;
  count = N.count;
  if (!vox.grids || N.grid < 0) return;
  const GridD& G = vox.grids[N.grid];
  double q[3];
  to_local64(N, x, y, z, q[0], q[1], q[2]);
  int c[3];
  if (!grid_cell(G, q, c)) { count = 0; return; }
  const int cell = G.start + (c[2] * G.n[1] + c[1]) * G.n[0] + c[0];
  ids = vox.list + vox.cells[2 * cell];
  count = vox.cells[2 * cell + 1] - vox.cells[2 * cell];
}

struct NavArgs {
  const double *x, *y, *z, *u, *v, *w;
  const int32_t* node;
  double *step, *safety;
  int32_t* next;
  int64_t n;
};

// DistanceToIn of the daughters of N (which has a grid) for the ray p + t d (world):
// the cells the ray crosses are visited in t order and the walk stops once the best
// candidate so far is before the next cell by more than 4e-9 (1 + best) mm.  Candidates
// are ranked by (t, node index), the mother (who = -1) after every daughter; runner is the
// next smaller candidate among those seen (daughters not seen are farther than the margin).
// A 3-D DDA over the cells of a grid that a ray (node frame) crosses, in order of entry.
struct Dda {
  int c[3], step[3];
  double tnext[3], tdelta[3];
  double tenter, t1;  // entry of the current cell, exit from the grid
  int left;           // cells that may still be visited (a ray crosses at most n0 + n1 + n2 - 2)
  // false: the ray misses the grid
  __device__ __forceinline__ bool begin(const GridD& G, const double q[3], const double e[3]) {
    double t0 = 0.0;
    t1 = CUDART_INF;
    for (int k = 0; k < 3; k++) {
      const double lo = G.lo[k], hi = G.lo[k] + G.n[k] * G.cell[k];
      if (e[k] == 0.0) {
        if (q[k] < lo || q[k] > hi) return false;
        continue;
      }
      const double ta = (lo - q[k]) / e[k], tb = (hi - q[k]) / e[k];
      t0 = fmax(t0, fmin(ta, tb));
      t1 = fmin(t1, fmax(ta, tb));
    }
    if (!(t0 <= t1)) return false;
    for (int k = 0; k < 3; k++) {
      const double f = (q[k] + t0 * e[k] - G.lo[k]) * G.inv[k];
      c[k] = min(max((int)floor(f), 0), G.n[k] - 1);
      if (e[k] > 0) { step[k] = 1; tnext[k] = (G.lo[k] + (c[k] + 1) * G.cell[k] - q[k]) / e[k]; tdelta[k] = G.cell[k] / e[k]; }
      else if (e[k] < 0) { step[k] = -1; tnext[k] = (G.lo[k] + c[k] * G.cell[k] - q[k]) / e[k]; tdelta[k] = -G.cell[k] / e[k]; }
      else { step[k] = 0; tnext[k] = CUDART_INF; tdelta[k] = CUDART_INF; }
    }
    tenter = t0;
    left = G.n[0] + G.n[1] + G.n[2] + 3;
    return true;
  }
  __device__ __forceinline__ int cell(const GridD& G) const { return G.start + (c[2] * G.n[1] + c[1]) * G.n[0] + c[0]; }
  // to the next cell; false once the ray has left the grid
  __device__ __forceinline__ bool advance(const GridD& G) {
    int k = 0;
    if (tnext[1] < tnext[k]) k = 1;
    if (tnext[2] < tnext[k]) k = 2;
    tenter = tnext[k];
    if (!(tenter <= t1) || --left <= 0) return false;
    c[k] += step[k];
    if (c[k] < 0 || c[k] >= G.n[k]) return false;
    tnext[k] += tdelta[k];
    return true;
  }
};

// Stop rule of the walk: no daughter in a cell entered after t can give a distance within
// the tie margin of `best`.
__device__ __forceinline__ bool walk_done(double tenter, double best) { return tenter > best + 4e-9 * (1.0 + best); }

__device__ inline void grid_entries(const NodeD* __restrict__ nodes, const Desc* __restrict__ solids, const NodeD& N,
                                    const Vox& vox, const double p[3], const double d[3], double& best, int32_t& who,
                                    bool& have, double& runner) {
  const GridD& G = vox.grids[N.grid];
  double q[3], e[3];
  to_local64(N, p[0], p[1], p[2], q[0], q[1], q[2]);
  rot_local64(N, d[0], d[1], d[2], e[0], e[1], e[2]);
  Dda D;
  if (!D.begin(G, q, e)) return;
  int32_t recent[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  int slot = 0;
  f64::Track T;
  f64::Result R;
  do {
    if (have && walk_done(D.tenter, best)) break;
    const int cell = D.cell(G);
    for (int j = vox.cells[2 * cell]; j < vox.cells[2 * cell + 1]; j++) {
      const int32_t id = vox.list[j];
      bool seen = false;
      for (int r = 0; r < 8; r++) seen |= recent[r] == id;
      if (seen) continue;
      recent[slot] = id;
      slot = (slot + 1) & 7;
      const NodeD& C = nodes[id];
      to_local64(C, p[0], p[1], p[2], T.x, T.y, T.z);
      rot_local64(C, d[0], d[1], d[2], T.u, T.v, T.w);
      query64(solids[C.desc], T, f64::kWantDin, R);
      const double t = R.din;
      if (t >= 0 && (!have || t < best || (t == best && (who == -1 || id < who)))) {
        if (have && best < runner) runner = best;
        best = t; who = id; have = true;
      } else if (t >= 0 && id != who && t < runner) {  // a daughter seen again is not its own runner-up
        runner = t;
      }
    }
  } while (D.advance(G));
}

__device__ inline void nav_step64(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                  const Desc* __restrict__ solids, int nnodes, const NavArgs& a, int64_t i,
                                  const Vox& vox = Vox{nullptr, nullptr, nullptr}) {
  const int32_t v = a.node[i];
  if (v < 0 || v >= nnodes) {
    a.step[i] = -1.0; a.next[i] = -1;
    if (a.safety) a.safety[i] = -1.0;
    return;
  }
  const double x = a.x[i], y = a.y[i], z = a.z[i], u = a.u[i], vv = a.v[i], w = a.w[i];
  const NodeD& N = nodes[v];
  const bool want_saf = a.safety != nullptr;
  f64::Track T;
  f64::Result R;
  to_local64(N, x, y, z, T.x, T.y, T.z);
  rot_local64(N, u, vv, w, T.u, T.v, T.w);
  query64(solids[N.desc], T, f64::kWantDout | (want_saf ? f64::kWantSout : 0u), R);
  double best = R.dout, saf = R.sout;
  bool have = best >= 0, have_s = want_saf && saf >= 0;
  int32_t who = -1;
  const bool grid = vox.grids && N.grid >= 0;
  const unsigned want = (grid ? 0u : f64::kWantDin) | (want_saf ? f64::kWantSin : 0u);
  for (int j = 0; want != 0u && j < N.count; j++) {  // with a grid: only the safeties
    const int32_t c = children[N.first + j];
    const NodeD& C = nodes[c];
    to_local64(C, x, y, z, T.x, T.y, T.z);
    rot_local64(C, u, vv, w, T.u, T.v, T.w);
    query64(solids[C.desc], T, want, R);
    if (!grid && R.din >= 0 && (!have || R.din < best || (R.din == best && who == -1))) { best = R.din; who = c; have = true; }
    if (want_saf && R.sin >= 0 && (!have_s || R.sin < saf)) { saf = R.sin; have_s = true; }
  }
  if (grid) {
    const double p[3] = {x, y, z}, dd[3] = {u, vv, w};
    double runner = CUDART_INF;
    grid_entries(nodes, solids, N, vox, p, dd, best, who, have, runner);
  }
  a.step[i] = have ? best : -1.0;
  if (want_saf) a.safety[i] = have_s ? saf : -1.0;
  a.next[i] = have ? who : -1;
}

// Volume kinds for gathering tracks that run the same code (the paper's baskets of
// particles in one kind of volume): solid type, whether the volume has daughters and a grid.
constexpr int kKinds = 32;  // volume kinds (the last one: an empty slot)

__device__ __forceinline__ int volume_kind(const NodeD* __restrict__ nodes, const Desc* __restrict__ solids, int32_t v,
                                           const Vox& vox) {
  const NodeD& N = nodes[v];
  const int type = solids[N.desc].type;  // 0..6
  return type * 4 + (N.count > 0 ? 2 : 0) + (vox.grids && N.grid >= 0 ? 1 : 0);
}

// Order the m entries of a block by kind (counting sort in shared memory): perm[r] is the
// entry of rank r.  Block-uniform: every thread of the block calls it.
__device__ __forceinline__ void order_by_kind(int kind, int m, int* scount, int* perm) {
  const int t = threadIdx.x;
  if (t < kKinds) scount[t] = 0;
  __syncthreads();
  if (t < m) atomicAdd(&scount[kind], 1);
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < kKinds; k++) { const int c = scount[k]; scount[k] = acc; acc += c; }
  }
  __syncthreads();
  if (t < m) perm[atomicAdd(&scount[kind], 1)] = t;
  __syncthreads();
}

// One thread per track; the block's 256 tracks are taken in order of the kind of volume
// they are in, so that a warp runs one path through the geometry.
__global__ void __launch_bounds__(256) k_nav_fp64(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                                  const Desc* __restrict__ solids, int nnodes, NavArgs a, Vox vox) {
  __shared__ int scount[kKinds];
  __shared__ int sperm[256];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {  // block-uniform
    const int64_t i0 = base + threadIdx.x;
    int kind = kKinds - 1;
    if (i0 < a.n) {
      const int32_t v = a.node[i0];
      kind = (v >= 0 && v < nnodes) ? volume_kind(nodes, solids, v, vox) : kKinds - 2;
    }
    order_by_kind(kind, blockDim.x, scount, sperm);
    const int64_t i = base + sperm[threadIdx.x];
    if (i < a.n) nav_step64(nodes, children, solids, nnodes, a, i, vox);
    __syncthreads();
  }
}

// The same in tiles of 256 * kNavTileItems tracks per block iteration: longer runs of one kind, so
// fewer warps straddle two kinds.  Taken for baskets of at least four tiles per resident block
// (two per SM), so that the last round of tiles leaves few SMs idle.
constexpr int kNavTileItems = 4;
__global__ void __launch_bounds__(256) k_nav_fp64_tiles(const NodeD* __restrict__ nodes,
                                                        const int32_t* __restrict__ children,
                                                        const Desc* __restrict__ solids, int nnodes, NavArgs a,
                                                        Vox vox) {
  constexpr int TILE = 256 * kNavTileItems;
  __shared__ int scount[kKinds];
  __shared__ uint16_t sperm[TILE];
  __shared__ uint8_t skind[TILE];
  const int t = threadIdx.x;
  for (int64_t t0 = (int64_t)blockIdx.x * TILE; t0 < a.n; t0 += (int64_t)gridDim.x * TILE) {  // block-uniform
    const int len = a.n - t0 < TILE ? (int)(a.n - t0) : TILE;
    if (t < kKinds) scount[t] = 0;
    __syncthreads();
    for (int j = t; j < len; j += 256) {
      const int32_t v = a.node[t0 + j];
      const int kind = (v >= 0 && v < nnodes) ? volume_kind(nodes, solids, v, vox) : kKinds - 2;
      skind[j] = (uint8_t)kind;
      atomicAdd(&scount[kind], 1);
    }
    __syncthreads();
    if (t == 0) {
      int acc = 0;
      for (int k = 0; k < kKinds; k++) { const int c = scount[k]; scount[k] = acc; acc += c; }
    }
    __syncthreads();
    for (int j = t; j < len; j += 256) sperm[atomicAdd(&scount[skind[j]], 1)] = (uint16_t)j;
    __syncthreads();
    for (int r = t; r < len; r += 256) nav_step64(nodes, children, solids, nnodes, a, t0 + sperm[r], vox);
    __syncthreads();  // the tile's shared arrays are reused by the next tile
  }
}

__global__ void __launch_bounds__(256) k_nav_refine(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                                    const Desc* __restrict__ solids, int nnodes, NavArgs a,
                                                    const uint32_t* __restrict__ wl,
                                                    const unsigned long long* __restrict__ cnt, Vox vox) {
  const int64_t m = (int64_t)*cnt;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // consecutive entries go to consecutive blocks: a short worklist is spread over every
  // SM instead of filling the first few blocks (each entry is a long binary64 chain)
  for (int64_t j = (int64_t)threadIdx.x * gridDim.x + blockIdx.x; j < m; j += stride)
    nav_step64(nodes, children, solids, nnodes, a, wl[j], vox);
}

// ------------------------------------------------------------ binary32

// World point (split) -> node frame in double-float; direction rotated in binary32.
__device__ __forceinline__ f32::TrackF to_local32(const NodeD& N, const f32::TrackF& W) {
  using f32::F2;
  using f32::tprod;
  using f32::tsum;
  float dh[3], dl[3];
  const float ph[3] = {W.xh, W.yh, W.zh}, pl[3] = {W.xl, W.yl, W.zl};
  for (int k = 0; k < 3; k++) {
    const F2 s = tsum(ph[k], -N.th[k]);
    const float lo = s.l + (pl[k] - N.tl[k]);
    dh[k] = s.h + lo;
    dl[k] = lo - (dh[k] - s.h);
  }
  f32::TrackF L;
  float* oh[3] = {&L.xh, &L.yh, &L.zh};
  float* ol[3] = {&L.xl, &L.yl, &L.zl};
  for (int i = 0; i < 3; i++) {
    const F2 p0 = tprod(N.Rh[i], dh[0]), p1 = tprod(N.Rh[3 + i], dh[1]), p2 = tprod(N.Rh[6 + i], dh[2]);
    const F2 s1 = tsum(p0.h, p1.h), s2 = tsum(s1.h, p2.h);
    float lo = (s1.l + s2.l) + ((p0.l + p1.l) + p2.l);
    lo += N.Rh[i] * dl[0] + N.Rl[i] * dh[0];
    lo += N.Rh[3 + i] * dl[1] + N.Rl[3 + i] * dh[1];
    lo += N.Rh[6 + i] * dl[2] + N.Rl[6 + i] * dh[2];
    const float h = s2.h + lo;
    *oh[i] = h;
    *ol[i] = lo - (h - s2.h);
  }
  // direction in double-float as well: the quadratic coefficients use its low part
  const float uh[3] = {W.u, W.v, W.w}, ul[3] = {W.ul, W.vl, W.wl};
  float* dh_[3] = {&L.u, &L.v, &L.w};
  float* dl_[3] = {&L.ul, &L.vl, &L.wl};
  for (int i = 0; i < 3; i++) {
    const F2 p0 = tprod(N.Rh[i], uh[0]), p1 = tprod(N.Rh[3 + i], uh[1]), p2 = tprod(N.Rh[6 + i], uh[2]);
    const F2 s1 = tsum(p0.h, p1.h), s2 = tsum(s1.h, p2.h);
    float lo = (s1.l + s2.l) + ((p0.l + p1.l) + p2.l);
    lo += N.Rh[i] * ul[0] + N.Rl[i] * uh[0];
    lo += N.Rh[3 + i] * ul[1] + N.Rl[3 + i] * uh[1];
    lo += N.Rh[6 + i] * ul[2] + N.Rl[6 + i] * uh[2];
    const float h = s2.h + lo;
    *dh_[i] = h;
    *dl_[i] = lo - (h - s2.h);
  }
  L.zkey = 0;
  L.keyed = false;
  // The local point differs from the binary64 R^T (p - t) by the splits of p and t and the
  // double-float rounding: 2^-42 of |p|_1 + |t|_1 bounds it per coordinate; the rotated
  // direction is good to 2^-42 per component.
  L.fl = fmaf(f32::G42, fabsf(W.xh) + fabsf(W.yh) + fabsf(W.zh) + fabsf(N.th[0]) + fabsf(N.th[1]) + fabsf(N.th[2]),
              f32::FLOOR);
  L.dfl = f32::G42;
  L.bad = W.bad;
  return L;
}

// The planar and polycone-family passes are called, not inlined: inlined into the
// navigation kernel, the union of every family's code needed 247 registers (one block per
// SM); called, the kernel fits two blocks per SM (boxes, the common daughters, stay inline).
__device__ __noinline__ void planar32_call(const Desc& S, const f32::TrackF& T, unsigned want, f32::R32& R) {
  f32::planar32<true>(S, T, want, R);
}
__device__ __noinline__ void tube32_call(const Desc& S, const f32::TrackF& T, unsigned want, f32::R32& R) {
  f32::pcon32<true, true>(S, T, want, R);
}
__device__ __noinline__ void pcon32_call(const Desc& S, const f32::TrackF& T, unsigned want, f32::R32& R) {
  f32::pcon32<false, true>(S, T, want, R);
}

__device__ __forceinline__ void query32(const Desc& S, const f32::TrackF& T, unsigned want, f32::R32& R) {
  R.flag = T.bad;
  R.code = 1;
  R.din = R.dout = R.sin = R.sout = 0.f;
  if (R.flag) return;
  if (S.flags & kFp64Only) {  // features finer than binary32 resolves: binary64 only
    R.flag = true;
    return;
  }
  // frame tracks: the bounds add the local coordinates' and direction's own errors
  if (S.type == kBox) f32::box32<true>(S, T, want, R);
  else if (S.type == kTrd || S.type == kTrap) planar32_call(S, T, want, R);
  else if (S.type == kTube) tube32_call(S, T, want, R);
  else if (S.type == kBool) R.flag = true;  // booleans: binary64 only
  else pcon32_call(S, T, want, R);
}

// half of the output tolerance: the certified binary32 results are within it
__device__ __forceinline__ float half_tol(float t) { return 0.5f * (t < 1e-4f ? 1e-9f : 1e-5f * t); }

// Two smallest candidates (value, error, key); key = daughter order (or node index on a
// grid walk), mother = kMother.  With DEDUP the two keys are distinct: a key already held
// is not added again (a daughter met in several cells gives the same value each time);
// without it (every daughter evaluated once) the second key is not tracked.
template <bool DEDUP>
struct Top2 {
  float b1, e1, b2, e2;
  int w1, w2;
  __device__ __forceinline__ void add(float t, float e, int w) {
    if (DEDUP && (w == w1 || w == w2)) return;
    if (t < b1 || (t == b1 && w < w1)) {
      if (DEDUP) w2 = w1;
      b2 = b1; e2 = e1; b1 = t; e1 = e; w1 = w;
    } else if (t < b2) {
      b2 = t; e2 = e;
      if (DEDUP) w2 = w;
    }
  }
};

// Merge the Top2 of the lanes selected by `mask` (a group of kLanes lanes, xor offsets).
template <bool DEDUP>
__device__ __forceinline__ void group_merge(unsigned mask, Top2<DEDUP>& top) {
  constexpr int kNone = 0x7fffffff;
  for (int off = kLanes / 2; off > 0; off >>= 1) {
    const float ob1 = __shfl_xor_sync(mask, top.b1, off), oe1 = __shfl_xor_sync(mask, top.e1, off);
    const float ob2 = __shfl_xor_sync(mask, top.b2, off), oe2 = __shfl_xor_sync(mask, top.e2, off);
    const int ow1 = __shfl_xor_sync(mask, top.w1, off);
    const int ow2 = DEDUP ? __shfl_xor_sync(mask, top.w2, off) : kNone;
    top.add(ob1, oe1, ow1);
    top.add(ob2, oe2, ow2);
  }
}

// WALK: the geometry has nodes whose daughters the pass finds by walking their grid (the
// instance without it keeps the registers of the plain scan).
template <bool WALK>
__global__ void __launch_bounds__(256, 2) k_nav_fp32(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                                  const Desc* __restrict__ solids, int nnodes, NavArgs a,
                                                  uint32_t* __restrict__ wl, unsigned long long* __restrict__ cnt,
                                                  Vox vox) {
  constexpr int kMother = 0x7ffffffe, kNone = 0x7fffffff;
  const unsigned lane = threadIdx.x & 31u, sub = lane & (kLanes - 1);
  const unsigned gmask = ((1u << kLanes) - 1u) << (lane & ~(unsigned)(kLanes - 1));
  const bool want_saf = a.safety != nullptr;
  const int64_t tracks_per_block = blockDim.x / kLanes;
  const int64_t stride = (int64_t)gridDim.x * tracks_per_block;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  __shared__ int scount[kKinds];
  __shared__ int sperm[256];
  for (int64_t base = (int64_t)blockIdx.x * tracks_per_block; base < a.n; base += stride) {  // block-uniform
    // the block's tracks in order of the kind of volume they are in (a warp's four tracks
    // then mostly run the same path)
    int kind = kKinds - 1;
    if (threadIdx.x < tracks_per_block && base + threadIdx.x < a.n) {
      const int32_t v0 = a.node[base + threadIdx.x];
      kind = (v0 >= 0 && v0 < nnodes) ? volume_kind(nodes, solids, v0, vox) : kKinds - 2;
    }
    order_by_kind(kind, (int)tracks_per_block, scount, sperm);
    const int64_t i = base + sperm[threadIdx.x / kLanes];
    const bool valid = i < a.n;
    bool flag = false;
    Top2<WALK> top{F_INF, 0.f, F_INF, 0.f, kNone, kNone};
    float saf = F_INF;
    int32_t v = -1;
    bool walked = false;  // keys are node indices (grid walk) rather than daughter order
    if (valid) {
      v = a.node[i];
      if (v < 0 || v >= nnodes) flag = true;
    }
    if (valid && !flag) {
      const f32::TrackF W = f32::load_track(X, Y, Z, Ux, Uy, Uz, i, true);
      const NodeD& N = nodes[v];
      if (sub == 0) {  // the mother on the group's first lane
        const f32::TrackF L = to_local32(N, W);
        f32::R32 R;
        query32(solids[N.desc], L, f32::kWantDout | (want_saf ? f32::kWantSout : 0u), R);
        flag |= R.flag || R.dout < 0;  // a point outside its own volume: binary64 decides
        top.add(R.dout, half_tol(R.dout), kMother);
        if (want_saf) saf = R.sout;
      }
      walked = WALK && vox.grids && N.grid >= 0 && N.count >= kWalk32Min;
      const unsigned want = (walked ? 0u : f32::kWantDin) | (want_saf ? f32::kWantSin : 0u);
      for (int j = sub; want != 0u && j < N.count; j += kLanes) {
        const NodeD& C = nodes[children[N.first + j]];
        const f32::TrackF L = to_local32(C, W);
        f32::R32 R;
        query32(solids[C.desc], L, want, R);
        flag |= R.flag;
        if (!walked && R.din >= 0) top.add(R.din, half_tol(R.din), j);
        if (want_saf && R.sin >= 0) saf = fminf(saf, R.sin);
      }
      if (WALK && walked) {  // DistanceToIn of the daughters listed along the ray, cell by cell
        const GridD& G = vox.grids[N.grid];
        double q[3], e[3];
        to_local64(N, a.x[i], a.y[i], a.z[i], q[0], q[1], q[2]);
        rot_local64(N, a.u[i], a.v[i], a.w[i], e[0], e[1], e[2]);
        Dda D;
        if (D.begin(G, q, e)) {
          do {
            // every lane of the group holds the group's two best after the merge
            group_merge(gmask, top);
            const double bound = (double)top.b1 + (double)top.e1;
            if (isfinite(top.b1) && walk_done(D.tenter, bound)) break;
            const int cell = D.cell(G);
            for (int j = vox.cells[2 * cell] + (int)sub; j < vox.cells[2 * cell + 1]; j += kLanes) {
              const int32_t id = vox.list[j];
              const NodeD& C = nodes[id];
              const f32::TrackF L = to_local32(C, W);
              f32::R32 R;
              query32(solids[C.desc], L, f32::kWantDin, R);
              flag |= R.flag;
              if (R.din >= 0) top.add(R.din, half_tol(R.din), id);
            }
          } while (D.advance(G));
        }
      }
    }
    // combine the group's lanes with shuffles (xor within the group of kLanes)
    group_merge(0xffffffffu, top);
    for (int off = kLanes / 2; off > 0; off >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, saf, off);
      const int of = __shfl_xor_sync(0xffffffffu, (int)flag, off);
      saf = fminf(saf, os);
      flag |= of != 0;
    }
    // the winner must be certain: the runner-up's interval may not meet it
    if (valid && !flag && isfinite(top.b1) && top.b2 - top.e2 <= top.b1 + top.e1) flag = true;
    if (valid && !flag && !isfinite(top.b1)) flag = true;  // no finite step: binary64 decides
    if (valid && sub == 0 && !flag) {
      const NodeD& N = nodes[v];
      a.step[i] = (double)top.b1;
      if (want_saf) a.safety[i] = isfinite(saf) ? (double)saf : -1.0;
      a.next[i] = top.w1 == kMother ? -1 : walked ? top.w1 : children[N.first + top.w1];
    }
    const bool push = valid && sub == 0 && flag;
    const unsigned m = __ballot_sync(0xffffffffu, push);
    if (m) {
      unsigned long long at = 0;
      const int leader = __ffs(m) - 1;
      if ((int)lane == leader) at = atomicAdd(cnt, (unsigned long long)__popc(m));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (push) wl[at + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
    }
  }
}

// ------------------------------------------------------------ transport loop

// Locate one point in binary64 (gv_nav_locate's definition: from the world down, enter
// the first daughter, in index order or in the point's grid cell, that does not classify
// the point OUTSIDE; -1 outside the world) and report whether any classification on the
// way was SURFACE (the point lies on a boundary within the tolerance).
__device__ inline int32_t locate64_surf(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                        const Desc* __restrict__ solids, double x, double y, double z, bool& surf,
                                        const Vox& vox) {
  f64::Track T{0, 0, 0, 0, 0, 0};
  f64::Result R;
  to_local64(nodes[0], x, y, z, T.x, T.y, T.z);
  query64(solids[nodes[0].desc], T, f64::kWantCode, R);
  surf |= R.code == 1;
  if (R.code == 2) return -1;
  int32_t v = 0;
  for (int depth = 0; depth < 64; depth++) {
    const NodeD& N = nodes[v];
    int32_t into = -1;
    const int32_t* ids;
    int count;
    candidates64(N, children, vox, x, y, z, ids, count);  // a daughter whose band holds the point is listed
    for (int j = 0; j < count; j++) {
      const int32_t c = ids[j];
      to_local64(nodes[c], x, y, z, T.x, T.y, T.z);
      query64(solids[nodes[c].desc], T, f64::kWantCode, R);
      surf |= R.code == 1;
      if (R.code != 2) { into = c; break; }
    }
    if (into < 0) break;
    v = into;
  }
  return v;
}

// The geometry half of a step for one point in node v (as nav_step64, without the
// safety), and the next smaller candidate distance.
__device__ inline void nav_one64(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                 const Desc* __restrict__ solids, int32_t v, const double p[3], const double d[3],
                                 double& step, int32_t& next, double& second, const Vox& vox) {
  const NodeD& N = nodes[v];
  f64::Track T;
  f64::Result R;
  to_local64(N, p[0], p[1], p[2], T.x, T.y, T.z);
  rot_local64(N, d[0], d[1], d[2], T.u, T.v, T.w);
  query64(solids[N.desc], T, f64::kWantDout, R);
  double best = R.dout, runner = CUDART_INF;
  bool have = best >= 0;
  int32_t who = -1;
  if (vox.grids && N.grid >= 0) {
    grid_entries(nodes, solids, N, vox, p, d, best, who, have, runner);
    step = have ? best : -1.0;
    next = have ? who : -1;
    second = runner;
    return;
  }
  for (int j = 0; j < N.count; j++) {
    const int32_t c = children[N.first + j];
    const NodeD& C = nodes[c];
    to_local64(C, p[0], p[1], p[2], T.x, T.y, T.z);
    rot_local64(C, d[0], d[1], d[2], T.u, T.v, T.w);
    query64(solids[C.desc], T, f64::kWantDin, R);
    const double t = R.din;
    if (t >= 0 && (!have || t < best || (t == best && who == -1))) {
      if (have && best < runner) runner = best;
      best = t; who = c; have = true;
    } else if (t >= 0 && t < runner) {
      runner = t;
    }
  }
  step = have ? best : -1.0;
  next = have ? who : -1;
  second = runner;
}

// The binary32 track of a binary64 point and direction, split as the bulk pass splits its
// inputs (world frame: no frame error yet).
__device__ __forceinline__ f32::TrackF track_from(const double p[3], const double d[3]) {
  auto bits = [](double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return make_uint2((unsigned)b, (unsigned)(b >> 32));
  };
  f32::TrackF T;
  T.bad = false;
  T.fl = f32::FLOOR;
  T.dfl = 0.f;
  T.keyed = false;
  T.zkey = 0;
  f32::split(bits(p[0]), T.xh, T.xl, T.bad);
  f32::split(bits(p[1]), T.yh, T.yl, T.bad);
  f32::split(bits(p[2]), T.zh, T.zl, T.bad);
  T.u = f32::trunc_hi(bits(d[0]), T.bad);
  T.v = f32::trunc_hi(bits(d[1]), T.bad);
  T.w = f32::trunc_hi(bits(d[2]), T.bad);
  bool unused = false;
  float h;
  f32::split(bits(d[0]), h, T.ul, unused);
  f32::split(bits(d[1]), h, T.vl, unused);
  f32::split(bits(d[2]), h, T.wl, unused);
  return T;
}

// The geometry half of a step as nav_one64 gives it, with the candidates ranked in binary32
// first: when the binary32 pass certifies the nearest boundary (its interval apart from every
// other candidate's) and puts the runner-up beyond the near-tie margin, only that candidate
// is evaluated in binary64.  Its binary64 distance is then the minimum nav_one64 finds (each
// binary64 value lies in its candidate's interval), and the runner-up's lower bound gives the
// same near-tie decision.  A node with a grid, a flagged query or a close runner-up goes to
// nav_one64.
__device__ __noinline__ void nav_one_rank32(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                      const Desc* __restrict__ solids, int32_t v, const double p[3], const double d[3],
                                      double& step, int32_t& next, double& second, const Vox& vox) {
  constexpr int kMother = 0x7ffffffe, kNone = 0x7fffffff;
  const NodeD& N = nodes[v];
  const f32::TrackF W = track_from(p, d);
  bool ok = !W.bad && !(vox.grids && N.grid >= 0);
  Top2<false> top{F_INF, 0.f, F_INF, 0.f, kNone, kNone};
  if (ok) {
    f32::R32 R;
    query32(solids[N.desc], to_local32(N, W), f32::kWantDout, R);
    ok = !R.flag && R.dout >= 0;
    if (ok) top.add(R.dout, half_tol(R.dout), kMother);
    for (int j = 0; ok && j < N.count; j++) {
      const NodeD& C = nodes[children[N.first + j]];
      query32(solids[C.desc], to_local32(C, W), f32::kWantDin, R);
      if (R.flag) ok = false;
      else if (R.din >= 0) top.add(R.din, half_tol(R.din), j);
    }
    ok = ok && isfinite(top.b1) && top.b2 - top.e2 > top.b1 + top.e1;
  }
  if (ok) {
    const bool mother = top.w1 == kMother;
    const NodeD& M = mother ? N : nodes[children[N.first + top.w1]];
    f64::Track T;
    f64::Result R;
    to_local64(M, p[0], p[1], p[2], T.x, T.y, T.z);
    rot_local64(M, d[0], d[1], d[2], T.u, T.v, T.w);
    query64(solids[M.desc], T, mother ? f64::kWantDout : f64::kWantDin, R);
    const double t = mother ? R.dout : R.din;
    const double lo2 = (double)top.b2 - (double)top.e2;  // the runner-up's lower bound
    if (t >= 0 && lo2 - t > 2e-9 * (1.0 + t)) {
      step = t;
      next = mother ? -1 : children[N.first + top.w1];
      second = lo2;
      return;
    }
  }
  nav_one64(nodes, children, solids, v, p, d, step, next, second, vox);
}

// Locate as locate64_surf, with the codes taken in binary32 when every one on the way is
// certified (a certified code is the binary64 one); otherwise locate64_surf decides.
__device__ __noinline__ int32_t locate_rank32(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                        const Desc* __restrict__ solids, double x, double y, double z, bool& surf,
                                        const Vox& vox) {
  const double p[3] = {x, y, z}, d0[3] = {0.0, 0.0, 0.0};
  const f32::TrackF W = track_from(p, d0);
  if (!W.bad) {
    bool sf = false;
    f32::R32 R;
    query32(solids[nodes[0].desc], to_local32(nodes[0], W), f32::kWantCode, R);
    bool ok = !R.flag;
    int32_t v = -1;
    if (ok) {
      sf |= R.code == 1;
      if (R.code != 2) {
        v = 0;
        for (int depth = 0; ok && depth < 64; depth++) {
          const NodeD& N = nodes[v];
          int32_t into = -1;
          const int32_t* ids;
          int count;
          candidates64(N, children, vox, x, y, z, ids, count);
          for (int j = 0; j < count; j++) {
            const int32_t c = ids[j];
            query32(solids[nodes[c].desc], to_local32(nodes[c], W), f32::kWantCode, R);
            if (R.flag) { ok = false; break; }
            sf |= R.code == 1;
            if (R.code != 2) { into = c; break; }
          }
          if (!ok || into < 0) break;
          v = into;
        }
      }
    }
    if (ok) {
      surf |= sf;
      return v;
    }
  }
  return locate64_surf(nodes, children, solids, x, y, z, surf, vox);
}

// Locate with the codes ranked in binary32 first (the same nodes as k_locate).
__global__ void __launch_bounds__(256, 2) k_locate32(const NodeD* __restrict__ nodes,
                                                  const int32_t* __restrict__ children,
                                                  const Desc* __restrict__ solids, const double* __restrict__ x,
                                                  const double* __restrict__ y, const double* __restrict__ z,
                                                  int32_t* __restrict__ out, int64_t n, Vox vox) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    bool surf = false;
    out[i] = locate_rank32(nodes, children, solids, x[i], y[i], z[i], surf, vox);
  }
}

struct TransportArgs {
  const double *x, *y, *z, *u, *v, *w;  // start points and directions
  const int32_t* node0;                 // start volumes
  const int32_t* material;              // material of every node
  const double* sigma_n;                // n sigma of (scatter, absorb) per material, 1/mm
  const double* xi;                     // random numbers, [n][kmax][4], in (0, 1]
  int32_t kmax, nmat, nnodes;
  int32_t rank32;                       // rank the step's candidates and the codes in binary32
  int8_t* reason;
  int32_t* steps;
  double *xo, *yo, *zo, *path;
  int32_t* last;
  int8_t* tie;
  int64_t n;
};

constexpr double kPush = 1e-6;  // probe distance past a boundary for the relocation (mm)

// The state of one track in the loop.
struct Flight {
  double p[3], d[3], len;
  int32_t v, k, why;
  bool near, live;
  bool reloc;  // at a boundary, to be located again (the second half of a step)
};

__device__ __forceinline__ void flight_begin(const TransportArgs& a, int64_t i, Flight& F) {
  F.p[0] = a.x[i]; F.p[1] = a.y[i]; F.p[2] = a.z[i];
  F.d[0] = a.u[i]; F.d[1] = a.v[i]; F.d[2] = a.w[i];
  F.v = a.node0[i];
  F.k = 0;
  F.why = GV_TRUNCATED;
  F.near = false;
  F.reloc = false;
  F.len = 0.0;
  F.live = F.v >= 0 && F.v < a.nnodes && a.kmax > 0;
  if (F.v < 0) F.why = GV_ESCAPED;
  else if (F.v >= a.nnodes) F.why = GV_LOST;
}

// The first half of one step of the loop of the Physics subsection (see gv.h) for track i:
// the boundary distance, the physics step and, when the process acts first, the process.
__device__ inline void flight_step(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                   const Desc* __restrict__ solids, const TransportArgs& a, int64_t i, Flight& F,
                                   const Vox& vox) {
  const double* r = a.xi + ((size_t)i * (size_t)a.kmax + (size_t)F.k) * 4;
  double dgeo, second;
  int32_t next;
  if (a.rank32) nav_one_rank32(nodes, children, solids, F.v, F.p, F.d, dgeo, next, second, vox);
  else nav_one64(nodes, children, solids, F.v, F.p, F.d, dgeo, next, second, vox);
  const int32_t m = a.material[F.v];
  if (dgeo < 0 || m < 0 || m >= a.nmat) { F.why = GV_LOST; F.live = false; return; }
  const double sig0 = a.sigma_n[2 * m], sig1 = a.sigma_n[2 * m + 1];
  const double s0 = sig0 > 0 ? -log(r[0]) / sig0 : CUDART_INF;
  const double s1 = sig1 > 0 ? -log(r[1]) / sig1 : CUDART_INF;
  const int proc = s1 < s0 ? 1 : 0;
  const double sp = proc ? s1 : s0;
  const double scale = 1.0 + dgeo;
  if (fabs(sp - dgeo) <= 1e-9 * scale || fabs(second - dgeo) <= 1e-9 * scale) F.near = true;
  F.k++;
  if (sp < dgeo) {  // the process acts before the boundary
    for (int j = 0; j < 3; j++) F.p[j] = xadd(F.p[j], xmul(sp, F.d[j]));
    F.len = xadd(F.len, sp);
    if (proc == 1) { F.why = GV_ABSORBED; F.live = false; return; }
    const double ca = xsub(xmul(2.0, r[2]), 1.0), b = xmul(6.283185307179586, r[3]);
    const double sa = sqrt(fmax(0.0, xsub(1.0, xmul(ca, ca))));
    double sb, cb;
    sincos(b, &sb, &cb);
    F.d[0] = xmul(sa, cb); F.d[1] = xmul(sa, sb); F.d[2] = ca;
  } else {  // to the boundary; the probe point past it is located by flight_locate
    for (int j = 0; j < 3; j++) F.p[j] = xadd(F.p[j], xmul(dgeo, F.d[j]));
    F.len = xadd(F.len, dgeo);
    F.reloc = true;
    return;
  }
  if (F.k >= a.kmax) F.live = false;  // truncated
}

// The second half of a step that ended at a boundary: locate the probe point past it.
__device__ inline void flight_locate(const NodeD* __restrict__ nodes, const int32_t* __restrict__ children,
                                     const Desc* __restrict__ solids, const TransportArgs& a, Flight& F,
                                     const Vox& vox) {
  bool surf = false;
  F.reloc = false;
  const double q0 = xadd(F.p[0], xmul(kPush, F.d[0])), q1 = xadd(F.p[1], xmul(kPush, F.d[1])),
               q2 = xadd(F.p[2], xmul(kPush, F.d[2]));
  F.v = a.rank32 ? locate_rank32(nodes, children, solids, q0, q1, q2, surf, vox)
                 : locate64_surf(nodes, children, solids, q0, q1, q2, surf, vox);
  F.near |= surf;
  if (F.v < 0) { F.why = GV_ESCAPED; F.live = false; return; }
  if (F.k >= a.kmax) F.live = false;  // truncated
}

__device__ __forceinline__ void flight_end(const TransportArgs& a, int64_t i, const Flight& F) {
  a.reason[i] = (int8_t)F.why;
  a.steps[i] = F.k;
  a.xo[i] = F.p[0]; a.yo[i] = F.p[1]; a.zo[i] = F.p[2];
  a.path[i] = F.len;
  a.last[i] = F.why == GV_ESCAPED ? -1 : F.v;
  a.tie[i] = F.near ? 1 : 0;
}

// Binary64, in baskets (the paper's scheduler gathers particles that sit in the same kind
// of volume, so that they run the same code): a block keeps a pool of one track per
// thread in shared memory and loops: dead slots take the next tracks of the block's range;
// the live tracks are ordered by the kind of volume they are in (solid type, whether the
// volume has daughters and a grid), so that each warp steps tracks of one kind and its
// lanes follow one path through the geometry; every thread then takes one step for the
// track of its rank.  Tracks take from one to kmax steps; the pool keeps the block busy
// until its range is used up.
constexpr int kTransportThreads = 512;

__global__ void __launch_bounds__(kTransportThreads) k_transport(const NodeD* __restrict__ nodes,
                                                                 const int32_t* __restrict__ children,
                                                                 const Desc* __restrict__ solids, TransportArgs a,
                                                                 Vox vox) {
  constexpr int B = kTransportThreads;
  __shared__ double sp[3][B], sd[3][B], slen[B];
  __shared__ int64_t sidx[B];
  __shared__ int32_t sv[B], sk[B], swhy[B];
  __shared__ unsigned char snear[B], slive[B], sreloc[B];
  __shared__ int sperm[B];
  __shared__ int scount[kKinds];
  __shared__ unsigned long long snext;
  const int t = threadIdx.x;
  const int64_t chunk = (a.n + gridDim.x - 1) / gridDim.x;
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  const int64_t end = begin + chunk < a.n ? begin + chunk : a.n;
  if (t == 0) snext = (unsigned long long)(begin < end ? begin : end);
  slive[t] = 0;
  __syncthreads();
  while (true) {
    // dead slots take the next tracks of the range
    if (!slive[t]) {
      const unsigned long long j = atomicAdd(&snext, 1ull);
      if ((int64_t)j < end) {
        Flight F;
        flight_begin(a, (int64_t)j, F);
        if (F.live) {
          for (int c = 0; c < 3; c++) { sp[c][t] = F.p[c]; sd[c][t] = F.d[c]; }
          slen[t] = F.len; sidx[t] = (int64_t)j; sv[t] = F.v; sk[t] = F.k; swhy[t] = F.why;
          snear[t] = F.near; slive[t] = 1;
        } else {
          flight_end(a, (int64_t)j, F);
        }
      }
    }
    if (t < kKinds) scount[t] = 0;
    __syncthreads();
    const bool live = slive[t];
    if (!__syncthreads_or(live ? 1 : ((int64_t)snext < end ? 1 : 0))) break;
    // order the live tracks by volume kind (counting sort; empty slots last)
    const int kind = live ? volume_kind(nodes, solids, sv[t], vox) : kKinds - 1;
    atomicAdd(&scount[kind], 1);
    __syncthreads();
    if (t == 0) {
      int acc = 0;
      for (int k = 0; k < kKinds; k++) { const int c = scount[k]; scount[k] = acc; acc += c; }
    }
    __syncthreads();
    sperm[atomicAdd(&scount[kind], 1)] = t;
    __syncthreads();
    // first half of a step for the track of rank t
    int s = sperm[t];
    sreloc[t] = 0;
    __syncthreads();
    if (slive[s]) {
      Flight F;
      for (int c = 0; c < 3; c++) { F.p[c] = sp[c][s]; F.d[c] = sd[c][s]; }
      F.len = slen[s]; F.v = sv[s]; F.k = sk[s]; F.why = swhy[s]; F.near = snear[s]; F.live = true; F.reloc = false;
      const int64_t i = sidx[s];
      flight_step(nodes, children, solids, a, i, F, vox);
      if (F.live) {
        for (int c = 0; c < 3; c++) { sp[c][s] = F.p[c]; sd[c][s] = F.d[c]; }
        slen[s] = F.len; sv[s] = F.v; sk[s] = F.k; swhy[s] = F.why; snear[s] = F.near; sreloc[s] = F.reloc;
      } else {
        flight_end(a, i, F);
        slive[s] = 0;
      }
    }
    // second half for the tracks at a boundary, gathered into the first warps
    if (t < 2) scount[t] = 0;
    __syncthreads();
    const int rk = sreloc[t] ? 0 : 1;
    if (rk == 0) atomicAdd(&scount[0], 1);
    __syncthreads();
    const int nreloc = scount[0];
    __syncthreads();
    if (t == 0) { scount[0] = 0; scount[1] = nreloc; }
    __syncthreads();
    sperm[atomicAdd(&scount[rk], 1)] = t;
    __syncthreads();
    s = sperm[t];
    if (t < nreloc) {
      Flight F;
      for (int c = 0; c < 3; c++) { F.p[c] = sp[c][s]; F.d[c] = sd[c][s]; }
      F.len = slen[s]; F.v = sv[s]; F.k = sk[s]; F.why = swhy[s]; F.near = snear[s]; F.live = true; F.reloc = true;
      const int64_t i = sidx[s];
      flight_locate(nodes, children, solids, a, F, vox);
      if (F.live) {
        sv[s] = F.v; snear[s] = F.near;
      } else {
        flight_end(a, i, F);
        slive[s] = 0;
      }
      sreloc[s] = 0;
    }
    __syncthreads();
  }
}

}  // namespace gv

using namespace gv;

static void split_f(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

namespace gv {

// Half-extents of an origin-centred box holding the solid in its own frame, recorded by
// the solid's constructor.
static void solid_half(const Desc& h, double e[3]) {
  for (int i = 0; i < 3; i++) e[i] = h.ext[i];
}

// Grids for the nodes with at least kVoxelMin daughters: the box around the daughters'
// (padded) bounding boxes in the node's frame, cut into about one cell per daughter.
static void build_grids(gv_geom* g) {
  for (int v = 0; v < g->nnodes; v++) {
    NodeD& N = g->nodes[v];
    N.grid = -1;
    if (N.count < kVoxelMin) continue;
    std::vector<std::array<double, 6>> box(N.count);  // lo, hi per daughter in v's frame
    double glo[3] = {1e300, 1e300, 1e300}, ghi[3] = {-1e300, -1e300, -1e300};
    for (int j = 0; j < N.count; j++) {
      const NodeD& C = g->nodes[g->children[N.first + j]];
      // p_v = Rv^T (Rc p_c + tc - tv): M = Rv^T Rc, b = Rv^T (tc - tv)
      double M[9], b[3], e[3];
      for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++)
          M[3 * r + c] = N.R[0 * 3 + r] * C.R[0 * 3 + c] + N.R[1 * 3 + r] * C.R[1 * 3 + c] + N.R[2 * 3 + r] * C.R[2 * 3 + c];
        b[r] = N.R[0 * 3 + r] * (C.t[0] - N.t[0]) + N.R[1 * 3 + r] * (C.t[1] - N.t[1]) + N.R[2 * 3 + r] * (C.t[2] - N.t[2]);
      }
      solid_half(g->solids[C.desc], e);
      for (int r = 0; r < 3; r++) {
        const double h = std::fabs(M[3 * r]) * e[0] + std::fabs(M[3 * r + 1]) * e[1] + std::fabs(M[3 * r + 2]) * e[2];
        const double pad = 1e-6 * (1.0 + std::fabs(b[r]) + h);  // far above the rounding of any frame change
        box[j][r] = b[r] - h - pad;
        box[j][3 + r] = b[r] + h + pad;
        glo[r] = std::fmin(glo[r], box[j][r]);
        ghi[r] = std::fmax(ghi[r], box[j][3 + r]);
      }
    }
    GridD G;
    const double vol = std::fmax((ghi[0] - glo[0]) * (ghi[1] - glo[1]) * (ghi[2] - glo[2]), 1e-300);
    const double edge = std::cbrt(vol / N.count);
    for (int r = 0; r < 3; r++) {
      G.n[r] = (int)std::min(64.0, std::max(1.0, std::ceil((ghi[r] - glo[r]) / edge)));
      G.lo[r] = glo[r];
      G.cell[r] = (ghi[r] - glo[r]) / G.n[r];
      G.inv[r] = 1.0 / G.cell[r];
    }
    G.start = (int)(g->cells.size() / 2);
    const int ncell = G.n[0] * G.n[1] * G.n[2];
    std::vector<std::vector<int32_t>> lists(ncell);
    for (int j = 0; j < N.count; j++) {  // daughters in increasing node index
      int c0[3], c1[3];
      for (int r = 0; r < 3; r++) {
        c0[r] = std::max(0, std::min(G.n[r] - 1, (int)std::floor((box[j][r] - G.lo[r]) * G.inv[r])));
        c1[r] = std::max(0, std::min(G.n[r] - 1, (int)std::floor((box[j][3 + r] - G.lo[r]) * G.inv[r])));
      }
      for (int k = c0[2]; k <= c1[2]; k++)
        for (int jj = c0[1]; jj <= c1[1]; jj++)
          for (int i = c0[0]; i <= c1[0]; i++) lists[(k * G.n[1] + jj) * G.n[0] + i].push_back(g->children[N.first + j]);
    }
    for (int q = 0; q < ncell; q++) {
      g->cells.push_back((int32_t)g->list.size());
      g->list.insert(g->list.end(), lists[q].begin(), lists[q].end());
      g->cells.push_back((int32_t)g->list.size());
    }
    N.grid = (int)g->grids.size();
    g->grids.push_back(G);
    if (N.count >= kWalk32Min) g->walk32 = true;
  }
}

}  // namespace gv

extern "C" {

gv_status gv_geom_create(int32_t nnodes, const gv_solid* const* node_solid, const int32_t* parent, const double* R,
                         const double* t, gv_geom** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "geom: out handle pointer is NULL");
  if (nnodes <= 0 || !node_solid || !parent || !R || !t) return set_error(GV_ERR_INVALID_ARG, "geom: empty or NULL table");
  if (parent[0] != -1) return set_error(GV_ERR_INVALID_ARG, "geom: node 0 must be the world (parent -1)");
  for (int i = 1; i < nnodes; i++)
    if (parent[i] < 0 || parent[i] >= i) return set_error(GV_ERR_INVALID_ARG, "geom: parents must precede children");
  for (int i = 0; i < nnodes; i++)
    if (!node_solid[i]) return set_error(GV_ERR_INVALID_ARG, "geom: NULL solid");
  for (int i = 0; i < 12 * nnodes; i++)
    if (!std::isfinite(i < 9 * nnodes ? R[i] : t[i - 9 * nnodes])) return set_error(GV_ERR_INVALID_ARG, "geom: non-finite placement");
  gv_geom* g = new (std::nothrow) gv_geom;
  if (!g) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  g->nnodes = nnodes;
  g->nodes.resize(nnodes);
  std::vector<const gv_solid*> uniq;
  for (int v = 0; v < nnodes; v++) {
    NodeD& N = g->nodes[v];
    std::memset(&N, 0, sizeof(N));
    const double* L = R + 9 * v;
    const double* tl = t + 3 * v;
    if (parent[v] < 0) {
      for (int k = 0; k < 9; k++) N.R[k] = L[k];
      for (int k = 0; k < 3; k++) N.t[k] = tl[k];
    } else {  // compose with the parent's global placement (binary64, no fused multiply-add)
      const NodeD& P = g->nodes[parent[v]];
      for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++)
          N.R[3 * i + j] = (P.R[3 * i + 0] * L[0 * 3 + j] + P.R[3 * i + 1] * L[1 * 3 + j]) + P.R[3 * i + 2] * L[2 * 3 + j];
        N.t[i] = ((P.R[3 * i + 0] * tl[0] + P.R[3 * i + 1] * tl[1]) + P.R[3 * i + 2] * tl[2]) + P.t[i];
      }
    }
    for (int k = 0; k < 9; k++) split_f(N.R[k], N.Rh[k], N.Rl[k]);
    for (int k = 0; k < 3; k++) split_f(N.t[k], N.th[k], N.tl[k]);
    N.parent = parent[v];
    int idx = -1;
    for (size_t k = 0; k < uniq.size(); k++)
      if (uniq[k] == node_solid[v]) { idx = (int)k; break; }
    if (idx < 0) { idx = (int)uniq.size(); uniq.push_back(node_solid[v]); }
    N.desc = idx;
  }
  // daughters in increasing node index
  std::vector<int> cnt(nnodes, 0);
  for (int v = 1; v < nnodes; v++) cnt[parent[v]]++;
  int acc = 0;
  for (int v = 0; v < nnodes; v++) { g->nodes[v].first = acc; g->nodes[v].count = cnt[v]; acc += cnt[v]; }
  g->children.assign(std::max(acc, 1), 0);
  std::vector<int> fill(nnodes, 0);
  for (int v = 1; v < nnodes; v++) {
    const int p = parent[v];
    g->children[g->nodes[p].first + fill[p]++] = v;
  }
  g->nsolids = (int)uniq.size();
  const int nrec = table_size(uniq.data(), g->nsolids);  // booleans carry their components along
  for (const gv_solid* u : uniq) g->solids.push_back(u->h);  // host copies for the grid builder
  build_grids(g);
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_nodes, sizeof(NodeD) * nnodes);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_children, sizeof(int32_t) * g->children.size());
  if (e == cudaSuccess) e = cudaMalloc(&g->d_solids, sizeof(Desc) * nrec);
  if (e == cudaSuccess) g->solids = table_records(uniq.data(), g->nsolids, g->d_solids);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_nodes, g->nodes.data(), sizeof(NodeD) * nnodes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_children, g->children.data(), sizeof(int32_t) * g->children.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_solids, g->solids.data(), sizeof(Desc) * nrec, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !g->grids.empty()) {
    e = cudaMalloc(&g->d_grids, sizeof(GridD) * g->grids.size());
    if (e == cudaSuccess) e = cudaMalloc(&g->d_cells, sizeof(int32_t) * g->cells.size());
    if (e == cudaSuccess) e = cudaMalloc(&g->d_list, sizeof(int32_t) * std::max<size_t>(g->list.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(g->d_grids, g->grids.data(), sizeof(GridD) * g->grids.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_cells, g->cells.data(), sizeof(int32_t) * g->cells.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !g->list.empty())
      e = cudaMemcpy(g->d_list, g->list.data(), sizeof(int32_t) * g->list.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    gv_geom_destroy(g);
    return e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "geom: cudaMalloc failed") : cuda_error(e, "geom upload");
  }
  *out = g;
  return GV_OK;
}

void gv_geom_destroy(gv_geom* g) {
  if (!g) return;
  if (g->d_nodes) cudaFree(g->d_nodes);
  if (g->d_children) cudaFree(g->d_children);
  if (g->d_solids) cudaFree(g->d_solids);
  if (g->d_grids) cudaFree(g->d_grids);
  if (g->d_cells) cudaFree(g->d_cells);
  if (g->d_list) cudaFree(g->d_list);
  delete g;
}

gv_status gv_geom_set_voxels(gv_geom* g, int32_t enable) {
  if (!g) return set_error(GV_ERR_INVALID_ARG, "geom: NULL geometry");
  g->use_vox = enable != 0;
  return GV_OK;
}

int32_t gv_geom_voxel_count(const gv_geom* g) { return g ? (int32_t)g->grids.size() : 0; }

int32_t gv_geom_node_count(const gv_geom* g) { return g ? g->nnodes : 0; }

static gv::Vox vox_of(const gv_geom* g) {
  if (!g->use_vox || !g->d_grids) return gv::Vox{nullptr, nullptr, nullptr};
  return gv::Vox{g->d_grids, g->d_cells, g->d_list};
}

gv_status gv_nav_locate(const gv_geom* g, const gv_tracks* t, int32_t* node, void* stream) {
  const gv::Range range("gv_nav_locate");
  if (!g || !t) return set_error(GV_ERR_INVALID_ARG, "locate: NULL geometry or tracks");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "locate: negative track count");
  if (t->n == 0) return GV_OK;
  if (!t->x || !t->y || !t->z || !node) return set_error(GV_ERR_INVALID_ARG, "locate: NULL array");
  int64_t blocks = std::min<int64_t>((t->n + 255) / 256, (int64_t)sm_count() * 8);
  k_locate32<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(g->d_nodes, g->d_children, g->d_solids, t->x, t->y,
                                                                   t->z, node, t->n, vox_of(g));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GV_OK : cuda_error(e, "locate launch");
}

gv_status gv_nav_step(const gv_geom* g, const gv_tracks* t, const int32_t* node, gv_precision prec, double* step,
                      double* safety, int32_t* next, gv_workspace* ws, void* stream) {
  const gv::Range range("gv_nav_step");
  if (!g || !t) return set_error(GV_ERR_INVALID_ARG, "nav: NULL geometry or tracks");
  if (prec != GV_FP64 && prec != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "unknown precision");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "nav: negative track count");
  if (t->n == 0) return GV_OK;
  if (!t->x || !t->y || !t->z || !t->dx || !t->dy || !t->dz || !node || !step || !next)
    return set_error(GV_ERR_INVALID_ARG, "nav: NULL array");
  const void* ptrs[8] = {t->x, t->y, t->z, t->dx, t->dy, t->dz, step, safety};  // safety may be NULL
  for (int i = 0; i < 8; i++)
    if ((uintptr_t)ptrs[i] & 7u) return set_error(GV_ERR_INVALID_ARG, "nav: arrays must be 8-byte aligned");
  NavArgs a{t->x, t->y, t->z, t->dx, t->dy, t->dz, node, step, safety, next, t->n};
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = sm_count();
  if (prec == GV_FP64) {
    const int64_t tile = 256 * kNavTileItems;
    if (t->n >= (int64_t)sms * 2 * 4 * tile) {
      const int64_t blocks = std::min<int64_t>((t->n + tile - 1) / tile, (int64_t)sms * 2);
      k_nav_fp64_tiles<<<(unsigned)blocks, 256, 0, st>>>(g->d_nodes, g->d_children, g->d_solids, g->nnodes, a,
                                                         vox_of(g));
    } else {
      int64_t blocks = std::min<int64_t>((t->n + 255) / 256, (int64_t)sms * 8);
      k_nav_fp64<<<(unsigned)blocks, 256, 0, st>>>(g->d_nodes, g->d_children, g->d_solids, g->nnodes, a, vox_of(g));
    }
  } else {
    if (!ws) return set_error(GV_ERR_INVALID_ARG, "nav: GV_FP32_REFINE needs a workspace");
    if (ws->cap < t->n) return set_error(GV_ERR_OUT_OF_MEMORY, "nav: workspace smaller than the basket");
    ws->fused_blocks = 0;  // this pass counts its refinements in the counter
    cudaError_t e = cudaMemsetAsync(ws->counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "nav: counter reset");
    const int64_t per_block = 256 / kLanes;
    int64_t blocks = std::min<int64_t>((t->n + per_block - 1) / per_block, (int64_t)sms * 8);
    const Vox vox = vox_of(g);
    if (vox.grids && g->walk32)
      k_nav_fp32<true><<<(unsigned)blocks, 256, 0, st>>>(g->d_nodes, g->d_children, g->d_solids, g->nnodes, a,
                                                         ws->idx, ws->counter, vox);
    else
      k_nav_fp32<false><<<(unsigned)blocks, 256, 0, st>>>(g->d_nodes, g->d_children, g->d_solids, g->nnodes, a,
                                                          ws->idx, ws->counter, vox);
    k_nav_refine<<<(unsigned)(sms * 2), 256, 0, st>>>(g->d_nodes, g->d_children, g->d_solids, g->nnodes, a, ws->idx,
                                                       ws->counter, vox_of(g));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GV_OK : cuda_error(e, "nav launch");
}

gv_status gv_transport(const gv_geom* g, const gv_tracks* t, const int32_t* node0, const int32_t* node_material,
                       const double* sigma_n, int32_t nmat, const double* xi, int32_t kmax, gv_precision prec,
                       const gv_transport_out* out, void* stream) {
  const gv::Range range("gv_transport");
  if (!g || !t || !out) return set_error(GV_ERR_INVALID_ARG, "transport: NULL geometry, tracks or outputs");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "transport: negative track count");
  if (kmax < 1 || nmat < 1) return set_error(GV_ERR_INVALID_ARG, "transport: kmax and nmat must be >= 1");
  if (prec != GV_FP64 && prec != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "unknown precision");
  if (t->n == 0) return GV_OK;
  if (!t->x || !t->y || !t->z || !t->dx || !t->dy || !t->dz || !node0 || !node_material || !sigma_n || !xi ||
      !out->reason || !out->steps || !out->x || !out->y || !out->z || !out->path || !out->last || !out->tie)
    return set_error(GV_ERR_INVALID_ARG, "transport: NULL array");
  const void* ptrs[11] = {t->x, t->y, t->z, t->dx, t->dy, t->dz, sigma_n, xi, out->x, out->y, out->path};
  for (int i = 0; i < 11; i++)
    if ((uintptr_t)ptrs[i] & 7u) return set_error(GV_ERR_INVALID_ARG, "transport: arrays must be 8-byte aligned");
  if ((uintptr_t)out->z & 7u) return set_error(GV_ERR_INVALID_ARG, "transport: arrays must be 8-byte aligned");
  TransportArgs a{t->x, t->y, t->z, t->dx, t->dy, t->dz, node0, node_material, sigma_n, xi, kmax, nmat, g->nnodes,
                  prec == GV_FP32_REFINE ? 1 : 0, out->reason, out->steps, out->x, out->y, out->z, out->path, out->last, out->tie, t->n};
  // Resident blocks only: each block owns a contiguous range of tracks and keeps its pool
  // full from it, so it drains (slots empty while its last tracks finish) once per range.
  static int resident = 0;
  if (resident == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_transport, kTransportThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    resident = nb;
  }
  const int sms = sm_count();
  const int64_t blocks = std::min<int64_t>((t->n + kTransportThreads - 1) / kTransportThreads, (int64_t)sms * resident);
  k_transport<<<(unsigned)blocks, kTransportThreads, 0, (cudaStream_t)stream>>>(g->d_nodes, g->d_children, g->d_solids, a,
                                                                                  vox_of(g));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GV_OK : cuda_error(e, "transport launch");
}

}  // extern "C"
