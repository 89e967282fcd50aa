// batched.cu -- mixed-solid, mixed-size baskets in persistent launches.
//
// The scheduler of the paper (Project goals, item 1) hands the geometry baskets
// of particles that sit in the same kind of volume; here many such baskets,
// each against its own solid, are cut into fixed-size tiles (never crossing a
// basket), grouped by solid family.  Binary32: one persistent kernel per family
// that has tiles (box; trd/trap; tube; one-section cone; multi-section polycone;
// boolean), each with the block shape its registers allow, all captured on
// parallel branches of one CUDA graph so that their tails overlap.  CTAs take
// tiles from the family's atomic counter and stage the tile's solid descriptor in
// shared memory when it changes; the polycone kernel hands tiles to warps, which
// keep one track per lane and refill idle lanes from their tile (its walk visits
// one to several sections); booleans, which have no binary32 form, are evaluated
// in binary64 directly.  Uncertain tracks of every solid go to one worklist of
// (solid, track) pairs that a last kernel recomputes in binary64.  Binary64: one
// persistent kernel over all tiles.  An autotuner picks the tile length and the
// resident CTAs per SM (and, in binary64, the block size) by timing graph replays.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "gv_internal.h"
#include "solid_fp32.cuh"
#include "solid_fp64.cuh"
#include "work_class.cuh"

namespace gv {

struct Tile {
  long long start;  // first track (index into the caller's arrays)
  int len;          // tracks in the tile
  int solid;        // index into the solid table
};

__device__ __forceinline__ void stage_any(Desc& dst, const Desc* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 16); i += blockDim.x) d[i] = s[i];
}

// Binary64: one persistent kernel over all tiles; a CTA takes a tile, stages its solid when
// it changes, orders the tile's tracks by work class (f32::track_class) in shared memory and
// evaluates them one per thread in that order.  The FP64 pipe spends the same on a warp
// instruction whatever its active lanes, so warps of one class run fewer instructions; the
// per-track arithmetic, and so every output bit, is the same in any order.
constexpr int kTileItemsMax = 16;  // tracks per thread of a tile (the batch configuration's limit)
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_batched(const Desc* __restrict__ solids, const Tile* __restrict__ tiles,
                                                     int ntiles, unsigned* __restrict__ next, QueryArgs a) {
  constexpr uint32_t NC = f32::kClasses;
  __shared__ Desc S;
  __shared__ int s_tile;
  __shared__ uint16_t ord[THREADS * kTileItemsMax];  // tile offsets in class order
  __shared__ unsigned cnt[NC], cur[NC];
  int loaded = -1;
  const unsigned want = (a.inside ? 1u : 0u) | (a.din ? 2u : 0u) | (a.dout ? 4u : 0u) | (a.sin ? 8u : 0u) |
                        (a.sout ? 16u : 0u);
  const bool dirs = want & 6u;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  auto cls_of = [&](int64_t i) -> uint32_t {
    bool bad = false;  // a value outside the binary32 range only lands in some class
    const float x = f32::trunc_hi(__ldg(X + i), bad), y = f32::trunc_hi(__ldg(Y + i), bad),
                z = f32::trunc_hi(__ldg(Z + i), bad);
    float u = 0.f, v = 0.f, w = 0.f;
    if (dirs) {
      u = f32::trunc_hi(__ldg(Ux + i), bad);
      v = f32::trunc_hi(__ldg(Uy + i), bad);
      w = f32::trunc_hi(__ldg(Uz + i), bad);
    }
    return f32::track_class(S, x, y, z, u, v, w, dirs);
  };
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(next, 1u);
    if (threadIdx.x < NC) cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const Tile tl = tiles[t];
    if (tl.solid != loaded) {
      stage_any(S, solids + tl.solid);
      loaded = tl.solid;
      __syncthreads();
    }
    const int type = S.type;
    // a tile longer than the order array (never with a valid configuration) keeps index order
    const bool order = tl.len <= THREADS * kTileItemsMax;
    if (order) {
      for (int j = threadIdx.x; j < tl.len; j += THREADS) atomicAdd(&cnt[cls_of(tl.start + j)], 1u);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned run = 0;
        for (uint32_t q = 0; q < NC; q++) {
          cur[q] = run;
          run += cnt[q];
        }
      }
      __syncthreads();
      for (int j = threadIdx.x; j < tl.len; j += THREADS) ord[atomicAdd(&cur[cls_of(tl.start + j)], 1u)] = (uint16_t)j;
      __syncthreads();
    }
    for (int p = threadIdx.x; p < tl.len; p += THREADS) {
      const int64_t i = tl.start + (order ? (int)ord[p] : p);
      f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
      if (dirs) { T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i]; }
      f64::Result R;
      if (type == kBox) f64::box_query(S, T, want, R);
      else if (type == kTrd || type == kTrap) f64::planar_query(S, T, want, R);
      else if (type == kBool) f64::bool_query(S, T, want, R);
      else f64::pcon_query(S, T, want, R);
      if (a.inside) a.inside[i] = (int8_t)R.code;
      if (a.din) a.din[i] = R.din;
      if (a.dout) a.dout[i] = R.dout;
      if (a.sin) a.sin[i] = R.sin;
      if (a.sout) a.sout[i] = R.sout;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_batched_refine(const Desc* __restrict__ solids, QueryArgs a,
                                                        const unsigned long long* __restrict__ worklist,
                                                        const unsigned long long* __restrict__ wl_count) {
  const unsigned want = (a.inside ? 1u : 0u) | (a.din ? 2u : 0u) | (a.dout ? 4u : 0u) | (a.sin ? 8u : 0u) |
                        (a.sout ? 16u : 0u);
  const int64_t nref = (int64_t)*wl_count;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // consecutive entries go to consecutive blocks: a short worklist is spread over every
  // SM instead of filling the first few blocks (each entry is a long binary64 chain)
  for (int64_t j = (int64_t)threadIdx.x * gridDim.x + blockIdx.x; j < nref; j += stride) {
    const unsigned long long e = worklist[j];
    const int64_t i = (int64_t)(e & ((1ull << 40) - 1));
    const Desc& S = solids[e >> 40];
    f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
    if (want & 6u) { T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i]; }
    f64::Result R;
    if (S.type == kBox) f64::box_query(S, T, want, R);
    else if (S.type == kTrd || S.type == kTrap) f64::planar_query(S, T, want, R);
    else if (S.type == kBool) f64::bool_query(S, T, want, R);
    else f64::pcon_query(S, T, want, R);
    if (a.inside) a.inside[i] = (int8_t)R.code;
    if (a.din) a.din[i] = R.din;
    if (a.dout) a.dout[i] = R.dout;
    if (a.sin) a.sin[i] = R.sin;
    if (a.sout) a.sout[i] = R.sout;
  }
}

// ------------------------------------------------ binary32, one kernel per family

enum : int { kFamBox = 0, kFamPlanar = 1, kFamTube = 2, kFamCone = 3, kFamWalk = 4, kFamBool = 5, kFams = 6 };

// Block shapes per family, from the registers each needs: threads and resident blocks per
// SM (one-track-per-thread families use 256 threads, so that tiles of 128 * 2^k tracks
// fill them).
template <int FAM> struct BShape { static constexpr int threads = 256, blocks = 3; };
template <> struct BShape<kFamBox> { static constexpr int threads = 256, blocks = 4; };
template <> struct BShape<kFamWalk> { static constexpr int threads = 320, blocks = 2; };
template <> struct BShape<kFamBool> { static constexpr int threads = 256, blocks = 2; };
// Tiles of the polycone family hold one track per lane of a warp.
constexpr int kWalkTile = 32;

int family_of(const Desc& h) {
  if (h.flags & kFp64Only) return kFamBool;  // binary64 only, with the booleans
  switch (h.type) {
    case kBox: return kFamBox;
    case kTrd:
    case kTrap: return kFamPlanar;
    case kTube: return kFamTube;
    case kBool: return kFamBool;
    default: return h.nz > 2 ? kFamWalk : kFamCone;
  }
}

__device__ __forceinline__ void write32(const QueryArgs& a, int64_t i, const f32::R32& R) {
  if (a.inside) a.inside[i] = (int8_t)R.code;
  if (a.din) reinterpret_cast<unsigned long long*>(a.din)[i] = f32::f2d_bits(R.din);
  if (a.dout) reinterpret_cast<unsigned long long*>(a.dout)[i] = f32::f2d_bits(R.dout);
  if (a.sin) reinterpret_cast<unsigned long long*>(a.sin)[i] = f32::f2d_bits(R.sin);
  if (a.sout) reinterpret_cast<unsigned long long*>(a.sout)[i] = f32::f2d_bits(R.sout);
}

// A finished track: its results, or its (solid, track) pair on the refinement worklist.
__device__ __forceinline__ void finish32(const QueryArgs& a, unsigned long long* worklist, unsigned long long* wl_count,
                                         int solid, int64_t i, const f32::R32& R) {
  if (R.flag) worklist[atomicAdd(wl_count, 1ull)] = ((unsigned long long)(unsigned)solid << 40) | (unsigned long long)i;
  else write32(a, i, R);
}

__device__ __forceinline__ unsigned want_of(const QueryArgs& a) {
  return (a.inside ? 1u : 0u) | (a.din ? 2u : 0u) | (a.dout ? 4u : 0u) | (a.sin ? 8u : 0u) | (a.sout ? 16u : 0u);
}

// One track per thread (box, trd/trap, tube, one-section cone): a CTA takes a tile, stages
// its solid when it changes, runs the family's binary32 pass over the tile.
template <int FAM>
__global__ void __launch_bounds__(BShape<FAM>::threads, BShape<FAM>::blocks)
    k_bfam32(const Desc* __restrict__ solids, const Tile* __restrict__ tiles, int ntiles, unsigned* __restrict__ next,
             QueryArgs a, unsigned long long* __restrict__ worklist, unsigned long long* __restrict__ wl_count) {
  constexpr int THREADS = BShape<FAM>::threads;
  __shared__ Desc S;
  __shared__ int s_tile;
  int loaded = -1;
  const unsigned want = want_of(a);
  const bool dirs = want & 6u;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  const unsigned lane = threadIdx.x & 31u;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const Tile tl = tiles[t];
    if (tl.solid != loaded) {
      stage_any(S, solids + tl.solid);
      loaded = tl.solid;
      __syncthreads();
    }
    for (int j0 = 0; j0 < tl.len; j0 += THREADS) {
      const int j = j0 + threadIdx.x;
      const int64_t i = tl.start + j;
      bool flag = false;
      if (j < tl.len) {
        const f32::TrackF T = f32::load_track(X, Y, Z, Ux, Uy, Uz, i, dirs);
        f32::R32 R;
        R.flag = T.bad;
        R.code = 1;
        R.din = R.dout = R.sin = R.sout = 0.f;
        if (!R.flag) {
          if (FAM == kFamBox) f32::box32(S, T, want, R);
          else if (FAM == kFamPlanar) f32::planar32(S, T, want, R);
          else if (FAM == kFamTube) f32::pcon32<true>(S, T, want, R);
          else f32::pcon32<false>(S, T, want, R);
        }
        flag = R.flag;
        if (!flag) write32(a, i, R);
      }
      const unsigned m = __ballot_sync(0xffffffffu, flag);
      if (m) {
        unsigned long long at = 0;
        const int leader = __ffs(m) - 1;
        if ((int)lane == leader) at = atomicAdd(wl_count, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (flag)
          worklist[at + __popc(m & ((1u << lane) - 1u))] = ((unsigned long long)(unsigned)tl.solid << 40) | (unsigned long long)i;
      }
    }
    __syncthreads();
  }
}

// Multi-section polycones with lane refill: each warp keeps one track per lane; when at
// least half its lanes are idle they take the next tracks from the family's tiles (32
// tracks each, fetched from the family counter as the warp uses them up), so lanes of one
// warp may hold tracks of different solids: each lane reads its solid's descriptor from
// the table in global memory (a few KB per solid, cached).  Every busy lane then advances
// its walk by one section.
__global__ void __launch_bounds__(BShape<kFamWalk>::threads, BShape<kFamWalk>::blocks)
    k_bwalk32(const Desc* __restrict__ solids, const Tile* __restrict__ tiles, int ntiles, unsigned* __restrict__ next,
              QueryArgs a, unsigned long long* __restrict__ worklist, unsigned long long* __restrict__ wl_count) {
  const unsigned want = want_of(a);
  const bool dirs = want & 6u;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  const unsigned lane = threadIdx.x & 31u, below = (1u << lane) - 1u;
  Tile tl{0, 0, 0};  // the warp's current tile (warp-uniform)
  int pos = 0;       // its next track
  bool more = true, busy = false;
  int64_t i = 0;
  int sid = 0;
  f32::TrackF T;
  f32::R32 R;
  f32::Walk W;
  while (true) {
    const unsigned idle = __ballot_sync(0xffffffffu, !busy);
    if (more && (__popc(idle) >= 16 || idle == 0xffffffffu)) {
      // hand the idle lanes, in lane order, the next tracks of the current tile and of as
      // many further tiles as they need
      const int need = __popc(idle), rank = __popc(idle & below);
      int given = 0;
      int64_t my_i = -1;
      int my_sid = 0;
      while (given < need) {  // warp-uniform
        if (pos >= tl.len) {
          int t = 0;
          if (lane == 0) t = (int)atomicAdd(next, 1u);
          t = __shfl_sync(0xffffffffu, t, 0);
          if (t >= ntiles) { more = false; break; }
          tl = tiles[t];
          pos = 0;
        }
        const int take = min(tl.len - pos, need - given);
        if (!busy && rank >= given && rank < given + take) {
          my_i = tl.start + pos + (rank - given);
          my_sid = tl.solid;
        }
        pos += take;
        given += take;
      }
      if (my_i >= 0) {
        i = my_i;
        sid = my_sid;
        const Desc& S = solids[sid];
        T = f32::load_track<true>(X, Y, Z, Ux, Uy, Uz, i, dirs);
        R.flag = T.bad;
        R.code = 1;
        R.din = R.dout = R.sin = R.sout = 0.f;
        W.need_in = W.need_out = false;
        W.live = false;
        if (!R.flag) busy = f32::pcon_begin<false>(S, T, want, R, W);
        if (!busy) finish32(a, worklist, wl_count, sid, i, R);
      }
    }
    if (__ballot_sync(0xffffffffu, busy) == 0u) {
      if (!more) break;
      continue;
    }
    if (busy) {
      f32::pcon_step<false>(solids[sid], T, W);
      if (!W.live) {
        f32::pcon_end(W, R);
        finish32(a, worklist, wl_count, sid, i, R);
        busy = false;
      }
    }
  }
}

// Booleans and solids with features finer than binary32 resolves: binary64 directly, one
// track per thread.
__global__ void __launch_bounds__(BShape<kFamBool>::threads, BShape<kFamBool>::blocks)
    k_bbool64(const Desc* __restrict__ solids, const Tile* __restrict__ tiles, int ntiles, unsigned* __restrict__ next,
              QueryArgs a) {
  constexpr int THREADS = BShape<kFamBool>::threads;
  __shared__ int s_tile;
  const unsigned want = want_of(a);
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const Tile tl = tiles[t];
    const Desc& S = solids[tl.solid];
    for (int j = threadIdx.x; j < tl.len; j += THREADS) {
      const int64_t i = tl.start + j;
      f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
      if (want & 6u) { T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i]; }
      f64::Result R;
      f64::query(S, T, want, R);
      if (a.inside) a.inside[i] = (int8_t)R.code;
      if (a.din) a.din[i] = R.din;
      if (a.dout) a.dout[i] = R.dout;
      if (a.sin) a.sin[i] = R.sin;
      if (a.sout) a.sout[i] = R.sout;
    }
    __syncthreads();
  }
}

template <int FAM>
static int fam_occupancy() {
  int n = 0;
  if constexpr (FAM == kFamWalk) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bwalk32, BShape<kFamWalk>::threads, 0) != cudaSuccess) return 1;
  } else if constexpr (FAM == kFamBool) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bbool64, BShape<kFamBool>::threads, 0) != cudaSuccess) return 1;
  } else {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bfam32<FAM>, BShape<FAM>::threads, 0) != cudaSuccess) return 1;
  }
  return n > 0 ? n : 1;
}

static int fam_occupancy(int f) {
  switch (f) {
    case kFamBox: return fam_occupancy<kFamBox>();
    case kFamPlanar: return fam_occupancy<kFamPlanar>();
    case kFamTube: return fam_occupancy<kFamTube>();
    case kFamCone: return fam_occupancy<kFamCone>();
    case kFamWalk: return fam_occupancy<kFamWalk>();
    default: return fam_occupancy<kFamBool>();
  }
}

// Launch family f over its tiles with at most per_sm resident CTAs per SM.
static cudaError_t launch_family(int f, int per_sm, const Desc* solids, const Tile* tiles, int ntiles, unsigned* next,
                                 const QueryArgs& a, unsigned long long* wl, unsigned long long* cnt, cudaStream_t st) {
  const int occ = fam_occupancy(f);
  const int cap = (per_sm > 0 ? std::min(per_sm, occ) : occ) * sm_count();
  const int per_block = f == kFamWalk ? BShape<kFamWalk>::threads / 32 : 1;  // tiles a CTA works on at once
  const int grid = std::max(1, std::min(cap, (ntiles + per_block - 1) / per_block));
  // (the polycone family's tiles are one warp-refill long: a warp goes through several)
  switch (f) {
    case kFamBox: k_bfam32<kFamBox><<<grid, BShape<kFamBox>::threads, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt); break;
    case kFamPlanar: k_bfam32<kFamPlanar><<<grid, BShape<kFamPlanar>::threads, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt); break;
    case kFamTube: k_bfam32<kFamTube><<<grid, BShape<kFamTube>::threads, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt); break;
    case kFamCone: k_bfam32<kFamCone><<<grid, BShape<kFamCone>::threads, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt); break;
    case kFamWalk:
      k_bwalk32<<<grid, BShape<kFamWalk>::threads, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt);
      break;
    default: k_bbool64<<<grid, BShape<kFamBool>::threads, 0, st>>>(solids, tiles, ntiles, next, a); break;
  }
  return cudaGetLastError();
}

template <int THREADS>
static cudaError_t launch_batched_t(int grid, const Desc* solids, const Tile* tiles, int ntiles, unsigned* next,
                                    const QueryArgs& a, cudaStream_t st) {
  k_batched<THREADS><<<grid, THREADS, 0, st>>>(solids, tiles, ntiles, next, a);
  return cudaGetLastError();
}

template <int THREADS>
static int occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched<THREADS>, THREADS, 0) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

// resident CTAs per SM of the binary64 kernel
static int occupancy(int threads) {
  switch (threads) {
    case 128: return occupancy_t<128>();
    case 512: return occupancy_t<512>();
    default: return occupancy_t<256>();
  }
}

static cudaError_t launch_batched(int threads, int grid, const Desc* solids, const Tile* tiles, int ntiles,
                                  unsigned* next, const QueryArgs& a, cudaStream_t st) {
  switch (threads) {
    case 128: return launch_batched_t<128>(grid, solids, tiles, ntiles, next, a, st);
    case 512: return launch_batched_t<512>(grid, solids, tiles, ntiles, next, a, st);
    default: return launch_batched_t<256>(grid, solids, tiles, ntiles, next, a, st);
  }
}

}  // namespace gv

using namespace gv;

struct gv_batch {
  int device;
  int nsolids, nbaskets;
  int64_t total;                          // one past the largest track index used
  std::vector<gv_basket> baskets;
  std::vector<int> solid_types;
  std::vector<int> solid_fam;             // binary32 family of every solid
  Desc* d_solids = nullptr;
  Tile* d_tiles = nullptr;                // binary32 tiles grouped by family, then the binary64 tiles
  int64_t tile_cap = 0;                   // tiles allocated
  int ntiles = 0;
  int first64 = 0, ntiles64 = 0;
  int fam_first[kFams] = {0}, fam_count[kFams] = {0};
  unsigned* d_next = nullptr;             // tile counters: [0] all tiles, [1 + f] family f; worklist length at byte 64
  cudaStream_t fam_stream[kFams] = {nullptr};  // branches of the captured graph
  cudaEvent_t fork_ev = nullptr, join_ev[kFams] = {nullptr};
  unsigned long long* d_wl = nullptr;     // worklist of (solid << 40 | track), one segment per family
  int64_t wl_seg[kFams] = {0};            // first entry of every family's segment
  gv_batch_config cfg{256, 2, 0, 0};
  // captured graph and the arguments it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  QueryArgs cap_args{};
  int cap_prec = -1;
  gv_batch_config cap_cfg{0, 0, 0, 0};
};

// worklist length of family f (all of the binary64 kernel's tiles use none)
static unsigned long long* wl_count_ptr(gv_batch* b, int f) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(b->d_next) + 64) + f;
}
constexpr size_t kCounterBytes = 128;

static gv_status build_tiles(gv_batch* b) {
  const int64_t tile = (int64_t)b->cfg.threads * b->cfg.items;
  std::vector<Tile> t;
  t.reserve((size_t)b->tile_cap);
  for (int f = 0; f < kFams; f++) {  // grouped by family, baskets in order within one
    b->fam_first[f] = (int)t.size();
    for (const gv_basket& k : b->baskets) {
      if (b->solid_fam[k.solid] != f) continue;
      const int64_t len = f == kFamWalk ? kWalkTile : tile;
      for (int64_t off = 0; off < k.n; off += len) {
        Tile x;
        x.start = k.offset + off;
        x.len = (int)std::min<int64_t>(len, k.n - off);
        x.solid = k.solid;
        t.push_back(x);
      }
    }
    b->fam_count[f] = (int)t.size() - b->fam_first[f];
  }
  // then the binary64 kernel's tiles: every basket in order, tiles of the configured length
  b->first64 = (int)t.size();
  for (const gv_basket& k : b->baskets)
    for (int64_t off = 0; off < k.n; off += tile) {
      Tile x;
      x.start = k.offset + off;
      x.len = (int)std::min<int64_t>(tile, k.n - off);
      x.solid = k.solid;
      t.push_back(x);
    }
  b->ntiles64 = (int)t.size() - b->first64;
  if ((int64_t)t.size() > b->tile_cap) return set_error(GV_ERR_INVALID_ARG, "batch: too many tiles");
  b->ntiles = (int)t.size();
  if (!t.empty()) {
    cudaError_t e = cudaMemcpy(b->d_tiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "batch: tile upload");
  }
  return GV_OK;
}

static void drop_graph(gv_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->cap_prec = -1;
}

static gv_status check_config(const gv_batch_config* c) {
  if (!(c->threads == 128 || c->threads == 256 || c->threads == 512))
    return set_error(GV_ERR_INVALID_ARG, "batch config: threads must be 128, 256 or 512");
  if (c->items < 1 || c->items > 16) return set_error(GV_ERR_INVALID_ARG, "batch config: items must be in 1..16");
  if (c->ctas_per_sm < 0 || c->ctas_per_sm > 32)
    return set_error(GV_ERR_INVALID_ARG, "batch config: ctas_per_sm must be in 0..32 (0 = as many as fit)");
  return GV_OK;
}

static gv_status capture(gv_batch* b, const QueryArgs& a, int prec) {
  drop_graph(b);
  const bool fp64 = prec == GV_FP64;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_error(e, "batch: begin capture");
  cudaError_t le = cudaMemsetAsync(b->d_next, 0, kCounterBytes, b->cap_stream);
  if (le == cudaSuccess && fp64) {
    const int occ = occupancy(b->cfg.threads);
    const int per_sm = b->cfg.ctas_per_sm > 0 ? std::min(b->cfg.ctas_per_sm, occ) : occ;
    le = launch_batched(b->cfg.threads, std::max(1, per_sm * sm_count()), b->d_solids, b->d_tiles + b->first64, b->ntiles64,
                        b->d_next, a, b->cap_stream);
  }
  if (le == cudaSuccess && !fp64) {
    // the families on parallel branches, each followed by the binary64 pass over its own
    // worklist segment (a refinement's latency then overlaps the other families' work)
    le = cudaEventRecord(b->fork_ev, b->cap_stream);
    for (int f = 0; f < kFams && le == cudaSuccess; f++) {
      if (b->fam_count[f] == 0) continue;
      cudaStream_t fs = b->fam_stream[f];
      unsigned long long* wl = b->d_wl + b->wl_seg[f];
      le = cudaStreamWaitEvent(fs, b->fork_ev, 0);
      if (le == cudaSuccess)
        le = launch_family(f, b->cfg.ctas_per_sm, b->d_solids, b->d_tiles + b->fam_first[f], b->fam_count[f],
                           b->d_next + 1 + f, a, wl, wl_count_ptr(b, f), fs);
      if (le == cudaSuccess && f != kFamBool) {
        k_batched_refine<<<sm_count() * 2, 256, 0, fs>>>(b->d_solids, a, wl, wl_count_ptr(b, f));
        le = cudaGetLastError();
      }
      if (le == cudaSuccess) le = cudaEventRecord(b->join_ev[f], fs);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(b->cap_stream, b->join_ev[f], 0);
    }
  }
  e = cudaStreamEndCapture(b->cap_stream, &g);
  if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_error(le, "batch: capture launch"); }
  if (e != cudaSuccess) return cuda_error(e, "batch: end capture");
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { b->exec = nullptr; return cuda_error(e, "batch: graph instantiate"); }
  b->cap_args = a;
  b->cap_prec = prec;
  b->cap_cfg = b->cfg;
  return GV_OK;
}

static bool same_args(const QueryArgs& x, const QueryArgs& y) { return std::memcmp(&x, &y, sizeof(QueryArgs)) == 0; }

static gv_status batch_args(gv_batch* b, const gv_tracks* t, const gv_results* r, QueryArgs& a) {
  if (!t || !r) return set_error(GV_ERR_INVALID_ARG, "batch: NULL tracks or results");
  if (t->n < b->total) return set_error(GV_ERR_INVALID_ARG, "batch: tracks->n smaller than the baskets' extent");
  a = QueryArgs{t->x, t->y, t->z, t->dx, t->dy, t->dz, r->inside, r->dist_in, r->dist_out, r->safety_in,
                r->safety_out, t->n};
  if (b->total > 0) {
    if (!a.x || !a.y || !a.z) return set_error(GV_ERR_INVALID_ARG, "batch: NULL point array");
    if ((a.din || a.dout) && (!a.u || !a.v || !a.w))
      return set_error(GV_ERR_INVALID_ARG, "batch: distances requested without directions");
  }
  const void* ptrs[10] = {a.x, a.y, a.z, a.u, a.v, a.w, a.din, a.dout, a.sin, a.sout};
  for (int i = 0; i < 10; i++)
    if (ptrs[i] && ((uintptr_t)ptrs[i] & 7u)) return set_error(GV_ERR_INVALID_ARG, "batch: arrays must be 8-byte aligned");
  return GV_OK;
}

extern "C" {

gv_status gv_batch_create(const gv_solid* const* solids, int32_t nsolids, const gv_basket* baskets, int32_t nbaskets,
                          gv_batch** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "batch: out handle pointer is NULL");
  if (nsolids <= 0 || !solids) return set_error(GV_ERR_INVALID_ARG, "batch: no solids");
  if (nsolids > (1 << 23)) return set_error(GV_ERR_UNSUPPORTED, "batch: too many solids");
  if (nbaskets < 0 || (nbaskets > 0 && !baskets)) return set_error(GV_ERR_INVALID_ARG, "batch: bad basket table");
  int64_t total = 0, tile_cap = 0;
  for (int i = 0; i < nbaskets; i++) {
    const gv_basket& k = baskets[i];
    if (k.offset < 0 || k.n < 0 || k.solid < 0 || k.solid >= nsolids)
      return set_error(GV_ERR_INVALID_ARG, "batch: basket with a negative offset/size or an unknown solid");
    if (k.offset + k.n > ((int64_t)1 << 40)) return set_error(GV_ERR_UNSUPPORTED, "batch: track index beyond 2^40");
    total = std::max(total, k.offset + k.n);
    tile_cap += (k.n + 31) / 32 + (k.n + 127) / 128;  // binary32 tiles (at least 32 tracks), binary64 (128)
  }
  for (int i = 0; i < nsolids; i++)
    if (!solids[i]) return set_error(GV_ERR_INVALID_ARG, "batch: NULL solid");
  if (tile_cap > (int64_t)1 << 30) return set_error(GV_ERR_UNSUPPORTED, "batch: too many tiles");
  gv_batch* b = new (std::nothrow) gv_batch;
  if (!b) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  b->nsolids = nsolids;
  b->nbaskets = nbaskets;
  b->total = total;
  b->baskets.assign(baskets, baskets + nbaskets);
  b->tile_cap = std::max<int64_t>(tile_cap, 1);
  cudaError_t e = cudaGetDevice(&b->device);
  for (int i = 0; i < nsolids; i++) {
    b->solid_types.push_back(solids[i]->h.type);
    b->solid_fam.push_back(family_of(solids[i]->h));
  }
  const int nrec = table_size(solids, nsolids);  // booleans carry their components along
  if (e == cudaSuccess) e = cudaMalloc(&b->d_solids, sizeof(Desc) * nrec);
  if (e == cudaSuccess) {
    const std::vector<Desc> h = table_records(solids, nsolids, b->d_solids);
    e = cudaMemcpy(b->d_solids, h.data(), sizeof(Desc) * nrec, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(Tile) * b->tile_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_next, kCounterBytes);
  if (e == cudaSuccess) e = cudaMemset(b->d_next, 0, kCounterBytes);
  int64_t wl_total = 0;  // a family's segment holds every track of its baskets
  for (int f = 0; f < kFams; f++) {
    b->wl_seg[f] = wl_total;
    for (const gv_basket& k : b->baskets)
      if (b->solid_fam[k.solid] == f) wl_total += k.n;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_wl, sizeof(unsigned long long) * (size_t)std::max<int64_t>(wl_total, 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int f = 0; f < kFams && e == cudaSuccess; f++) {
    e = cudaStreamCreateWithFlags(&b->fam_stream[f], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[f], cudaEventDisableTiming);
  }
  gv_status st = GV_OK;
  if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "batch: cudaMalloc failed")
                                                           : cuda_error(e, "batch: create");
  if (st == GV_OK) st = build_tiles(b);
  if (st != GV_OK) { gv_batch_destroy(b); return st; }
  *out = b;
  return GV_OK;
}

gv_status gv_batch_set_config(gv_batch* b, const gv_batch_config* c) {
  if (!b || !c) return set_error(GV_ERR_INVALID_ARG, "batch: NULL argument");
  gv_status st = check_config(c);
  if (st != GV_OK) return st;
  const bool tiles_change = c->threads * c->items != b->cfg.threads * b->cfg.items;
  b->cfg = *c;
  drop_graph(b);
  return tiles_change ? build_tiles(b) : GV_OK;
}

gv_status gv_batch_get_config(const gv_batch* b, gv_batch_config* c) {
  if (!b || !c) return set_error(GV_ERR_INVALID_ARG, "batch: NULL argument");
  *c = b->cfg;
  return GV_OK;
}

gv_status gv_batch_run(gv_batch* b, const gv_tracks* t, gv_precision prec, const gv_results* r, void* stream) {
  const gv::Range range("gv_batch_run");
  if (!b) return set_error(GV_ERR_INVALID_ARG, "batch: NULL handle");
  if (prec != GV_FP64 && prec != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "unknown precision");
  QueryArgs a;
  gv_status st = batch_args(b, t, r, a);
  if (st != GV_OK) return st;
  if (!b->exec || b->cap_prec != (int)prec || !same_args(a, b->cap_args) ||
      std::memcmp(&b->cap_cfg, &b->cfg, sizeof(gv_batch_config)) != 0) {
    st = capture(b, a, prec);
    if (st != GV_OK) return st;
  }
  const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "batch: graph launch");
  return GV_OK;
}

gv_status gv_batch_refined(gv_batch* b, void* stream, int64_t* n) {
  if (!b || !n) return set_error(GV_ERR_INVALID_ARG, "batch: NULL argument");
  unsigned long long h[kFams] = {0};
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h, wl_count_ptr(b, 0), sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "gv_batch_refined");
  int64_t sum = 0;
  for (int f = 0; f < kFams; f++) sum += (int64_t)h[f];
  *n = sum;
  return GV_OK;
}

// Autotuner: times graph replays of every candidate (block size x tile length x
// resident CTAs per SM) and keeps the fastest.  With GV_AUTOTUNE_CACHE set to a
// file name, a result found there for the same workload signature is reused and
// new results are appended.
gv_status gv_batch_autotune(gv_batch* b, const gv_tracks* t, gv_precision prec, const gv_results* r, void* stream,
                            gv_batch_config* best_out) {
  const gv::Range range("gv_batch_autotune");
  if (!b) return set_error(GV_ERR_INVALID_ARG, "batch: NULL handle");
  QueryArgs a;
  gv_status st = batch_args(b, t, r, a);
  if (st != GV_OK) return st;
  // workload signature
  unsigned long long sig = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { sig = (sig ^ v) * 1099511628211ull; };
  mix((unsigned long long)b->nsolids); mix((unsigned long long)b->nbaskets); mix((unsigned long long)b->total);
  mix((unsigned long long)prec); mix((unsigned long long)sm_count());
  for (int ty : b->solid_types) mix((unsigned long long)ty);
  for (const gv_basket& k : b->baskets) { mix((unsigned long long)k.n); mix((unsigned long long)k.solid); }
  const char* cache = std::getenv("GV_AUTOTUNE_CACHE");
  if (cache && *cache) {
    if (FILE* f = std::fopen(cache, "r")) {
      unsigned long long s2;
      gv_batch_config c{};
      float us;
      while (std::fscanf(f, "%llx %d %d %d %f", &s2, &c.threads, &c.items, &c.ctas_per_sm, &us) == 5) {
        if (s2 == sig && check_config(&c) == GV_OK) {
          std::fclose(f);
          st = gv_batch_set_config(b, &c);
          if (st == GV_OK && best_out) *best_out = c;
          return st;
        }
      }
      std::fclose(f);
    }
  }
  const gv_batch_config start = b->cfg;
  gv_batch_config best = start;
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t s = (cudaStream_t)stream;
  const int thr[3] = {128, 256, 512};
  const int items[3] = {1, 2, 4};
  int occ32 = 1;  // binary32: the most CTAs per SM any family kernel can hold
  for (int f = 0; f < kFams; f++) occ32 = std::max(occ32, fam_occupancy(f));
  for (int ti = 0; ti < 3; ti++) {
    const int occ = prec == GV_FP64 ? occupancy(thr[ti]) : occ32;
    for (int ii = 0; ii < 3; ii++) {
      for (int c = 1; c <= occ; c++) {
        gv_batch_config cfg{thr[ti], items[ii], c, 0};
        st = gv_batch_set_config(b, &cfg);
        if (st != GV_OK) break;
        st = gv_batch_run(b, t, prec, r, stream);  // capture + warm
        if (st != GV_OK) break;
        cudaEventRecord(e0, s);
        const int reps = 3;
        for (int k = 0; k < reps && st == GV_OK; k++) st = gv_batch_run(b, t, prec, r, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_error(cudaGetLastError(), "autotune"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_ms) { best_ms = ms; best = cfg; }
      }
      if (st != GV_OK) break;
    }
    if (st != GV_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GV_OK) { gv_batch_set_config(b, &start); return st; }
  st = gv_batch_set_config(b, &best);
  if (st == GV_OK && best_out) *best_out = best;
  if (st == GV_OK && cache && *cache) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "%llx %d %d %d %.3f\n", sig, best.threads, best.items, best.ctas_per_sm, best_ms * 1000.f);
      std::fclose(f);
    }
  }
  return st;
}

void gv_batch_destroy(gv_batch* b) {
  if (!b) return;
  drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int f = 0; f < kFams; f++) {
    if (b->fam_stream[f]) cudaStreamDestroy(b->fam_stream[f]);
    if (b->join_ev[f]) cudaEventDestroy(b->join_ev[f]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->d_solids) cudaFree(b->d_solids);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_next) cudaFree(b->d_next);
  if (b->d_wl) cudaFree(b->d_wl);
  delete b;
}

}  // extern "C"
