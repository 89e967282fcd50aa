// batched.cu -- mixed-solid, mixed-size baskets in one persistent launch.
//
// The scheduler of the paper (Project goals, item 1) hands the geometry baskets
// of particles that sit in the same kind of volume; here many such baskets,
// each against its own solid, are evaluated by one persistent kernel: CTAs take
// fixed-size tiles (never crossing a basket) from an atomic counter, stage the
// tile's solid descriptor in shared memory when it changes, and run the binary32
// bulk pass (or the binary64 pass) on the tile.  Uncertain tracks of every solid
// go to one worklist of (solid, track) pairs that a second kernel recomputes in
// binary64.  The counter reset, both kernels and the worklist pass are captured
// once into a CUDA graph and replayed; an autotuner picks the block size, the
// tile length and the number of resident CTAs per SM by timing graph replays.
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

template <int THREADS, bool FP64>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_batched(const Desc* __restrict__ solids, const Tile* __restrict__ tiles,
                                                     int ntiles, unsigned* __restrict__ next_tile, QueryArgs a,
                                                     unsigned long long* __restrict__ worklist,
                                                     unsigned long long* __restrict__ wl_count) {
  __shared__ Desc S;
  __shared__ int s_tile;
  int loaded = -1;
  const unsigned want = (a.inside ? 1u : 0u) | (a.din ? 2u : 0u) | (a.dout ? 4u : 0u) | (a.sin ? 8u : 0u) |
                        (a.sout ? 16u : 0u);
  const bool dirs = want & 6u;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  const unsigned lane = threadIdx.x & 31u;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(next_tile, 1u);
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
    for (int j0 = 0; j0 < tl.len; j0 += THREADS) {
      const int j = j0 + threadIdx.x;
      const bool valid = j < tl.len;
      const int64_t i = tl.start + j;
      bool flag = false;
      if (valid) {
        if (FP64) {
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
        } else {
          const f32::TrackF T = f32::load_track(X, Y, Z, Ux, Uy, Uz, i, dirs);
          f32::R32 R;
          R.flag = T.bad;
          R.code = 1;
          R.din = R.dout = R.sin = R.sout = 0.f;
          if (!R.flag) {
            if (type == kBox) f32::box32(S, T, want, R);
            else if (type == kTrd || type == kTrap) f32::planar32(S, T, want, R);
            else if (type == kTube) f32::pcon32<true>(S, T, want, R);
            else if (type == kBool) R.flag = true;  // booleans: binary64 only
            else f32::pcon32<false>(S, T, want, R);
          }
          flag = R.flag;
          if (!flag) {
            if (a.inside) a.inside[i] = (int8_t)R.code;
            if (a.din) reinterpret_cast<unsigned long long*>(a.din)[i] = f32::f2d_bits(R.din);
            if (a.dout) reinterpret_cast<unsigned long long*>(a.dout)[i] = f32::f2d_bits(R.dout);
            if (a.sin) reinterpret_cast<unsigned long long*>(a.sin)[i] = f32::f2d_bits(R.sin);
            if (a.sout) reinterpret_cast<unsigned long long*>(a.sout)[i] = f32::f2d_bits(R.sout);
          }
        }
      }
      if (!FP64) {
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (m) {
          unsigned long long at = 0;
          const int leader = __ffs(m) - 1;
          if ((int)lane == leader) at = atomicAdd(wl_count, (unsigned long long)__popc(m));
          at = __shfl_sync(0xffffffffu, at, leader);
          if (flag)
            worklist[at + __popc(m & ((1u << lane) - 1u))] =
                ((unsigned long long)(unsigned)tl.solid << 40) | (unsigned long long)i;
        }
      }
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
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nref; j += stride) {
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

template <int THREADS, bool FP64>
static cudaError_t launch_batched_t(int grid, const Desc* solids, const Tile* tiles, int ntiles, unsigned* next,
                                    const QueryArgs& a, unsigned long long* wl, unsigned long long* cnt,
                                    cudaStream_t st) {
  k_batched<THREADS, FP64><<<grid, THREADS, 0, st>>>(solids, tiles, ntiles, next, a, wl, cnt);
  return cudaGetLastError();
}

template <int THREADS, bool FP64>
static int occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched<THREADS, FP64>, THREADS, 0) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

static int occupancy(int threads, bool fp64) {
  switch (threads) {
    case 128: return fp64 ? occupancy_t<128, true>() : occupancy_t<128, false>();
    case 512: return fp64 ? occupancy_t<512, true>() : occupancy_t<512, false>();
    default: return fp64 ? occupancy_t<256, true>() : occupancy_t<256, false>();
  }
}

static cudaError_t launch_batched(int threads, bool fp64, int grid, const Desc* solids, const Tile* tiles, int ntiles,
                                  unsigned* next, const QueryArgs& a, unsigned long long* wl,
                                  unsigned long long* cnt, cudaStream_t st) {
  switch (threads) {
    case 128:
      return fp64 ? launch_batched_t<128, true>(grid, solids, tiles, ntiles, next, a, wl, cnt, st)
                  : launch_batched_t<128, false>(grid, solids, tiles, ntiles, next, a, wl, cnt, st);
    case 512:
      return fp64 ? launch_batched_t<512, true>(grid, solids, tiles, ntiles, next, a, wl, cnt, st)
                  : launch_batched_t<512, false>(grid, solids, tiles, ntiles, next, a, wl, cnt, st);
    default:
      return fp64 ? launch_batched_t<256, true>(grid, solids, tiles, ntiles, next, a, wl, cnt, st)
                  : launch_batched_t<256, false>(grid, solids, tiles, ntiles, next, a, wl, cnt, st);
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
  Desc* d_solids = nullptr;
  Tile* d_tiles = nullptr;
  int64_t tile_cap = 0;                   // tiles allocated
  int ntiles = 0;
  unsigned* d_next = nullptr;             // [0] tile counter; then (8-aligned) worklist length
  unsigned long long* d_wl = nullptr;     // worklist of (solid << 40 | track)
  gv_batch_config cfg{256, 2, 0, 0};
  // captured graph and the arguments it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  QueryArgs cap_args{};
  int cap_prec = -1;
  gv_batch_config cap_cfg{0, 0, 0, 0};
};

static unsigned long long* wl_count_ptr(gv_batch* b) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(b->d_next) + 8);
}

static gv_status build_tiles(gv_batch* b) {
  const int64_t tile = (int64_t)b->cfg.threads * b->cfg.items;
  std::vector<Tile> t;
  t.reserve((size_t)b->tile_cap);
  for (const gv_basket& k : b->baskets)
    for (int64_t off = 0; off < k.n; off += tile) {
      Tile x;
      x.start = k.offset + off;
      x.len = (int)std::min<int64_t>(tile, k.n - off);
      x.solid = k.solid;
      t.push_back(x);
    }
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
  const int occ = occupancy(b->cfg.threads, fp64);
  const int per_sm = b->cfg.ctas_per_sm > 0 ? std::min(b->cfg.ctas_per_sm, occ) : occ;
  const int grid = std::max(1, per_sm * sm_count());
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_error(e, "batch: begin capture");
  cudaError_t le = cudaMemsetAsync(b->d_next, 0, 16, b->cap_stream);
  if (le == cudaSuccess)
    le = launch_batched(b->cfg.threads, fp64, grid, b->d_solids, b->d_tiles, b->ntiles, b->d_next, a, b->d_wl,
                        wl_count_ptr(b), b->cap_stream);
  if (le == cudaSuccess && !fp64) {
    k_batched_refine<<<sm_count() * 2, 256, 0, b->cap_stream>>>(b->d_solids, a, b->d_wl, wl_count_ptr(b));
    le = cudaGetLastError();
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
    tile_cap += (k.n + 127) / 128;
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
  for (int i = 0; i < nsolids; i++) b->solid_types.push_back(solids[i]->h.type);
  const int nrec = table_size(solids, nsolids);  // booleans carry their components along
  if (e == cudaSuccess) e = cudaMalloc(&b->d_solids, sizeof(Desc) * nrec);
  if (e == cudaSuccess) {
    const std::vector<Desc> h = table_records(solids, nsolids, b->d_solids);
    e = cudaMemcpy(b->d_solids, h.data(), sizeof(Desc) * nrec, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(Tile) * b->tile_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_next, 64);
  if (e == cudaSuccess) e = cudaMemset(b->d_next, 0, 64);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_wl, sizeof(unsigned long long) * (size_t)std::max<int64_t>(total, 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
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
  unsigned long long h = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, wl_count_ptr(b), sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "gv_batch_refined");
  *n = (int64_t)h;
  return GV_OK;
}

// Autotuner: times graph replays of every candidate (block size x tile length x
// resident CTAs per SM) and keeps the fastest.  With GV_AUTOTUNE_CACHE set to a
// file name, a result found there for the same workload signature is reused and
// new results are appended.
gv_status gv_batch_autotune(gv_batch* b, const gv_tracks* t, gv_precision prec, const gv_results* r, void* stream,
                            gv_batch_config* best_out) {
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
  for (int ti = 0; ti < 3; ti++) {
    const int occ = occupancy(thr[ti], prec == GV_FP64);
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
  if (b->d_solids) cudaFree(b->d_solids);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_next) cudaFree(b->d_next);
  if (b->d_wl) cudaFree(b->d_wl);
  delete b;
}

}  // extern "C"
