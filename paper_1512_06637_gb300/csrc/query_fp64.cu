// query_fp64.cu -- the plain binary64 query pass: one thread per track, the solid
// descriptor staged in shared memory.  A basket of a primitive solid large enough to give every
// SM a 2048-track tile is evaluated in tiles ordered by work class (k_query_fp64_tiles): the pass is bound
// by the FP64 pipe, which spends the same on a warp instruction whatever its active lanes, so
// warps of one class (inside, outside and entering, outside and missing, near a surface) run
// fewer instructions for the same tracks.  Smaller baskets and booleans go in index order,
// grid-stride over the basket (k_query_fp64).  Per track the arithmetic is the same either way.
#include "gv_debug.cuh"
#include "gv_internal.h"
#include "solid_fp64.cuh"
#include "work_class.cuh"

namespace gv {

// Copy a descriptor into shared memory with 16-byte loads.
__device__ __forceinline__ void stage_desc(Desc& dst, const Desc* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 16); i += blockDim.x) d[i] = s[i];
}

template <int FAMILY>
__global__ void __launch_bounds__(256) k_query_fp64(const Desc* __restrict__ desc, QueryArgs a) {
  __shared__ Desc S;
  stage_desc(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f64::kWantCode : 0u) | (a.din ? f64::kWantDin : 0u) |
                        (a.dout ? f64::kWantDout : 0u) | (a.sin ? f64::kWantSin : 0u) |
                        (a.sout ? f64::kWantSout : 0u);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
    if (want & (f64::kWantDin | f64::kWantDout)) {
      T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i];
      GV_DCHECK(dbg_unit(T.u, T.v, T.w), kDbgDirection, i);
    }
    f64::Result R;
    if (FAMILY == 0) f64::box_query(S, T, want, R);
    else if (FAMILY == 1) f64::planar_query(S, T, want, R);
    else if (FAMILY == 4) f64::bool_query(S, T, want, R);
    else f64::pcon_query(S, T, want, R);
    if (a.inside) a.inside[i] = (int8_t)R.code;
    if (a.din) a.din[i] = R.din;
    if (a.dout) a.dout[i] = R.dout;
    if (a.sin) a.sin[i] = R.sin;
    if (a.sout) a.sout[i] = R.sout;
  }
}

// The binary64 pass in tiles ordered by work class: a block takes a tile of 256 * ITEMS
// consecutive tracks, classifies them (f32::track_class, from the high parts; the reads bring the
// tile into the caches), orders the tile's offsets by class in shared memory (a count, a scan
// and a scatter) and evaluates them in that order.
template <int FAMILY, int ITEMS>
__global__ void __launch_bounds__(256) k_query_fp64_tiles(const Desc* __restrict__ desc, QueryArgs a) {
  constexpr int NT = 256, TILE = NT * ITEMS;
  constexpr uint32_t NC = f32::kClasses;
  __shared__ Desc S;
  __shared__ uint16_t ord[TILE];
  __shared__ uint8_t cls[TILE];
  __shared__ unsigned cnt[NC], cur[NC];
  stage_desc(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f64::kWantCode : 0u) | (a.din ? f64::kWantDin : 0u) |
                        (a.dout ? f64::kWantDout : 0u) | (a.sin ? f64::kWantSin : 0u) |
                        (a.sout ? f64::kWantSout : 0u);
  const bool dirs = want & (f64::kWantDin | f64::kWantDout);
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  const int tid = threadIdx.x;
  for (int64_t t0 = (int64_t)blockIdx.x * TILE; t0 < a.n; t0 += (int64_t)gridDim.x * TILE) {
    const int len = a.n - t0 < TILE ? (int)(a.n - t0) : TILE;
    if (tid < (int)NC) cnt[tid] = 0u;
    __syncthreads();
    for (int j = tid; j < len; j += NT) {
      const int64_t i = t0 + j;
      bool bad = false;  // a value outside the binary32 range only lands in some class
      const float x = f32::trunc_hi(__ldg(X + i), bad), y = f32::trunc_hi(__ldg(Y + i), bad),
                  z = f32::trunc_hi(__ldg(Z + i), bad);
      float u = 0.f, v = 0.f, w = 0.f;
      if (dirs) {
        u = f32::trunc_hi(__ldg(Ux + i), bad);
        v = f32::trunc_hi(__ldg(Uy + i), bad);
        w = f32::trunc_hi(__ldg(Uz + i), bad);
      }
      const uint32_t c = f32::track_class(S, x, y, z, u, v, w, dirs);
      cls[j] = (uint8_t)c;
      atomicAdd(&cnt[c], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      unsigned run = 0;
      for (uint32_t q = 0; q < NC; q++) {
        cur[q] = run;
        run += cnt[q];
      }
    }
    __syncthreads();
    for (int j = tid; j < len; j += NT) ord[atomicAdd(&cur[cls[j]], 1u)] = (uint16_t)j;
    __syncthreads();
    for (int p = tid; p < len; p += NT) {
      const int64_t i = t0 + ord[p];
      f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
      if (dirs) {
        T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i];
        GV_DCHECK(dbg_unit(T.u, T.v, T.w), kDbgDirection, i);
      }
      f64::Result R;
      if (FAMILY == 0) f64::box_query(S, T, want, R);
      else if (FAMILY == 1) f64::planar_query(S, T, want, R);
      else f64::pcon_query(S, T, want, R);
      if (a.inside) a.inside[i] = (int8_t)R.code;
      if (a.din) a.din[i] = R.din;
      if (a.dout) a.dout[i] = R.dout;
      if (a.sin) a.sin[i] = R.sin;
      if (a.sout) a.sout[i] = R.sout;
    }
    __syncthreads();  // the tile's shared arrays are reused by the next tile
  }
}

template <int FAMILY, int ITEMS>
static int64_t tiles_grid(int64_t tiles, int sms) {
  // resident blocks per SM of the kernel (queried once: it depends only on the kernel and the GPU)
  static const int occ = [] {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_query_fp64_tiles<FAMILY, ITEMS>, 256, 0) != cudaSuccess || o < 1) {
      cudaGetLastError();  // leave no error behind for the launch check
      o = 1;
    }
    return o;
  }();
  return tiles < (int64_t)sms * occ ? tiles : (int64_t)sms * occ;
}

cudaError_t launch_query_fp64(const gv_solid* s, const QueryArgs& a, cudaStream_t stream) {
  if (a.n == 0) return cudaSuccess;
  const int threads = 256;
  const int sms = sm_count();
  // tiles of 2048 tracks when the basket gives four of them to every resident block (two per SM),
  // else of 1024 (more tiles, fewer SMs idle in the last round); none below one 2048 tile per SM
  if (s->h.type != kBool && a.n >= (int64_t)sms * 2048) {
    const bool big = a.n >= (int64_t)sms * 2 * 4 * 2048;
    const int64_t tiles = big ? (a.n + 2047) / 2048 : (a.n + 1023) / 1024;
    switch (s->h.type) {
      case kBox:
        if (big) k_query_fp64_tiles<0, 8><<<(unsigned)tiles_grid<0, 8>(tiles, sms), 256, 0, stream>>>(s->d, a);
        else k_query_fp64_tiles<0, 4><<<(unsigned)tiles_grid<0, 4>(tiles, sms), 256, 0, stream>>>(s->d, a);
        break;
      case kTrd:
      case kTrap:
        if (big) k_query_fp64_tiles<1, 8><<<(unsigned)tiles_grid<1, 8>(tiles, sms), 256, 0, stream>>>(s->d, a);
        else k_query_fp64_tiles<1, 4><<<(unsigned)tiles_grid<1, 4>(tiles, sms), 256, 0, stream>>>(s->d, a);
        break;
      default:
        if (big) k_query_fp64_tiles<2, 8><<<(unsigned)tiles_grid<2, 8>(tiles, sms), 256, 0, stream>>>(s->d, a);
        else k_query_fp64_tiles<2, 4><<<(unsigned)tiles_grid<2, 4>(tiles, sms), 256, 0, stream>>>(s->d, a);
        break;
    }
    return cudaGetLastError();
  }
  int64_t blocks = (a.n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  switch (s->h.type) {
    case kBox: k_query_fp64<0><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a); break;
    case kTrd:
    case kTrap: k_query_fp64<1><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a); break;
    case kBool: k_query_fp64<4><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a); break;
    default: k_query_fp64<2><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a); break;
  }
  return cudaGetLastError();
}

#ifdef GV_DEBUG
cudaError_t debug_read_query64(unsigned long long out[2], bool clear) { return dbg_read(out, clear); }
#endif

}  // namespace gv
