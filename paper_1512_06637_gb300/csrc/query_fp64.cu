// query_fp64.cu -- the plain binary64 query pass: one thread per track, the
// solid descriptor staged in shared memory, grid-stride over the basket.  With scratch
// for it (a workspace), a primitive solid's basket is first ordered by work class within
// tiles (k_sort_classes), and the pass takes its tracks in that order: the pass is bound by
// the FP64 pipe, which spends the same on a warp instruction whatever its active lanes, so
// warps of one class (inside, outside and entering, outside and missing, near a surface)
// run fewer instructions for the same tracks.
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

// Within each tile of kSortTile consecutive positions, perm lists the tile's track indices
// grouped by work class (f32::track_class, in its order), each group in index order.
constexpr int kSortTile = 4096;
constexpr int kSortThreads = 256;
constexpr int kSortGroups = kSortTile / 32;  // groups of 32 consecutive positions
// baskets smaller than this are not sorted (the extra launch would not pay)
constexpr int64_t kSortMin = int64_t(1) << 16;

__global__ void __launch_bounds__(kSortThreads) k_sort_classes(const Desc* __restrict__ desc, QueryArgs a,
                                                              uint32_t* __restrict__ perm) {
  constexpr uint32_t NC = f32::kClasses;
  __shared__ Desc S;
  __shared__ uint8_t cls[kSortTile];
  __shared__ uint32_t cnt[NC][kSortGroups];  // per class and group: count, then exclusive prefix
  __shared__ uint32_t off[NC];               // first position of each class in the tile
  stage_desc(S, desc);
  __syncthreads();
  const bool dirs = a.din || a.dout;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  for (int64_t t0 = (int64_t)blockIdx.x * kSortTile; t0 < a.n; t0 += (int64_t)gridDim.x * kSortTile) {
    const int64_t len = a.n - t0 < kSortTile ? a.n - t0 : kSortTile;
    for (int g = warp; g < kSortGroups; g += nwarps) {
      const int j = g * 32 + (int)lane;
      uint32_t c = NC;  // no track at this position
      if (j < len) {
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
        c = f32::track_class(S, x, y, z, u, v, w, dirs);
      }
      cls[j] = (uint8_t)c;
#pragma unroll
      for (uint32_t q = 0; q < NC; q++) {
        const unsigned m = __ballot_sync(0xffffffffu, c == q);
        if (lane == 0) cnt[q][g] = __popc(m);
      }
    }
    __syncthreads();
    // exclusive prefix of each class's counts over the groups: one warp per class
    if (warp < NC) {
      constexpr int G = kSortGroups / 32;
      uint32_t v[G], sum = 0;
#pragma unroll
      for (int e = 0; e < G; e++) {
        v[e] = cnt[warp][lane * G + e];
        sum += v[e];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int e = 0; e < G; e++) {
        cnt[warp][lane * G + e] = run;
        run += v[e];
      }
      if (lane == 31) off[warp] = incl;  // the class's total, turned into offsets below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (uint32_t q = 0; q < NC; q++) {
        const uint32_t t = off[q];
        off[q] = run;
        run += t;
      }
    }
    __syncthreads();
    for (int g = warp; g < kSortGroups; g += nwarps) {
      const int j = g * 32 + (int)lane;
      const uint32_t c = cls[j];
      uint32_t pos = 0;
#pragma unroll
      for (uint32_t q = 0; q < NC; q++) {
        const unsigned m = __ballot_sync(0xffffffffu, c == q);
        if (c == q) pos = off[q] + cnt[q][g] + __popc(m & below);
      }
      if (c < NC) perm[t0 + pos] = (uint32_t)(t0 + j);
    }
    __syncthreads();  // the tile's shared arrays are reused by the next tile
  }
}

template <int FAMILY>
__global__ void __launch_bounds__(256) k_query_fp64(const Desc* __restrict__ desc, QueryArgs a,
                                                    const uint32_t* __restrict__ perm) {
  __shared__ Desc S;
  stage_desc(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f64::kWantCode : 0u) | (a.din ? f64::kWantDin : 0u) |
                        (a.dout ? f64::kWantDout : 0u) | (a.sin ? f64::kWantSin : 0u) |
                        (a.sout ? f64::kWantSout : 0u);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride) {
    const int64_t i = perm ? (int64_t)__ldg(perm + p) : p;  // the track at position p
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

cudaError_t launch_query_fp64(const gv_solid* s, const QueryArgs& a, uint32_t* perm, cudaStream_t stream) {
  if (a.n == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (a.n + threads - 1) / threads;
  const int sms = sm_count();
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  const uint32_t* order = nullptr;
  if (perm && s->h.type != kBool && a.n >= kSortMin) {
    int64_t sb = (a.n + kSortTile - 1) / kSortTile;
    if (sb > (int64_t)sms * 4) sb = (int64_t)sms * 4;
    k_sort_classes<<<(unsigned)sb, kSortThreads, 0, stream>>>(s->d, a, perm);
    order = perm;
  }
  switch (s->h.type) {
    case kBox: k_query_fp64<0><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, order); break;
    case kTrd:
    case kTrap: k_query_fp64<1><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, order); break;
    case kBool: k_query_fp64<4><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, nullptr); break;
    default: k_query_fp64<2><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, order); break;
  }
  return cudaGetLastError();
}

#ifdef GV_DEBUG
cudaError_t debug_read_query64(unsigned long long out[2], bool clear) { return dbg_read(out, clear); }
#endif

}  // namespace gv
