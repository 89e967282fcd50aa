// query_fp32.cu -- the binary32 bulk pass with binary64 refinement.
//
// Pass 1 (k_query_fp32): one thread per track; the solid descriptor staged in
// shared memory; inputs read as raw 64-bit words and split into binary32 pairs
// with integer operations; every certified result is written; the indices of
// the others are appended to a worklist (one atomicAdd per warp after a ballot).
// Pass 2 (k_refine_fp64): the same binary64 evaluation as the plain FP64 pass,
// over the worklist only; its length is read on the device, so the two launches
// need no host round trip.
#include "gv_internal.h"
#include "solid_fp32.cuh"
#include "solid_fp64.cuh"

namespace gv {

__device__ __forceinline__ void stage_desc32(Desc& dst, const Desc* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 16); i += blockDim.x) d[i] = s[i];
}

template <int FAMILY>
__global__ void __launch_bounds__(256, FAMILY == 0 ? 4 : (FAMILY == 1 ? 2 : 3)) k_query_fp32(const Desc* __restrict__ desc, QueryArgs a,
                                                    uint32_t* __restrict__ worklist,
                                                    unsigned long long* __restrict__ counter) {
  __shared__ Desc S;
  stage_desc32(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f32::kWantCode : 0u) | (a.din ? f32::kWantDin : 0u) |
                        (a.dout ? f32::kWantDout : 0u) | (a.sin ? f32::kWantSin : 0u) |
                        (a.sout ? f32::kWantSout : 0u);
  const bool dirs = want & (f32::kWantDin | f32::kWantDout);
  const uint2 *X = reinterpret_cast<const uint2*>(a.x), *Y = reinterpret_cast<const uint2*>(a.y),
              *Z = reinterpret_cast<const uint2*>(a.z), *Ux = reinterpret_cast<const uint2*>(a.u),
              *Uy = reinterpret_cast<const uint2*>(a.v), *Uz = reinterpret_cast<const uint2*>(a.w);
  const unsigned lane = threadIdx.x & 31u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // Polycones of several sections: inside and outside tracks take different paths (one
  // section and the exit search, against every section and the entry search), so each block first sorts
  // its chunk of tracks by a binary32 estimate of the side and hands inside tracks to the
  // first warps and outside tracks to the last; results do not depend on the estimate.
  __shared__ uint16_t perm[256];
  __shared__ int n_side[2];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
    int64_t i = base + threadIdx.x;
    if (FAMILY == 3 && S.nz > 2) {
      if (threadIdx.x < 2) n_side[threadIdx.x] = 0;
      __syncthreads();
      const bool in_est = i < a.n && f32::inside_estimate(S, X, Y, Z, i);
      const int at = in_est ? atomicAdd(&n_side[0], 1) : (int)blockDim.x - 1 - atomicAdd(&n_side[1], 1);
      perm[at] = (uint16_t)threadIdx.x;
      __syncthreads();
      i = base + perm[threadIdx.x];
      __syncthreads();
    }
    const bool valid = i < a.n;
    bool flag = false;
    if (valid) {
      const f32::TrackF T = f32::load_track<(FAMILY >= 2)>(X, Y, Z, Ux, Uy, Uz, i, dirs);
      f32::R32 R;
      R.flag = T.bad;
      R.code = 1;
      R.din = R.dout = R.sin = R.sout = 0.f;
      if (!R.flag) {
        if (FAMILY == 0) f32::box32(S, T, want, R);
        else if (FAMILY == 1) f32::planar32(S, T, want, R);
        else if (FAMILY == 2) f32::pcon32<true>(S, T, want, R);
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
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (m) {
      unsigned long long at = 0;
      const int leader = __ffs(m) - 1;
      if ((int)lane == leader) at = atomicAdd(counter, (unsigned long long)__popc(m));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (flag) worklist[at + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
    }
  }
}

template <int FAMILY>
__global__ void __launch_bounds__(256) k_refine_fp64(const Desc* __restrict__ desc, QueryArgs a,
                                                     const uint32_t* __restrict__ worklist,
                                                     const unsigned long long* __restrict__ counter) {
  __shared__ Desc S;
  stage_desc32(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f64::kWantCode : 0u) | (a.din ? f64::kWantDin : 0u) |
                        (a.dout ? f64::kWantDout : 0u) | (a.sin ? f64::kWantSin : 0u) |
                        (a.sout ? f64::kWantSout : 0u);
  const int64_t nref = (int64_t)*counter;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nref; j += stride) {
    const int64_t i = worklist[j];
    f64::Track T{a.x[i], a.y[i], a.z[i], 0, 0, 0};
    if (want & (f64::kWantDin | f64::kWantDout)) { T.u = a.u[i]; T.v = a.v[i]; T.w = a.w[i]; }
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
}

cudaError_t launch_query_fp32(const gv_solid* s, const QueryArgs& a, uint32_t* worklist,
                              unsigned long long* counter, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess || a.n == 0) return e;
  const int threads = 256;
  int64_t blocks = (a.n + threads - 1) / threads;
  const int sms = sm_count();
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  const unsigned rblocks = (unsigned)sms * 2;
  switch (s->h.type) {
    case kBox:
      k_query_fp32<0><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      k_refine_fp64<0><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    case kTrd:
    case kTrap:
      k_query_fp32<1><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      k_refine_fp64<1><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    case kTube:
      k_query_fp32<2><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      k_refine_fp64<2><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    default:
      k_query_fp32<3><<<(unsigned)blocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      k_refine_fp64<2><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
  }
  return cudaGetLastError();
}

}  // namespace gv
