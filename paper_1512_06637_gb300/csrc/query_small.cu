// query_small.cu -- the binary32 pass for small baskets in one launch.
#include "gv_debug.cuh"
#include "gv_internal.h"
#include "solid_fp32.cuh"
#include "solid_fp64.cuh"

namespace gv {

__device__ __forceinline__ void stage_desc_small(Desc& dst, const Desc* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 16); i += blockDim.x) d[i] = s[i];
}

// Small baskets (at most kFusedMax tracks) in one launch: the binary32 pass evaluates a track it
// cannot certify in binary64 on the spot (the same binary64 functions as the refinement pass, so
// the same bits) instead of appending it to a worklist; each block writes how many tracks it
// evaluated in binary64 to slots[blockIdx.x].  A call is then one launch with no counter reset:
// for a basket this small the launches, not the tracks, set the time.
constexpr int64_t kFusedMax = 65536;
template <int FAMILY>
__global__ void __launch_bounds__(256) k_query_fused(const Desc* __restrict__ desc, QueryArgs a,
                                                     uint32_t* __restrict__ slots) {
  __shared__ Desc S;
  stage_desc_small(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f32::kWantCode : 0u) | (a.din ? f32::kWantDin : 0u) |
                        (a.dout ? f32::kWantDout : 0u) | (a.sin ? f32::kWantSin : 0u) |
                        (a.sout ? f32::kWantSout : 0u);
  const bool dirs = want & (f32::kWantDin | f32::kWantDout);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool flag = false;
  if (i < a.n) {
    const f32::TrackF T = f32::load_track<(FAMILY >= 2)>(
        reinterpret_cast<const uint2*>(a.x), reinterpret_cast<const uint2*>(a.y), reinterpret_cast<const uint2*>(a.z),
        reinterpret_cast<const uint2*>(a.u), reinterpret_cast<const uint2*>(a.v), reinterpret_cast<const uint2*>(a.w),
        i, dirs);
    GV_DCHECK(!dirs || dbg_unit(a.u[i], a.v[i], a.w[i]), kDbgDirection, i);
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
    } else {
      const unsigned w64 = (a.inside ? f64::kWantCode : 0u) | (a.din ? f64::kWantDin : 0u) |
                           (a.dout ? f64::kWantDout : 0u) | (a.sin ? f64::kWantSin : 0u) |
                           (a.sout ? f64::kWantSout : 0u);
      f64::Track T64{a.x[i], a.y[i], a.z[i], 0, 0, 0};
      if (dirs) { T64.u = a.u[i]; T64.v = a.v[i]; T64.w = a.w[i]; }
      f64::Result R64;
      if (FAMILY == 0) f64::box_query(S, T64, w64, R64);
      else if (FAMILY == 1) f64::planar_query(S, T64, w64, R64);
      else f64::pcon_query(S, T64, w64, R64);
      if (a.inside) a.inside[i] = (int8_t)R64.code;
      if (a.din) a.din[i] = R64.din;
      if (a.dout) a.dout[i] = R64.dout;
      if (a.sin) a.sin[i] = R64.sin;
      if (a.sout) a.sout[i] = R64.sout;
    }
  }
  const int c = __syncthreads_count(flag);
  if (threadIdx.x == 0) slots[blockIdx.x] = (uint32_t)c;
}

#ifdef GV_DEBUG
cudaError_t debug_read_query_small(unsigned long long out[2], bool clear) { return dbg_read(out, clear); }
#endif

bool launch_query_small(const gv_solid* s, const QueryArgs& a, uint32_t* slots, cudaStream_t stream,
                        int* fused_blocks) {
  if (fused_blocks) *fused_blocks = 0;
  if (!(a.n > 0 && a.n <= kFusedMax && s->h.type != kBool && !(s->h.flags & kFp64Only))) return false;
  const unsigned blocks = (unsigned)((a.n + 255) / 256);
  switch (s->h.type) {
    case kBox: k_query_fused<0><<<blocks, 256, 0, stream>>>(s->d, a, slots); break;
    case kTrd:
    case kTrap: k_query_fused<1><<<blocks, 256, 0, stream>>>(s->d, a, slots); break;
    case kTube: k_query_fused<2><<<blocks, 256, 0, stream>>>(s->d, a, slots); break;
    default: k_query_fused<3><<<blocks, 256, 0, stream>>>(s->d, a, slots); break;
  }
  if (fused_blocks) *fused_blocks = (int)blocks;
  return true;
}

}  // namespace gv
