// query_fp64.cu -- the plain binary64 query pass: one thread per track, the
// solid descriptor staged in shared memory, grid-stride over the basket.
#include "gv_debug.cuh"
#include "gv_internal.h"
#include "solid_fp64.cuh"

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

cudaError_t launch_query_fp64(const gv_solid* s, const QueryArgs& a, cudaStream_t stream) {
  if (a.n == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (a.n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * 8;
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
