// query_fp32.cu -- the binary32 bulk pass with binary64 refinement.
//
// Pass 1 (k_query_fp32): one thread per track; the solid descriptor staged in
// shared memory; each thread stages its next track's raw 64-bit words in shared
// memory (cp.async) while it computes the current one, splits them into binary32
// pairs with integer operations; every certified result is written; the indices of
// the others are appended to a worklist (one atomicAdd per warp after a ballot).
// Pass 2 (k_refine_fp64): the same binary64 evaluation as the plain FP64 pass,
// over the worklist only; its length is read on the device, so the two launches
// need no host round trip.
#include "gv_debug.cuh"
#include "gv_internal.h"
#include "solid_fp32.cuh"
#include "solid_fp64.cuh"

namespace gv {

__device__ __forceinline__ void stage_desc32(Desc& dst, const Desc* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 16); i += blockDim.x) d[i] = s[i];
}

// Asynchronous global -> shared copies (8 bytes each) that the issuing thread waits for
// with cp.async.wait_group: a thread stages its next track while it computes the current
// one, so the loads' latency overlaps the arithmetic without holding registers.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Block shape of the one-track-per-thread pass per family (box, trd/trap, tube, cone):
// threads and resident blocks per SM, from the registers each family needs.
template <int FAMILY> struct Shape32 { static constexpr int threads = 256, blocks = 3; };
template <> struct Shape32<0> { static constexpr int threads = 288, blocks = 4; };
template <> struct Shape32<1> { static constexpr int threads = 288, blocks = 3; };

template <int FAMILY>
__global__ void __launch_bounds__(Shape32<FAMILY>::threads, Shape32<FAMILY>::blocks) k_query_fp32(const Desc* __restrict__ desc, QueryArgs a,
                                                    uint32_t* __restrict__ worklist,
                                                    unsigned long long* __restrict__ counter) {
  constexpr int NT = Shape32<FAMILY>::threads;
  __shared__ Desc S;
  __shared__ uint2 stage[2][6][NT];  // this thread's current and next track, raw words
  stage_desc32(S, desc);
  __syncthreads();
  const unsigned want = (a.inside ? f32::kWantCode : 0u) | (a.din ? f32::kWantDin : 0u) |
                        (a.dout ? f32::kWantDout : 0u) | (a.sin ? f32::kWantSin : 0u) |
                        (a.sout ? f32::kWantSout : 0u);
  const bool dirs = want & (f32::kWantDin | f32::kWantDout);
  const uint2* src[6] = {reinterpret_cast<const uint2*>(a.x), reinterpret_cast<const uint2*>(a.y),
                         reinterpret_cast<const uint2*>(a.z), reinterpret_cast<const uint2*>(a.u),
                         reinterpret_cast<const uint2*>(a.v), reinterpret_cast<const uint2*>(a.w)};
  const unsigned lane = threadIdx.x & 31u;
  const unsigned tid = threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // stage the words of track i into buffer b (nothing for i beyond the basket); one commit
  // group per call, so that wait_group<1> always means "all but the latest group landed"
  auto prefetch = [&](int64_t i, int b) {
    if (i < a.n) {
#pragma unroll
      for (int c = 0; c < 6; c++)
        if (c < 3 || dirs) cp_async8(&stage[b][c][tid], src[c] + i);
    }
    cp_async_commit();
  };
  int buf = 0;
  prefetch((int64_t)blockIdx.x * blockDim.x + tid, 0);
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
    const int64_t i = base + tid;
    prefetch(i + stride, buf ^ 1);
    cp_async_wait<1>();
    const bool valid = i < a.n;
    bool flag = false;
    if (valid) {
      const uint2 zero{0u, 0u};
      const f32::TrackF T = f32::track_from_words<(FAMILY >= 2)>(
          stage[buf][0][tid], stage[buf][1][tid], stage[buf][2][tid], dirs ? stage[buf][3][tid] : zero,
          dirs ? stage[buf][4][tid] : zero, dirs ? stage[buf][5][tid] : zero, dirs);
#ifdef GV_DEBUG
      if (dirs) {
        const uint2 bu = stage[buf][3][tid], bv = stage[buf][4][tid], bw = stage[buf][5][tid];
        GV_DCHECK(dbg_unit(__hiloint2double(bu.y, bu.x), __hiloint2double(bv.y, bv.x), __hiloint2double(bw.y, bw.x)),
                  kDbgDirection, i);
      }
#endif
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
    buf ^= 1;
  }
  cp_async_wait<0>();  // no copy outlives the block
}

// Results of one finished track: written when certified, else its index appended to
// the worklist of the binary64 pass.
__device__ __forceinline__ void finish_track(const QueryArgs& a, int64_t i, const f32::R32& R, uint32_t* worklist,
                                             unsigned long long* counter) {
  if (R.flag) {
    worklist[atomicAdd(counter, 1ull)] = (uint32_t)i;
    return;
  }
  if (a.inside) a.inside[i] = (int8_t)R.code;
  if (a.din) reinterpret_cast<unsigned long long*>(a.din)[i] = f32::f2d_bits(R.din);
  if (a.dout) reinterpret_cast<unsigned long long*>(a.dout)[i] = f32::f2d_bits(R.dout);
  if (a.sin) reinterpret_cast<unsigned long long*>(a.sin)[i] = f32::f2d_bits(R.sin);
  if (a.sout) reinterpret_cast<unsigned long long*>(a.sout)[i] = f32::f2d_bits(R.sout);
}

// Tube / cone / polycone with lane refill.  A track's distance walk visits one to several
// sections, and lanes of a warp finish at different times.  Each warp keeps one track
// per lane in registers (its point, direction and walk state) and loops: when at least
// half its lanes are idle, the idle lanes take the next tracks from a dispenser counter
// (one atomicAdd per warp) and run the setup (code, safeties, first section); then every
// busy lane advances its walk by one section; a lane whose walk ends writes its results
// and becomes idle.  Warps stay mostly full until the dispenser runs dry.
constexpr int kRefillIdle = 16;
// tube and one-section cones: the walk is one or two sections long, so the plain kernel
// (one track per thread, no refill) is used for them
constexpr bool kWalkOneSection = false;
// threads per block of the walk kernel and resident blocks per SM (the register budget sets
// them; 224-384 threads and 2-3 blocks measured within 4% of each other)
constexpr int kWalkThreads = 320;
constexpr int kWalkBlocks = 2;

template <int FAMILY>
__global__ void __launch_bounds__(kWalkThreads, kWalkBlocks) k_query_walk(const Desc* __restrict__ desc, QueryArgs a,
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
  constexpr bool TUBE = FAMILY == 2;
  unsigned long long* dispenser = counter + 1;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  bool busy = false, more = true;
  int64_t i = 0;
  f32::TrackF T;
  f32::R32 R;
  f32::Walk W;
  while (true) {
    const unsigned idle = __ballot_sync(0xffffffffu, !busy);
    if (more && (__popc(idle) >= kRefillIdle || idle == 0xffffffffu)) {
      unsigned long long first = 0;
      if (lane == 0) first = atomicAdd(dispenser, (unsigned long long)__popc(idle));
      first = __shfl_sync(0xffffffffu, first, 0);
      if (first + __popc(idle) >= (unsigned long long)a.n) more = false;
      if (!busy) {
        const unsigned long long j = first + __popc(idle & below);
        if (j < (unsigned long long)a.n) {
          i = (int64_t)j;
          T = f32::load_track<true>(X, Y, Z, Ux, Uy, Uz, i, dirs);
          GV_DCHECK(!dirs || dbg_unit(a.u[i], a.v[i], a.w[i]), kDbgDirection, i);
          R.flag = T.bad;
          R.code = 1;
          R.din = R.dout = R.sin = R.sout = 0.f;
          W.need_in = W.need_out = false;
          W.live = false;
          if (!R.flag) busy = f32::pcon_begin<TUBE>(S, T, want, R, W);
          if (!busy) finish_track(a, i, R, worklist, counter);
        }
      }
    }
    if (__ballot_sync(0xffffffffu, busy) == 0u) {
      if (!more) break;
      continue;
    }
    if (busy) {
      f32::pcon_step<TUBE>(S, T, W);
      if (!W.live) {
        f32::pcon_end(W, R);
        finish_track(a, i, R, worklist, counter);
        busy = false;
      }
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
  GV_DCHECK(nref <= a.n, kDbgWorklist, nref);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // consecutive entries go to consecutive blocks: a short worklist is spread over every
  // SM instead of filling the first few blocks (each entry is a long binary64 chain)
  for (int64_t j = (int64_t)threadIdx.x * gridDim.x + blockIdx.x; j < nref; j += stride) {
    const int64_t i = worklist[j];
    GV_DCHECK(i < a.n, kDbgIndex, i);
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

// The binary32 pass of one family: a grid of at most eight blocks' worth of tracks per SM
// (grid-stride loop inside).
template <int FAMILY>
void launch_pass32(const gv_solid* s, const QueryArgs& a, uint32_t* worklist, unsigned long long* counter,
                   cudaStream_t stream, int sms) {
  constexpr int T = Shape32<FAMILY>::threads;
  int64_t blocks = (a.n + T - 1) / T;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  k_query_fp32<FAMILY><<<(unsigned)blocks, T, 0, stream>>>(s->d, a, worklist, counter);
}

cudaError_t launch_query_fp32(const gv_solid* s, const QueryArgs& a, uint32_t* worklist,
                              unsigned long long* counter, cudaStream_t stream, int* fused_blocks) {
  // small baskets: one launch (query_small.cu)
  if (launch_query_small(s, a, worklist, stream, fused_blocks)) return cudaGetLastError();
  // counter[0]: worklist length; counter[1]: next track of the lane-refill dispenser
  cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned long long), stream);
  if (e != cudaSuccess || a.n == 0) return e;
  // boolean solids have no binary32 pass, and solids with features finer than binary32 resolves
  // are evaluated in binary64 too (nothing goes to the worklist)
  if (s->h.type == kBool || (s->h.flags & kFp64Only)) return launch_query_fp64(s, a, stream);
  const int threads = 256;
  int64_t blocks = (a.n + threads - 1) / threads;
  const int sms = sm_count();
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  // lane-refill kernel: resident blocks only, fed by the dispenser
  const unsigned wblocks = (unsigned)(blocks < (int64_t)sms * kWalkBlocks ? blocks : (int64_t)sms * kWalkBlocks);
  // the worklist holds at most n tracks: no more refinement blocks than that needs
  const unsigned rblocks = (unsigned)(blocks < (int64_t)sms * 2 ? blocks : (int64_t)sms * 2);
  switch (s->h.type) {
    case kBox:
      launch_pass32<0>(s, a, worklist, counter, stream, sms);
      k_refine_fp64<0><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    case kTrd:
    case kTrap:
      launch_pass32<1>(s, a, worklist, counter, stream, sms);
      k_refine_fp64<1><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    case kTube:
      if (kWalkOneSection)
        k_query_walk<2><<<wblocks, kWalkThreads, 0, stream>>>(s->d, a, worklist, counter);
      else
        launch_pass32<2>(s, a, worklist, counter, stream, sms);
      k_refine_fp64<2><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
    default:
      // without distances no track walks: one track per thread (measured 20% faster for the
      // code alone than the lane-refill pass, whose every refill waits on its loads)
      if ((s->h.nz > 2 || kWalkOneSection) && (a.din || a.dout))
        k_query_walk<3><<<wblocks, kWalkThreads, 0, stream>>>(s->d, a, worklist, counter);
      else
        launch_pass32<3>(s, a, worklist, counter, stream, sms);
      k_refine_fp64<2><<<rblocks, threads, 0, stream>>>(s->d, a, worklist, counter);
      break;
  }
  return cudaGetLastError();
}

#ifdef GV_DEBUG
cudaError_t debug_read_query32(unsigned long long out[2], bool clear) { return dbg_read(out, clear); }
#endif

}  // namespace gv
