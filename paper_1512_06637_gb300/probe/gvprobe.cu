// gvprobe.cu -- throughput probes for the roofline denominators that the copy and GEMM
// measurements do not give: binary32 and binary64 multiply-add rates, an integer-pipe
// rate, and the warp-instruction issue rate.  Measurement infrastructure for the
// benchmark only (libgvprobe.so); the geometry library does not use it.
//
// Each kernel runs `iters` rounds of 16 unrolled steps over 8 independent chains per
// thread (enough independent work per warp to cover the pipes' latency at full
// occupancy) and returns its elapsed device time from CUDA events on the given stream.
// Work per thread and launch:
//   gvp_fma32  16 * 8 * iters binary32 fused multiply-adds (2 flops each)
//   gvp_fma64  the same in binary64
//   gvp_alu    16 * 8 * iters steps of x = funnel_shift(x, x, 3) ^ y (shift and logic ops)
//   gvp_issue  16 * iters rounds of 4 binary32 multiply-adds and 4 integer steps on
//              separate chains: the warp instructions can go to two pipes, so the rate
//              is set by instruction issue
// The chains' results are folded into `sink` so that no work can be dropped.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void k_fma32(float* sink, int iters, float b, float c) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; j++) a[j] = (float)(threadIdx.x + j);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int j = 0; j < 8; j++) a[j] = fmaf(a[j], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; j++) s += a[j];
  if (s == -1.f) sink[blockIdx.x] = s;
}

__global__ void k_fma64(double* sink, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; j++) a[j] = (double)(threadIdx.x + j);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; j++) s += a[j];
  if (s == -1.0) sink[blockIdx.x] = s;
}

__global__ void k_alu(uint32_t* sink, int iters, uint32_t y) {
  uint32_t x[8];
#pragma unroll
  for (int j = 0; j < 8; j++) x[j] = threadIdx.x * 2654435761u + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int j = 0; j < 8; j++) x[j] = __funnelshift_l(x[j], x[j], 3) ^ y;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s ^= x[j];
  if (s == 0xFFFFFFFFu) sink[blockIdx.x] = s;
}

__global__ void k_issue(float* sink, int iters, float b, float c, uint32_t y) {
  float a[4];
  uint32_t x[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    a[j] = (float)(threadIdx.x + j);
    x[j] = threadIdx.x * 2654435761u + j;
  }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int j = 0; j < 4; j++) {
        a[j] = fmaf(a[j], b, c);
        x[j] = __funnelshift_l(x[j], x[j], 3) ^ y;
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 4; j++) s += a[j] + (float)(x[j] & 1u);
  if (s == -1.f) sink[blockIdx.x] = s;
}

template <class F>
int timed(F launch, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 1; }
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? 0 : 1;
}

}  // namespace

extern "C" {

// sink: device buffer of at least `blocks` elements of the kernel's type (4 or 8 bytes).
// Returns 0 on success (elapsed time in *ms), 1 on a CUDA error.
int gvp_fma32(int blocks, int threads, int iters, void* sink, void* stream, float* ms) {
  cudaStream_t st = (cudaStream_t)stream;
  return timed([&] { k_fma32<<<blocks, threads, 0, st>>>((float*)sink, iters, 1.0000001f, 1e-7f); }, st, ms);
}
int gvp_fma64(int blocks, int threads, int iters, void* sink, void* stream, float* ms) {
  cudaStream_t st = (cudaStream_t)stream;
  return timed([&] { k_fma64<<<blocks, threads, 0, st>>>((double*)sink, iters, 1.0000000001, 1e-12); }, st, ms);
}
int gvp_alu(int blocks, int threads, int iters, void* sink, void* stream, float* ms) {
  cudaStream_t st = (cudaStream_t)stream;
  return timed([&] { k_alu<<<blocks, threads, 0, st>>>((uint32_t*)sink, iters, 0x9E3779B9u); }, st, ms);
}
int gvp_issue(int blocks, int threads, int iters, void* sink, void* stream, float* ms) {
  cudaStream_t st = (cudaStream_t)stream;
  return timed([&] { k_issue<<<blocks, threads, 0, st>>>((float*)sink, iters, 1.0000001f, 1e-7f, 0x9E3779B9u); },
               st, ms);
}

}  // extern "C"
