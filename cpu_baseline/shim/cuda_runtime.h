// Host stand-ins for the CUDA qualifiers and round-to-nearest intrinsics used by the
// library's binary64 solid code, so that the CPU baseline compiles that same code for the
// host (plain C++ built with -ffp-contract=off: every + - * rounds once, to nearest, as the
// intrinsics do on the device; / and sqrt are IEEE on both).
#pragma once
#include <cmath>
#include <cstdint>

#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))

static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dsqrt_rn(double a) { return std::sqrt(a); }
using std::copysign;
using std::fabs;
using std::nan;
using std::sqrt;
