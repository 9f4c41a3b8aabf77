// Small device helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>

namespace tddft {

// 96 = 8 x 12: 384 threads give every two-factor item loop (768 and 1152 items) and every
// radix-stage butterfly loop (1152, 2304, 3072 butterflies) whole iterations.
template <int N> struct FFTThreads { static constexpr int value = (N >= 96) ? 384 : 256; };

// Minimum resident CTAs per SM requested from the register allocator: several CTAs of the
// FP32 passes up to 64^3 fit without spills, two of the FP32 96^3 passes (80 KB of shared
// memory each); FP64 variants keep their registers.
template <typename R, int N> struct FFTMinBlocks { static constexpr int value = 1; };
template <int N> struct FFTMinBlocks<float, N> { static constexpr int value = (N <= 64) ? 1024 / FFTThreads<N>::value : 2; };

template <int N> __device__ __forceinline__ int freq(int i) { return i < N / 2 ? i : i - N; }

// FP32 Chebyshev arithmetic with the series constants as float pairs hi + lo (see
// split_constants): (x - c p) / Delta with c = {hi, lo} and 1 / Delta = {hi, lo} ...
__device__ __forceinline__ float shifted_f(float x, float p, const float* c, const float* id) {
  const float d = (x - c[0] * p) - c[1] * p;
  return d * id[0] + d * id[1];
}
// ... and a z for the complex constant z = {re hi, im hi, re lo, im lo}.
__device__ __forceinline__ float2 cmul_split(float2 a, const float* z) {
  return make_float2((z[0] * a.x - z[1] * a.y) + (z[2] * a.x - z[3] * a.y),
                     (z[0] * a.y + z[1] * a.x) + (z[2] * a.y + z[3] * a.x));
}

// Accumulator updates acc += sum_j z_j t_j in float-float arithmetic, rounded to FP32 once.
// Rounding each product of FP32 data with a fixed FP32 constant (and each partial sum) is biased
// for a given constant: summed over a state the errors do not cancel, and the series output gains
// or loses ~1e-8 of its norm per series, every step in the same direction (an FP32 path drifted
// by ~6e-8 in norm per step).  Here every product is split exactly (p + pe = a b, by a fused
// multiply-add) and every sum is exact (hi + lo, Knuth's two-sum), so the update is the exact
// value rounded once.  __fmul_rn / __fadd_rn are never contracted into multiply-adds, which would
// break the splits.
__device__ __forceinline__ void ff_madd(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo += e + pe;
}
// (hi, lo) += t z for the complex constant z = {re hi, im hi, re lo, im lo}.
__device__ __forceinline__ void ff_cmadd(float2& hi, float2& lo, float2 t, const float* z) {
  ff_madd(hi.x, lo.x, z[0], t.x);
  ff_madd(hi.x, lo.x, -z[1], t.y);
  ff_madd(hi.y, lo.y, z[0], t.y);
  ff_madd(hi.y, lo.y, z[1], t.x);
  lo.x += z[2] * t.x - z[3] * t.y;
  lo.y += z[2] * t.y + z[3] * t.x;
}

#define TDDFT_DISPATCH_N(N, CALL)          \
  switch (N) {                             \
    case 8: { constexpr int NN = 8; return CALL; }   \
    case 12: { constexpr int NN = 12; return CALL; } \
    case 16: { constexpr int NN = 16; return CALL; } \
    case 24: { constexpr int NN = 24; return CALL; } \
    case 32: { constexpr int NN = 32; return CALL; } \
    case 48: { constexpr int NN = 48; return CALL; } \
    case 64: { constexpr int NN = 64; return CALL; } \
    case 96: { constexpr int NN = 96; return CALL; } \
    default: return cudaErrorInvalidValue;           \
  }

template <typename R> __device__ __forceinline__ void sincos_r(R x, R* s, R* c);
template <> __device__ __forceinline__ void sincos_r<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void sincos_r<double>(double x, double* s, double* c) { sincos(x, s, c); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}


}  // namespace tddft
