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
