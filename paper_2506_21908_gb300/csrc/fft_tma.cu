// xy pass of the kinetic term with its planes brought into shared memory by the bulk
// asynchronous copy engine (FP32, two-factor sizes).
//
// The plain two-factor pass reads its plane from HBM into registers, so the bytes in flight are
// bounded by the warps resident on the SM.  Here each CTA is persistent and double-buffers whole
// planes: while it transforms plane j in one buffer, the row copies of plane j + grid
// (`cp.async.bulk`, one 16-byte-aligned row each, completion counted in bytes on an mbarrier)
// fill the other.  The first DFT stage reads the buffer in place; the rest of the transform is
// that of k_fft_xy2 (one exchange per axis, the last stage writing HBM from registers), so the
// results are the same bits.  (The z pass gains nothing from this form: with one exchange its
// register-fed kernel keeps four CTAs per SM busy, against three for a double-buffered slab.)
//
// Source and destination may be the same array: a CTA reads each plane (by the copy engine)
// before it writes it, and no other CTA touches it.
//
// Every mbarrier wait has an iteration limit: on expiry the CTA sets bit 2 of the error word,
// waits once more (again with a limit) for the copy in flight and carries on with what the
// buffer holds; every index stays in bounds, and the host reports the flag.
#include <cstdint>

#include "bulk.cuh"
#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"

namespace tddft {

namespace {

// N rows of N complex values (row r at g + r * stride) into a buffer with row pitch P; called by
// the 32 lanes of warp 0.  Row bytes N * 8, the pitch P * 8 and the row addresses are
// multiples of 16 for every size used here (N even).
template <int N, int P>
__device__ __forceinline__ void issue_rows(const float2* g, size_t stride, float2* buf, uint32_t bar, int lane) {
  constexpr uint32_t ROW = N * sizeof(float2);
  if (lane == 0) bulk_expect(bar, ROW * N);
  __syncwarp();
  for (int row = lane; row < N; row += 32) bulk_copy(buf + row * P, g + (size_t)row * stride, ROW, bar);
}

// Threads and resident CTAs: 256 threads; the two 36 KB buffers of a 64^2 plane allow three
// CTAs per SM.  (512 threads at two CTAs per SM, one item per thread and side, were slower:
// 0.190 against 0.161 ms per pass at 64^3 x 208 components.)  At 96^2 the two 78 KB buffers leave
// one CTA per SM, and the register-fed pass is faster (7.2 against 9.0 ms per pass at 96^3 x 2048
// components), so 96 takes that pass.
template <int N> struct XyTmaThreads { static constexpr int value = 256; };
template <int N> struct XyTmaBlocks { static constexpr int value = 4; };
template <> struct XyTmaBlocks<64> { static constexpr int value = 3; };
template <> struct XyTmaBlocks<48> { static constexpr int value = 3; };

}  // namespace

// Barriers.  A stage whose items read and write the same cells (the y A side in both
// directions, whose rows n0 + R1 q are also its output rows K0 R1 + n0) runs in place without
// one.  A stage whose items share a row (the x sides) only needs the row's items, which sit on
// neighbouring lanes of one warp when the item count per row divides 32 and the CTA size.
template <int N, bool INV>
__global__ void __launch_bounds__(XyTmaThreads<N>::value, XyTmaBlocks<N>::value)
k_fft_xy2_tma(const float2* src, float2* dst, const float2* __restrict__ twg, int nplanes, int* err) {
  using C = float2;
  using T = TF<C, N, INV>;
  constexpr int NT = XyTmaThreads<N>::value;
  constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  constexpr int RS = TFPitch<N>::value;
  constexpr int IA = N * R1, IB = N * R2;
  constexpr int PA = (IA + NT - 1) / NT, PB = (IB + NT - 1) / NT;
  constexpr bool ROW1 = (32 % R1 == 0) && (NT % R1 == 0);  // x A-side rows within a warp
  constexpr bool ROW2 = (32 % R2 == 0) && (NT % R2 == 0);  // x B-side rows within a warp
  constexpr bool ROW12 = ROW1 && R1 == R2;                 // and on the same lanes for both sides
  static_assert(ROW1, "R1 divides the warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf0 = tw + N;
  C* buf1 = buf0 + N * RS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(buf1 + N * RS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = sm_addr(&bars[0]), bar1 = sm_addr(&bars[1]);
  if (threadIdx.x == 0) bulk_init(bar0, bar1);
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  __syncthreads();
  int pl = blockIdx.x;
  if (pl < nplanes && warp == 0) issue_rows<N, RS>(src + (size_t)pl * N * N, N, buf0, bar0, lane);
  C v[PA][R2];
  C u[PB][R1];
  // Buffer schedule: at the start of plane j the copies of plane j + grid go to the other buffer,
  // whose last reader (plane j - grid) ended with the CTA barrier closing the previous step.
  for (int it = 0; pl < nplanes; ++it, pl += gridDim.x) {
    const int sb = it & 1;
    C* s = sb ? buf1 : buf0;
    const int nx = pl + gridDim.x;
    if (nx < nplanes && warp == 0) issue_rows<N, RS>(src + (size_t)nx * N * N, N, sb ? buf0 : buf1, sb ? bar0 : bar1, lane);
    bulk_wait(sb ? bar1 : bar0, (uint32_t)(it >> 1) & 1u, err, 2);
    C* o = dst + (size_t)pl * N * N;
    if (!INV) {
      // x, A side in place: item (y, n0); a row's items share a warp
#pragma unroll
      for (int p = 0; p < PA; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IA % NT == 0 || i < IA) {
          const int y = i / R1, n0 = i - y * R1;
#pragma unroll
          for (int q = 0; q < R2; ++q) v[p][q] = s[y * RS + n0 + R1 * q];
        }
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < PA; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IA % NT == 0 || i < IA) {
          const int y = i / R1, n0 = i - y * R1;
          T::a_side(v[p], n0, tw);
#pragma unroll
          for (int k0 = 0; k0 < R2; ++k0) s[y * RS + k0 * R1 + (n0 + k0) % R1] = v[p][k0];
        }
      }
      if constexpr (ROW12) __syncwarp(); else __syncthreads();
      // x, B side: item (y, K0)
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int y = i / R2, k0 = i - y * R2;
#pragma unroll
          for (int n0 = 0; n0 < R1; ++n0) u[p][n0] = s[y * RS + k0 * R1 + (n0 + k0) % R1];
        }
      }
      if constexpr (ROW2) __syncwarp(); else __syncthreads();
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int y = i / R2, k0 = i - y * R2;
          T::b_side(u[p], k0, tw);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) s[y * RS + k0 + R2 * k1] = u[p][k1];
        }
      }
      __syncthreads();
      // y, A side in place: item (x, n0)
#pragma unroll
      for (int p = 0; p < PA; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IA % NT == 0 || i < IA) {
          const int n0 = i / N, x = i - n0 * N;
#pragma unroll
          for (int q = 0; q < R2; ++q) v[p][q] = s[(n0 + R1 * q) * RS + x];
          T::a_side(v[p], n0, tw);
#pragma unroll
          for (int k0 = 0; k0 < R2; ++k0) s[(k0 * R1 + n0) * RS + x] = v[p][k0];
        }
      }
      __syncthreads();
      // y, B side: item (x, K0) -> HBM
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int k0 = i / N, x = i - k0 * N;
#pragma unroll
          for (int n0 = 0; n0 < R1; ++n0) u[p][n0] = s[(k0 * R1 + n0) * RS + x];
          T::b_side(u[p], k0, tw);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) o[(k0 + R2 * k1) * N + x] = u[p][k1];
        }
      }
    } else {
      // y, B side in place: item (x, K0); a column's items sit in several warps, so every read of
      // the plane precedes the first write
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int k0 = i / N, x = i - k0 * N;
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) u[p][k1] = s[(k0 + R2 * k1) * RS + x];
        }
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int k0 = i / N, x = i - k0 * N;
          T::b_side(u[p], k0, tw);
#pragma unroll
          for (int n0 = 0; n0 < R1; ++n0) s[(k0 * R1 + n0) * RS + x] = u[p][n0];
        }
      }
      __syncthreads();
      // y, A side in place: item (x, n0)
#pragma unroll
      for (int p = 0; p < PA; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IA % NT == 0 || i < IA) {
          const int n0 = i / N, x = i - n0 * N;
#pragma unroll
          for (int k0 = 0; k0 < R2; ++k0) v[p][k0] = s[(k0 * R1 + n0) * RS + x];
          T::a_side(v[p], n0, tw);
#pragma unroll
          for (int n1 = 0; n1 < R2; ++n1) s[(n0 + R1 * n1) * RS + x] = v[p][n1];
        }
      }
      __syncthreads();
      // x, B side: item (y, K0)
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int y = i / R2, k0 = i - y * R2;
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) u[p][k1] = s[y * RS + k0 + R2 * k1];
        }
      }
      if constexpr (ROW2) __syncwarp(); else __syncthreads();
#pragma unroll
      for (int p = 0; p < PB; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IB % NT == 0 || i < IB) {
          const int y = i / R2, k0 = i - y * R2;
          T::b_side(u[p], k0, tw);
#pragma unroll
          for (int n0 = 0; n0 < R1; ++n0) s[y * RS + k0 * R1 + (n0 + k0) % R1] = u[p][n0];
        }
      }
      if constexpr (ROW12) __syncwarp(); else __syncthreads();
      // x, A side -> HBM: item (y, n0)
#pragma unroll
      for (int p = 0; p < PA; ++p) {
        const int i = threadIdx.x + p * NT;
        if (IA % NT == 0 || i < IA) {
          const int y = i / R1, n0 = i - y * R1;
#pragma unroll
          for (int k0 = 0; k0 < R2; ++k0) v[p][k0] = s[y * RS + k0 * R1 + (n0 + k0) % R1];
          T::a_side(v[p], n0, tw);
#pragma unroll
          for (int n1 = 0; n1 < R2; ++n1) o[y * N + n0 + R1 * n1] = v[p][n1];
        }
      }
    }
    __syncthreads();
  }
}

bool fft_xy_tma_supported(int N) { return N == 16 || N == 24 || N == 32 || N == 48 || N == 64; }

template <int N>
static cudaError_t xy_tma_n(cudaStream_t st, const void* src, void* dst, int nbatch, const void* tw, bool inv,
                            int* err) {
  const size_t smem = (size_t)(N + 2 * N * TFPitch<N>::value) * sizeof(float2) + 2 * sizeof(uint64_t);
  auto kf = inv ? k_fft_xy2_tma<N, true> : k_fft_xy2_tma<N, false>;
  static int per_sm[2] = {0, 0};
  static int sms = 0;
  int& ps = per_sm[inv ? 1 : 0];
  if (!ps) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kf, XyTmaThreads<N>::value, smem)) != cudaSuccess) return e;
    if (ps < 1) return cudaErrorInvalidConfiguration;
  }
  const int nplanes = N * nbatch;
  const int grid = std::min(nplanes, sms * ps);
  kf<<<grid, XyTmaThreads<N>::value, smem, st>>>((const float2*)src, (float2*)dst, (const float2*)tw, nplanes, err);
  return cudaGetLastError();
}

cudaError_t launch_fft_xy_tma(cudaStream_t st, int N, const void* src, void* dst, int nbatch, const void* tw, bool inv,
                              int* err) {
  if (nbatch <= 0) return cudaSuccess;
  if (((uintptr_t)src & 15) != 0 || !err) return cudaErrorInvalidValue;
  switch (N) {
    case 16: return xy_tma_n<16>(st, src, dst, nbatch, tw, inv, err);
    case 24: return xy_tma_n<24>(st, src, dst, nbatch, tw, inv, err);
    case 32: return xy_tma_n<32>(st, src, dst, nbatch, tw, inv, err);
    case 48: return xy_tma_n<48>(st, src, dst, nbatch, tw, inv, err);
    case 64: return xy_tma_n<64>(st, src, dst, nbatch, tw, inv, err);
    default: return cudaErrorNotSupported;
  }
}


cudaError_t set_first_wait_fft(unsigned polls) { return cudaMemcpyToSymbol(g_first_wait, &polls, sizeof(polls)); }

}  // namespace tddft
