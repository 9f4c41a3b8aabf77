// sm_103a kernels of the spinor propagation step.
//
//   k_fft_xy     one z-plane of one spinor component: 2D FFT along x then y in shared memory
//   k_fft_z      one y-slab of one component: FFT along z, multiply (kinetic 1/2|G+k+A|^2 or
//                Poisson 4 pi / G^2), inverse FFT along z -- the kinetic term of Eq. HNC-SDFT
//   k_proj_gather  c_{a,p,sigma} = sum_{r in S_a} beta~_p(r)^* psi_sigma(r) dV and D_a c
//                (the contraction of the separable projectors, Eq. Vps with the L.S block)
//   (k_epilogue, the pointwise Hamiltonian and Chebyshev update, is in epilogue.cu)
//   k_density    rho_v = sum_k w_k sum_i f_i {|u|^2, |d|^2, Re u d*, Im u d*}  (Eqs. rho1-rho3)
//   k_potential  locally collinear LSDA (Eqs. LC+ALDA2, LC+ALDA) and assembly of V_v
//   reductions   deterministic fixed-order block reductions for energies and norms
#include <cstdint>

#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"
#include "kepi.cuh"

namespace tddft {


// ============================================================================ FFT passes

template <typename R, int N, bool INV>
__global__ void __launch_bounds__(FFTThreads<N>::value, FFTMinBlocks<R, N>::value)
k_fft_xy(const typename CT<R>::type* src, typename CT<R>::type* dst, const typename CT<R>::type* __restrict__ twg) {
  using C = typename CT<R>::type;
  constexpr int NT = FFTThreads<N>::value;
  constexpr int RS = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;
  const size_t base = ((size_t)blockIdx.y * N + blockIdx.x) * (size_t)(N * N);
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  plane_load<N, NT, RS>(s, src + base);
  __syncthreads();
  fft_pass<C, N, NT, INV>(s, RS, 1, tw);  // along x (rows: y)
  fft_pass<C, N, NT, INV>(s, 1, RS, tw);  // along y (rows: x)
  plane_store<N, NT, RS>(dst + base, s);
}


// Per-axis multiplier tables for the z pass: the kinetic factor 1/2 |G + s|^2 scale is
// tx[x] + ty[y] + tz[z] with ta[i] = 1/2 (g_a f(i) + s_a)^2 scale (computed in FP64, stored in R).
template <typename R, int N, int MODE>
__device__ __forceinline__ void z_tables(R* tx, R* tz, R* ty, const ZParams& zp, int y, int k) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (MODE == Z_KIN) {
      const double qx = zp.gs[0] * freq<N>(i) + zp.shift[k][0];
      const double qz = zp.gs[2] * freq<N>(i) + zp.shift[k][2];
      tx[i] = (R)(0.5 * qx * qx * zp.scale);
      tz[i] = (R)(0.5 * qz * qz * zp.scale);
    } else {
      const double gx = zp.gs[0] * freq<N>(i), gz = zp.gs[2] * freq<N>(i);
      tx[i] = (R)(gx * gx);
      tz[i] = (R)(gz * gz);
    }
  }
  if (threadIdx.x == 0) {
    if (MODE == Z_KIN) {
      const double qy = zp.gs[1] * freq<N>(y) + zp.shift[k][1];
      *ty = (R)(0.5 * qy * qy * zp.scale);
    } else {
      const double gy = zp.gs[1] * freq<N>(y);
      *ty = (R)(gy * gy);
    }
  }
}

template <typename R, int N, int MODE>
__global__ void __launch_bounds__(FFTThreads<N>::value, FFTMinBlocks<R, N>::value)
k_fft_z(typename CT<R>::type* __restrict__ data, const typename CT<R>::type* __restrict__ twg, ZParams zp) {
  using C = typename CT<R>::type;
  constexpr int NT = FFTThreads<N>::value;
  // dense slab [z][x]: the z transforms run with x fastest across lanes, conflict-free at any pitch
  constexpr int RS = N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;
  R* tx = reinterpret_cast<R*>(s + N * RS);
  R* tz = tx + N;
  R* ty = tz + N;
  const int y = blockIdx.x;
  const int b = blockIdx.y;
  const size_t base = (size_t)b * N * N * N + (size_t)y * N;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  if (MODE != Z_INV_ONLY) z_tables<R, N, MODE>(tx, tz, ty, zp, y, (MODE == Z_KIN) ? b / zp.comps_per_k : 0);
  slab_load<N, NT, RS>(s, data + base, (size_t)N * N);
  __syncthreads();
  if (MODE != Z_INV_ONLY) {
    fft_pass<C, N, NT, false>(s, 1, RS, tw);  // along z (rows: x)
    const R tyv = *ty;
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int z = i / N, x = i - z * N;
      R m;
      if (MODE == Z_KIN) {
        m = tx[x] + tyv + tz[z];
      } else {
        const double g2 = (double)tx[x] + (double)tyv + (double)tz[z];
        m = (R)(g2 > 0.0 ? 4.0 * 3.14159265358979323846 / g2 * zp.scale : 0.0);
      }
      s[z * RS + x] = cscale(s[z * RS + x], m);
    }
    __syncthreads();
  }
  fft_pass<C, N, NT, true>(s, 1, RS, tw);
  slab_store<N, NT, RS>(data + base, s, (size_t)N * N);
}

// ---------------------------------------------------------------- two-factor passes (N = R1 R2)

// xy transform of one z-plane with one shared-memory exchange per axis: the x transform's A side
// reads global memory directly, the y transform's B side writes it directly (forward); the
// inverse runs the steps in the opposite order.  Column of the in-row exchange: K0 R1 + (n0 +
// K0) mod R1 (a rotation, so that the 8 lanes of a row hit distinct banks on both sides).
// Barriers: the y A side reads and writes the same rows of its item (n0 + R1 q = K0 R1 + n0)
// and runs in place without one; the x sides touch one row per item group, whose items sit on
// neighbouring lanes of a warp when their count divides 32, so a warp barrier orders them.
template <typename R, int N, bool INV>
__global__ void __launch_bounds__(FFTThreads<N>::value, FFTMinBlocks<R, N>::value)
k_fft_xy2(const typename CT<R>::type* src, typename CT<R>::type* dst, const typename CT<R>::type* __restrict__ twg) {
  using C = typename CT<R>::type;
  using T = TF<C, N, INV>;
  constexpr int NT = FFTThreads<N>::value;
  constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  constexpr int RS = TFPitch<N>::value;
  constexpr int IA = N * R1, IB = N * R2;                 // A / B items of one axis
  constexpr int PA = (IA + NT - 1) / NT, PB = (IB + NT - 1) / NT;
  constexpr bool ROW1 = (32 % R1 == 0) && (NT % R1 == 0);  // x A-side rows within a warp
  constexpr bool ROW2 = (32 % R2 == 0) && (NT % R2 == 0);  // x B-side rows within a warp
  constexpr bool ROW12 = ROW1 && R1 == R2;                 // and on the same lanes for both sides
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;
  const size_t base = ((size_t)blockIdx.y * N + blockIdx.x) * (size_t)(N * N);
  const C* g = src + base;
  C* o = dst + base;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  __syncthreads();
  C v[PA][R2];
  C u[PB][R1];
  if (!INV) {
    // x, A side: item (y, n0), n0 fastest
#pragma unroll
    for (int p = 0; p < PA; ++p) {
      const int i = threadIdx.x + p * NT;
      if (IA % NT == 0 || i < IA) {
        const int y = i / R1, n0 = i - y * R1;
#pragma unroll
        for (int q = 0; q < R2; ++q) v[p][q] = g[y * N + n0 + R1 * q];
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
    // y, A side in place: item (x, n0), x fastest; rows n0 + R1 q in, K0 R1 + n0 out (the same)
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
    // y, B side: item (x, K0) -> global
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
    // y, B side from global: item (x, K0)
#pragma unroll
    for (int p = 0; p < PB; ++p) {
      const int i = threadIdx.x + p * NT;
      if (IB % NT == 0 || i < IB) {
        const int k0 = i / N, x = i - k0 * N;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) u[p][k1] = g[(k0 + R2 * k1) * N + x];
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
    // x, A side -> global: item (y, n0)
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
}

// z transform + kinetic multiply + inverse z transform of one y-slab, one exchange each way:
// A side (x, n0) reads global memory along z, B side (x, K0) transforms, multiplies by
// tx[x] + ty + tz[kz] and transforms back in registers, A side writes global memory.
template <typename R, int N>
__global__ void __launch_bounds__(FFTThreads<N>::value, FFTMinBlocks<R, N>::value)
k_fft_z2_kin(typename CT<R>::type* __restrict__ data, const typename CT<R>::type* __restrict__ twg, ZParams zp) {
  using C = typename CT<R>::type;
  using TFW = TF<C, N, false>;
  using TIN = TF<C, N, true>;
  constexpr int NT = FFTThreads<N>::value;
  constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  constexpr int IA = N * R1, IB = N * R2;
  constexpr int PA = (IA + NT - 1) / NT, PB = (IB + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;                                  // [K0 R1 + n0][x], dense
  R* tx = reinterpret_cast<R*>(s + N * N);
  R* tz = tx + N;
  R* ty = tz + N;
  const int y = blockIdx.x;
  const int b = blockIdx.y;
  C* g = data + (size_t)b * N * N * N + (size_t)y * N;
  constexpr size_t ZS = (size_t)N * N;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  z_tables<R, N, Z_KIN>(tx, tz, ty, zp, y, b / zp.comps_per_k);
  C v[PA][R2];
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
#pragma unroll
      for (int q = 0; q < R2; ++q) v[p][q] = g[(size_t)(n0 + R1 * q) * ZS + x];
    }
  }
  __syncthreads();  // tables
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
      TFW::a_side(v[p], n0, tw);
#pragma unroll
      for (int k0 = 0; k0 < R2; ++k0) s[(k0 * R1 + n0) * N + x] = v[p][k0];
    }
  }
  __syncthreads();
  const R tyv = *ty;
#pragma unroll
  for (int p = 0; p < PB; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IB % NT == 0 || i < IB) {
      const int k0 = i / N, x = i - k0 * N;
      C u[R1];
#pragma unroll
      for (int n0 = 0; n0 < R1; ++n0) u[n0] = s[(k0 * R1 + n0) * N + x];
      TFW::b_side(u, k0, tw);
      const R txy = tx[x] + tyv;
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) u[k1] = cscale(u[k1], txy + tz[k0 + R2 * k1]);
      TIN::b_side(u, k0, tw);
#pragma unroll
      for (int n0 = 0; n0 < R1; ++n0) s[(k0 * R1 + n0) * N + x] = u[n0];
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
#pragma unroll
      for (int k0 = 0; k0 < R2; ++k0) v[p][k0] = s[(k0 * R1 + n0) * N + x];
      TIN::a_side(v[p], n0, tw);
#pragma unroll
      for (int n1 = 0; n1 < R2; ++n1) g[(size_t)(n0 + R1 * n1) * ZS + x] = v[p][n1];
    }
  }
}

template <typename R, int N>
static cudaError_t fft_xy_n(cudaStream_t st, const void* src, void* data, int nbatch, const void* tw, bool inv) {
  using C = typename CT<R>::type;
  dim3 grid(N, nbatch);
  if constexpr (TwoFactor<N>::ok) {
    const size_t smem2 = (size_t)(N + N * TFPitch<N>::value) * sizeof(C);
    auto kf = inv ? k_fft_xy2<R, N, true> : k_fft_xy2<R, N, false>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    kf<<<grid, FFTThreads<N>::value, smem2, st>>>((const C*)src, (C*)data, (const C*)tw);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)(N + N * (N + 1)) * sizeof(C);
  if (inv) {
    auto kf = k_fft_xy<R, N, true>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    kf<<<grid, FFTThreads<N>::value, smem, st>>>((const C*)src, (C*)data, (const C*)tw);
  } else {
    auto kf = k_fft_xy<R, N, false>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    kf<<<grid, FFTThreads<N>::value, smem, st>>>((const C*)src, (C*)data, (const C*)tw);
  }
  return cudaGetLastError();
}

template <typename R, int N, int MODE>
static cudaError_t fft_z_nm(cudaStream_t st, void* data, int nbatch, const void* tw, const ZParams& zp) {
  using C = typename CT<R>::type;
  const size_t smem = (size_t)(N + N * N) * sizeof(C) + (2 * N + 2) * sizeof(R);
  if constexpr (MODE == Z_KIN && TwoFactor<N>::ok) {
    auto kf = k_fft_z2_kin<R, N>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    kf<<<dim3(N, nbatch), FFTThreads<N>::value, smem, st>>>((C*)data, (const C*)tw, zp);
    return cudaGetLastError();
  }
  auto kf = k_fft_z<R, N, MODE>;
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  kf<<<dim3(N, nbatch), FFTThreads<N>::value, smem, st>>>((C*)data, (const C*)tw, zp);
  return cudaGetLastError();
}

template <typename R, int N>
static cudaError_t fft_z_n(cudaStream_t st, void* data, int nbatch, const void* tw, int mode, const ZParams& zp) {
  switch (mode) {
    case Z_KIN: return fft_z_nm<R, N, Z_KIN>(st, data, nbatch, tw, zp);
    case Z_POISSON: return fft_z_nm<R, N, Z_POISSON>(st, data, nbatch, tw, zp);
    default: return fft_z_nm<R, N, Z_INV_ONLY>(st, data, nbatch, tw, zp);
  }
}


template <typename R>
cudaError_t launch_fft_xy(cudaStream_t st, int N, const void* src, void* data, int nbatch, const void* tw, bool inv) {
  TDDFT_DISPATCH_N(N, (fft_xy_n<R, NN>(st, src, data, nbatch, tw, inv)));
}
template <typename R>
cudaError_t launch_fft_z(cudaStream_t st, int N, void* data, int nbatch, const void* tw, int mode, const ZParams& zp) {
  TDDFT_DISPATCH_N(N, (fft_z_n<R, NN>(st, data, nbatch, tw, mode, zp)));
}

// ============================================================================ projectors

// One CTA per (atom, spinor): c[p][sigma] = sum_e beta_p exp(+i s.d) psi_sigma(r_e) dV, then D c.
template <typename R> struct GatherMinBlocks { static constexpr int value = 1; };
template <> struct GatherMinBlocks<float> { static constexpr int value = 3; };

template <typename R, int NLM>
__global__ void __launch_bounds__(256, GatherMinBlocks<R>::value)
k_proj_gather(const typename CT<R>::type* __restrict__ psi, size_t N3, ProjTables<R> pt, R dV, EpiParams ep,
              typename CT<R>::type* __restrict__ c_out, typename CT<R>::type* __restrict__ dc_out) {
  using C = typename CT<R>::type;
  constexpr int NV = 4 * NLM;  // reals: (re, im) x (up, dn) x NLM
  const int a = blockIdx.x;
  const int kb = blockIdx.y;
  const int k = kb / ep.nstates;
  const R sx = (R)ep.shift[k][0], sy = (R)ep.shift[k][1], sz = (R)ep.shift[k][2];
  const C* up = psi + (size_t)(2 * kb) * N3;
  const C* dn = up + N3;
  R acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = (R)0;
  const int e0 = pt.g_ptr[a], e1 = pt.g_ptr[a + 1];
  R nl[4];
  load_row<R, 4>(pt.nrm + (size_t)a * 4, nl);
  // Software pipeline over this thread's entries e, e + 256, ...: the grid index of the entry
  // after next, and the table row and psi values of the next entry, are requested before the
  // current entry is processed, so two dependent load chains are in flight at a time.
  const C zc = cmake<C>((R)0, (R)0);
  int e = e0 + threadIdx.x;
  int r1 = (e + 256 < e1) ? pt.g_idx[e + 256] : 0;  // index of the next entry
  R tc[4] = {(R)0, (R)0, (R)0, (R)0};
  C uc = zc, dc = zc;
  if (e < e1) {
    const int r0 = pt.g_idx[e];
    load_row<R, 4>(pt.g_row + (size_t)e * 4, tc);
    uc = up[r0];
    dc = dn[r0];
  }
  for (; e < e1; e += 256) {
    R tn[4] = {(R)0, (R)0, (R)0, (R)0};
    C un = zc, dn_ = zc;
    int r2 = 0;
    if (e + 256 < e1) {
      load_row<R, 4>(pt.g_row + (size_t)(e + 256) * 4, tn);
      un = up[r1];
      dn_ = dn[r1];
      if (e + 512 < e1) r2 = pt.g_idx[e + 512];
    }
    R t[4] = {tc[0], tc[1], tc[2], tc[3]}, bt[NLM];
    beta_values<R, NLM>(t[0], t[1], t[2], t[3], nl, pt.yc, bt);
    R sn, cs;
    sincos_r<R>(sx * t[0] + sy * t[1] + sz * t[2], &sn, &cs);
    const C u = uc, d = dc;
    for (int i = 0; i < 4; ++i) tc[i] = tn[i];
    uc = un;
    dc = dn_;
    r1 = r2;
    const R pux = u.x * cs - u.y * sn, puy = u.x * sn + u.y * cs;  // u exp(+i arg)
    const R pdx = d.x * cs - d.y * sn, pdy = d.x * sn + d.y * cs;
#pragma unroll
    for (int p = 0; p < NLM; ++p) {
      const R bp = bt[p];
      acc[4 * p + 0] += bp * pux;
      acc[4 * p + 1] += bp * puy;
      acc[4 * p + 2] += bp * pdx;
      acc[4 * p + 3] += bp * pdy;
    }
  }
  __shared__ R red[8][NV];
  __shared__ C cv[2 * NLM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const R v = warp_sum(acc[i]);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * NLM) {
    R re = 0, im = 0;
    for (int w = 0; w < 8; ++w) {
      re += red[w][2 * threadIdx.x];
      im += red[w][2 * threadIdx.x + 1];
    }
    C c = cmake<C>(re * dV, im * dV);
    cv[threadIdx.x] = c;
    c_out[((size_t)kb * pt.natoms + a) * 2 * NLM + threadIdx.x] = c;
  }
  __syncthreads();
  if (threadIdx.x < 2 * NLM) {
    const R* D = pt.Dmat + ((size_t)a * 2 * NLM + threadIdx.x) * 2 * NLM * 2;
    R re = 0, im = 0;
    for (int u = 0; u < 2 * NLM; ++u) {
      const R dr = D[2 * u], di = D[2 * u + 1];
      re += dr * cv[u].x - di * cv[u].y;
      im += dr * cv[u].y + di * cv[u].x;
    }
    dc_out[((size_t)kb * pt.natoms + a) * 2 * NLM + threadIdx.x] = cmake<C>(re, im);
  }
}

template <typename R>
cudaError_t launch_proj_gather(cudaStream_t st, int N, const void* psi, int nkb, const ProjTables<R>& pt,
                               double dV, const EpiParams& ep, void* c_out, void* dc_out) {
  using C = typename CT<R>::type;
  if (pt.natoms == 0) return cudaSuccess;
  dim3 grid(pt.natoms, nkb);
  const size_t N3 = (size_t)N * N * N;
  switch (pt.nlm) {
    case 1: k_proj_gather<R, 1><<<grid, 256, 0, st>>>((const C*)psi, N3, pt, (R)dV, ep, (C*)c_out, (C*)dc_out); break;
    case 4: k_proj_gather<R, 4><<<grid, 256, 0, st>>>((const C*)psi, N3, pt, (R)dV, ep, (C*)c_out, (C*)dc_out); break;
    case 9: k_proj_gather<R, 9><<<grid, 256, 0, st>>>((const C*)psi, N3, pt, (R)dV, ep, (C*)c_out, (C*)dc_out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


// ============================================================================ density

// Band group g = blockIdx.y sums bands [kb0, kb1) for two neighbouring points per thread and
// writes its partial 4-vector; with one group it writes rho directly.  The groups are then
// added in a fixed order (deterministic result).
template <typename R>
__global__ void __launch_bounds__(256)
k_density(const typename CT<R>::type* __restrict__ psi, size_t N3, int nkb, int ngroups,
          const double* __restrict__ wf, double* __restrict__ out) {
  const size_t r = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (r >= N3) return;
  const int g = blockIdx.y;
  const int kb0 = (int)(((long long)nkb * g) / ngroups), kb1 = (int)(((long long)nkb * (g + 1)) / ngroups);
  double s[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  // FP32 spinors: bilinears of up to 8 bands are summed in FP32 (the inputs' own precision) and
  // each such partial sum is added to the FP64 accumulators; FP64 spinors: FP64 throughout
  constexpr int CH = sizeof(R) == 4 ? 8 : 1;
  for (int kc = kb0; kc < kb1; kc += CH) {
    R p[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const int kend = min(kb1, kc + CH);
#pragma unroll 1
    for (int kb = kc; kb < kend; ++kb) {
      const Pair<typename CT<R>::type> u = ld2(psi + (size_t)(2 * kb) * N3 + r);
      const Pair<typename CT<R>::type> d = ld2(psi + (size_t)(2 * kb + 1) * N3 + r);
      const R w = (R)wf[kb];
      const R ux[2] = {u.a.x, u.b.x}, uy[2] = {u.a.y, u.b.y};
      const R dx[2] = {d.a.x, d.b.x}, dy[2] = {d.a.y, d.b.y};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        p[j][0] += w * (ux[j] * ux[j] + uy[j] * uy[j]);
        p[j][1] += w * (dx[j] * dx[j] + dy[j] * dy[j]);
        p[j][2] += w * (ux[j] * dx[j] + uy[j] * dy[j]);  // Re(u conj d)
        p[j][3] += w * (uy[j] * dx[j] - ux[j] * dy[j]);  // Im(u conj d)
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) s[j][c] += (double)p[j][c];
  }
  double* o = out + (size_t)g * 4 * N3;
#pragma unroll
  for (int c = 0; c < 4; ++c) *reinterpret_cast<double2*>(o + c * N3 + r) = make_double2(s[0][c], s[1][c]);
}

__global__ void k_density_reduce(size_t n, int ngroups, const double* __restrict__ part, double* __restrict__ rho) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int g = 0; g < ngroups; ++g) t += part[(size_t)g * n + i];
  rho[i] = t;
}

int density_groups(size_t N3, int nkb) {
  // enough resident threads to hide the load latency: about 6e5 threads
  const size_t per = N3 / 2;
  int g = (int)((600000 + per - 1) / per);
  if (g > nkb) g = nkb;
  if (g > 16) g = 16;
  return g < 1 ? 1 : g;
}

template <typename R>
cudaError_t launch_density(cudaStream_t st, size_t N3, const void* psi, int nkb, const double* wf, double* rho,
                           double* part) {
  const int G = part ? density_groups(N3, nkb) : 1;
  const size_t nthreads = N3 / 2;
  dim3 grid((unsigned)((nthreads + 255) / 256), G);
  k_density<R><<<grid, 256, 0, st>>>((const typename CT<R>::type*)psi, N3, nkb, G, wf, G == 1 ? rho : part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || G == 1) return e;
  k_density_reduce<<<(unsigned)((4 * N3 + 255) / 256), 256, 0, st>>>(4 * N3, G, part, rho);
  return cudaGetLastError();
}

// ============================================================================ XC and potential

// PW92 interpolation G(rs) and dG/drs for one parameter row (A, a1, b1, b2, b3, b4), p = 1;
// sr = sqrt(rs) and isr = 1 / sr are shared by the three rows.
__device__ __forceinline__ void pw92_g(double rs, double sr, double isr, double A, double a1, double b1, double b2,
                                       double b3, double b4, double* g, double* dg) {
  const double q0 = -2.0 * A * (1.0 + a1 * rs);
  const double q1 = 2.0 * A * sr * (b1 + sr * (b2 + sr * (b3 + sr * b4)));
  const double q1p = A * (b1 * isr + 2.0 * b2 + 3.0 * b3 * sr + 4.0 * b4 * rs);
  const double iq1 = 1.0 / q1;
  const double lg = log1p(iq1);
  *g = q0 * lg;
  *dg = -2.0 * A * a1 * lg - q0 * q1p * iq1 / (q1 + 1.0);
}

// Slater exchange with spin scaling plus PW92 correlation on (nu, nd): energy density, v_up, v_dn.
// Three cube roots per point: with c = n^(1/3), rs = (3 / 4 pi)^(1/3) / c and
// (1 +- zeta)^(1/3) = 2^(1/3) n_up,dn^(1/3) / c (nu, nd >= 0, so |zeta| <= 1).
__device__ void lsda_point(double nu, double nd, double* e, double* vu, double* vd) {
  const double c6 = 1.240700981798800033;    // (6 / pi)^(1/3)
  const double crs = 0.6203504908994000167;  // (3 / (4 pi))^(1/3)
  const double c2 = 1.259921049894873165;    // 2^(1/3)
  const double fden = 1.923661050931536320;  // 1 / (2^(4/3) - 2)
  const double cbu = cbrt(nu), cbd = cbrt(nd);
  const double ex = -0.75 * c6 * (nu * cbu + nd * cbd);
  const double vxu = -c6 * cbu, vxd = -c6 * cbd;
  const double n = nu + nd;
  const double icn = 1.0 / cbrt(n);
  const double rs = crs * icn;
  double z = (nu - nd) / n;
  z = fmin(1.0, fmax(-1.0, z));
  const double sr = sqrt(rs), isr = 1.0 / sr;
  double ec0, d0, ec1, d1, mac, dmac;
  pw92_g(rs, sr, isr, 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294, &ec0, &d0);
  pw92_g(rs, sr, isr, 0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517, &ec1, &d1);
  pw92_g(rs, sr, isr, 0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671, &mac, &dmac);
  const double ac = -mac, dac = -dmac;
  const double opz = 1.0 + z, omz = 1.0 - z;
  const double cpz = c2 * cbu * icn, cmz = c2 * cbd * icn;
  const double f = (opz * cpz + omz * cmz - 2.0) * fden;
  const double fp = (4.0 / 3.0) * (cpz - cmz) * fden;
  const double fpp0 = 1.709921;
  const double z3 = z * z * z, z4 = z3 * z;
  const double ec = ec0 + ac * f * (1.0 - z4) / fpp0 + (ec1 - ec0) * f * z4;
  const double drs = d0 + dac * f * (1.0 - z4) / fpp0 + (d1 - d0) * f * z4;
  const double dz = ac / fpp0 * (fp * (1.0 - z4) - 4.0 * z3 * f) + (ec1 - ec0) * (fp * z4 + 4.0 * z3 * f);
  const double common = ec - rs / 3.0 * drs;
  *e = ex + n * ec;
  *vu = vxu + common - (z - 1.0) * dz;
  *vd = vxd + common - (z + 1.0) * dz;
}

__global__ void k_potential(size_t N3, const double* __restrict__ rho, const double* __restrict__ vH,
                            const double* __restrict__ vloc, double Bx, double By, double Bz, int xc, int mode,
                            double* __restrict__ V, float* __restrict__ Vf, double* __restrict__ exc,
                            double* __restrict__ vxc4) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
  const double n = r0 + r1, mx = 2.0 * r2, my = -2.0 * r3, mz = r0 - r1;
  double e = 0.0, vbar = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
  if (xc && n >= 1e-14 && mode == TDDFT_SPIN_COLLINEAR) {
    // Eq. HSDFT: LSDA on the channel densities, field along the quantisation axis
    double vu, vd;
    lsda_point(r0, r1, &e, &vu, &vd);
    vbar = 0.5 * (vu + vd);
    bz = 0.5 * (vu - vd);
  } else if (xc && n >= 1e-14 && mode == TDDFT_SPIN_UNPOLARISED) {
    double vu, vd;
    lsda_point(0.5 * n, 0.5 * n, &e, &vu, &vd);
    vbar = vu;
  } else if (xc && n >= 1e-14) {
    const double mag = sqrt(mx * mx + my * my + mz * mz);
    const double s = fmin(mag, n);
    double vu, vd;
    lsda_point(0.5 * (n + s), 0.5 * (n - s), &e, &vu, &vd);
    vbar = 0.5 * (vu + vd);
    if (mag > 1e-14) {
      const double bm = 0.5 * (vu - vd) / mag;
      bx = bm * mx; by = bm * my; bz = bm * mz;
    }
  }
  const double v = vloc[r] + vH[r] + vbar;
  const double tx = bx + 0.5 * Bx, ty = by + 0.5 * By, tz = bz + 0.5 * Bz;  // mu_B = 1/2
  const double V0 = v + tz, V1 = v - tz, V2 = 2.0 * tx, V3 = -2.0 * ty;
  V[r] = V0; V[N3 + r] = V1; V[2 * N3 + r] = V2; V[3 * N3 + r] = V3;
  if (Vf) {
    Vf[r] = (float)V0; Vf[N3 + r] = (float)V1; Vf[2 * N3 + r] = (float)V2; Vf[3 * N3 + r] = (float)V3;
  }
  exc[r] = e;
  vxc4[r] = vbar + bz; vxc4[N3 + r] = vbar - bz; vxc4[2 * N3 + r] = 2.0 * bx; vxc4[3 * N3 + r] = -2.0 * by;
}

cudaError_t launch_potential(cudaStream_t st, size_t N3, const double* rho, const double* vH, const double* vloc,
                             const double* B, int xc, int mode, double* V, float* Vf, double* exc, double* vxc4) {
  k_potential<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, rho, vH, vloc, B[0], B[1], B[2], xc, mode, V, Vf, exc,
                                                            vxc4);
  return cudaGetLastError();
}

// (rho_uu + rho_dd, 0): the total density as a complex field for the Poisson solve.
__global__ void k_density_to_complex(size_t n, const double* rho, double2* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(rho[i] + rho[n + i], 0.0);
}
cudaError_t launch_density_to_complex(cudaStream_t st, size_t N3, const double* rho, double2* out) {
  k_density_to_complex<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, rho, out);
  return cudaGetLastError();
}
__global__ void k_complex_real_part(size_t n, const double2* in, double* out, double scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i].x * scale;
}
cudaError_t launch_complex_real_part(cudaStream_t st, size_t N3, const double2* in, double* out, double scale) {
  k_complex_real_part<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, in, out, scale);
  return cudaGetLastError();
}

// V_loc(G) = sum_a [-4 pi Z / G^2 exp(-G^2 rc^2 / 4) exp(-i G.R_a)] / Omega, G = 0: sum_a pi Z rc^2 / Omega.
__global__ void k_vloc_G(int N, double gx0, double gy0, double gz0, int natoms, const double* __restrict__ pos,
                         const double* __restrict__ Zr, double omega, double2* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N3 = (size_t)N * N * N;
  if (i >= N3) return;
  const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
  auto fq = [N](int j) { return j < N / 2 ? j : j - N; };
  const double gx = gx0 * fq(x), gy = gy0 * fq(y), gz = gz0 * fq(z);
  const double g2 = gx * gx + gy * gy + gz * gz;
  const double kPi = 3.14159265358979323846;
  double re = 0.0, im = 0.0;
  for (int a = 0; a < natoms; ++a) {
    const double Z = Zr[2 * a], rc = Zr[2 * a + 1];
    const double t = g2 > 0.0 ? -4.0 * kPi * Z / g2 * exp(-g2 * rc * rc * 0.25) : kPi * Z * rc * rc;
    double sn, cs;
    sincos(gx * pos[3 * a] + gy * pos[3 * a + 1] + gz * pos[3 * a + 2], &sn, &cs);
    re += t * cs;
    im -= t * sn;
  }
  out[i] = make_double2(re / omega, im / omega);
}
cudaError_t launch_vloc_G(cudaStream_t st, int N, const double* L, int natoms, const double* pos, const double* Zr,
                          double omega, double2* out) {
  const size_t N3 = (size_t)N * N * N;
  const double kPi = 3.14159265358979323846;
  k_vloc_G<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N, 2 * kPi / L[0], 2 * kPi / L[1], 2 * kPi / L[2], natoms,
                                                         pos, Zr, omega, out);
  return cudaGetLastError();
}

// ============================================================================ conversions

// Precision conversion of spinor arrays.  The source or destination may be page-locked host
// memory read or written through its mapped address (over the CPU-GPU link), where the rate
// depends on the requests in flight: each warp moves 8 x 32 consecutive elements, eight
// independent 16-byte loads per thread, every load instruction covering 512 contiguous bytes.
constexpr int kConvPerThread = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_convert_in(size_t n, const double2* __restrict__ in, typename CT<R>::type* __restrict__ out) {
  using C = typename CT<R>::type;
  const size_t base = (((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 * kConvPerThread) + (threadIdx.x & 31);
  double2 v[kConvPerThread];
#pragma unroll
  for (int q = 0; q < kConvPerThread; ++q) {
    const size_t i = base + 32 * q;
    if (i < n) v[q] = in[i];
  }
#pragma unroll
  for (int q = 0; q < kConvPerThread; ++q) {
    const size_t i = base + 32 * q;
    if (i < n) out[i] = cmake<C>((R)v[q].x, (R)v[q].y);
  }
}
template <typename R>
__global__ void __launch_bounds__(256) k_convert_out(size_t n, const typename CT<R>::type* __restrict__ in, double2* __restrict__ out) {
  using C = typename CT<R>::type;
  const size_t base = (((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 * kConvPerThread) + (threadIdx.x & 31);
  C v[kConvPerThread];
#pragma unroll
  for (int q = 0; q < kConvPerThread; ++q) {
    const size_t i = base + 32 * q;
    if (i < n) v[q] = in[i];
  }
#pragma unroll
  for (int q = 0; q < kConvPerThread; ++q) {
    const size_t i = base + 32 * q;
    if (i < n) out[i] = make_double2((double)v[q].x, (double)v[q].y);
  }
}
template <typename R>
cudaError_t launch_convert_in(cudaStream_t st, size_t n, const double2* in, void* out) {
  if (n == 0) return cudaSuccess;
  const size_t per_cta = 256 * kConvPerThread;
  k_convert_in<R><<<(unsigned)((n + per_cta - 1) / per_cta), 256, 0, st>>>(n, in, (typename CT<R>::type*)out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_convert_out(cudaStream_t st, size_t n, const void* in, double2* out) {
  if (n == 0) return cudaSuccess;
  const size_t per_cta = 256 * kConvPerThread;
  k_convert_out<R><<<(unsigned)((n + per_cta - 1) / per_cta), 256, 0, st>>>(n, (const typename CT<R>::type*)in, out);
  return cudaGetLastError();
}

// ============================================================================ reductions (fixed order)

template <int NT>
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += sh[w];
  return t;  // valid in thread 0
}

// out2[band] = sum over npts of conj(a) b (complex, double accumulation) in two passes: CTA
// (chunk, band) sums a fixed range of points, then one thread per band adds the chunks in
// order (deterministic, and every SM busy).
constexpr int kDotChunks = 64;
template <typename R>
__global__ void __launch_bounds__(256) k_band_dot_part(size_t npts, const typename CT<R>::type* __restrict__ a,
                                                       const typename CT<R>::type* __restrict__ b, double* part) {
  __shared__ double sh[8];
  const size_t off = (size_t)blockIdx.y * npts;
  const size_t len = (npts + kDotChunks - 1) / kDotChunks;
  const size_t lo = (size_t)blockIdx.x * len, hi = lo + len < npts ? lo + len : npts;
  // groups of kDotGroup products are summed in R before entering the FP64 sum (FP64 arithmetic
  // is scarce on this part; in FP64 mode R is double and nothing changes)
  constexpr int kDotGroup = 8;
  double re = 0.0, im = 0.0;
  for (size_t i0 = lo + threadIdx.x; i0 < hi; i0 += (size_t)256 * kDotGroup) {
    R gr = (R)0, gi = (R)0;
#pragma unroll
    for (int j = 0; j < kDotGroup; ++j) {
      const size_t i = i0 + (size_t)j * 256;
      if (i < hi) {
        const auto x = a[off + i], y = b[off + i];
        gr += x.x * y.x + x.y * y.y;
        gi += x.x * y.y - x.y * y.x;
      }
    }
    re += (double)gr;
    im += (double)gi;
  }
  const double tr = block_sum<256>(re, sh);
  const double ti = block_sum<256>(im, sh);
  if (threadIdx.x == 0) {
    const size_t o = ((size_t)blockIdx.y * kDotChunks + blockIdx.x) * 2;
    part[o] = tr;
    part[o + 1] = ti;
  }
}
__global__ void k_band_dot_sum(int nbands, const double* __restrict__ part, double* out2) {
  const int band = blockIdx.x * blockDim.x + threadIdx.x;
  if (band >= nbands) return;
  double re = 0.0, im = 0.0;
  for (int ch = 0; ch < kDotChunks; ++ch) {
    re += part[((size_t)band * kDotChunks + ch) * 2];
    im += part[((size_t)band * kDotChunks + ch) * 2 + 1];
  }
  out2[2 * band] = re;
  out2[2 * band + 1] = im;
}
template <typename R>
cudaError_t launch_band_dot(cudaStream_t st, size_t npts, int nbands, const void* a, const void* b, double* out2,
                            double* part) {
  using C = typename CT<R>::type;
  k_band_dot_part<R><<<dim3(kDotChunks, nbands), 256, 0, st>>>(npts, (const C*)a, (const C*)b, part);
  k_band_dot_sum<<<(nbands + 127) / 128, 128, 0, st>>>(nbands, part, out2);
  return cudaGetLastError();
}
size_t band_dot_part_doubles(int nbands) { return (size_t)nbands * kDotChunks * 2; }

// out[kb] = Re sum conj(c) dc over atoms, projectors and spins.
template <typename R>
__global__ void k_nl_energy(int ncoef, const typename CT<R>::type* __restrict__ c,
                            const typename CT<R>::type* __restrict__ dc, double* out) {
  __shared__ double sh[8];
  const size_t off = (size_t)blockIdx.x * ncoef;
  double s = 0.0;
  for (int i = threadIdx.x; i < ncoef; i += 256) s += (double)c[off + i].x * dc[off + i].x + (double)c[off + i].y * dc[off + i].y;
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}
template <typename R>
cudaError_t launch_nl_energy(cudaStream_t st, int nkb, int ncoef, const void* c, const void* dc, double* out) {
  using C = typename CT<R>::type;
  k_nl_energy<R><<<nkb, 256, 0, st>>>(ncoef, (const C*)c, (const C*)dc, out);
  return cudaGetLastError();
}

// Spin-orbit torque of one spinor (block kb): sum over atoms and components i of
// Re c^dagger T^i c, the rows (atom, i, r) spread over the threads, fixed-order block sums.
template <typename R>
__global__ void __launch_bounds__(256)
k_soc_torque(int natoms, int M, const typename CT<R>::type* __restrict__ c, const double2* __restrict__ T,
             double* out) {
  __shared__ double sh[8];
  const typename CT<R>::type* ck = c + (size_t)blockIdx.x * natoms * M;
  double acc[3] = {0.0, 0.0, 0.0};
  const int rows = natoms * M;
  for (int i = 0; i < 3; ++i) {
    for (int t = threadIdx.x; t < rows; t += 256) {
      const int a = t / M, r = t - a * M;
      const double2* Tr = T + (((size_t)a * 3 + i) * M + r) * M;
      const typename CT<R>::type* ca = ck + (size_t)a * M;
      double re = 0.0, im = 0.0;  // (T c)_r
      for (int q = 0; q < M; ++q) {
        const double cr = (double)ca[q].x, ci = (double)ca[q].y;
        re += Tr[q].x * cr - Tr[q].y * ci;
        im += Tr[q].x * ci + Tr[q].y * cr;
      }
      acc[i] += (double)ca[r].x * re + (double)ca[r].y * im;  // Re conj(c_r) (T c)_r
    }
  }
  for (int i = 0; i < 3; ++i) {
    const double v = block_sum<256>(acc[i], sh);
    if (threadIdx.x == 0) out[(size_t)blockIdx.x * 3 + i] = v;
  }
}
template <typename R>
cudaError_t launch_soc_torque(cudaStream_t st, int nkb, int natoms, int M, const void* c, const double2* T,
                              double* out) {
  k_soc_torque<R><<<nkb, 256, 0, st>>>(natoms, M, (const typename CT<R>::type*)c, T, out);
  return cudaGetLastError();
}

// int b_xc x m and int m (without dV) from rho_v and the XC 4-vector [vbar + b_z, vbar - b_z,
// 2 b_x, -2 b_y]; one block, fixed order.
__global__ void __launch_bounds__(1024)
k_xc_torque(size_t N3, const double* __restrict__ rho, const double* __restrict__ vxc4, double* out) {
  __shared__ double sh[32];
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (size_t r = threadIdx.x; r < N3; r += 1024) {
    const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
    const double mx = 2.0 * r2, my = -2.0 * r3, mz = r0 - r1;
    const double bz = 0.5 * (vxc4[r] - vxc4[N3 + r]), bx = 0.5 * vxc4[2 * N3 + r], by = -0.5 * vxc4[3 * N3 + r];
    acc[0] += by * mz - bz * my;
    acc[1] += bz * mx - bx * mz;
    acc[2] += bx * my - by * mx;
    acc[3] += mx; acc[4] += my; acc[5] += mz;
  }
  for (int i = 0; i < 6; ++i) {
    const double t = block_sum<1024>(acc[i], sh);
    if (threadIdx.x == 0) out[i] = t;
  }
}
cudaError_t launch_xc_torque(cudaStream_t st, size_t N3, const double* rho, const double* vxc4, double* out6) {
  k_xc_torque<<<1, 1024, 0, st>>>(N3, rho, vxc4, out6);
  return cudaGetLastError();
}

// Field integrals (without dV): [0] v_loc n, [1] v_H n, [2] e_xc, [3..5] m, [6] n, [7] B.m,
// [8] <rho_v, V_v^xc>, [9] count of non-finite rho values.  Two passes: each of kFieldBlocks
// CTAs sums a fixed range of points, then one CTA adds the block partials in order.
constexpr int kFieldBlocks = 304;
__global__ void __launch_bounds__(256)
k_field_sums_part(size_t N3, const double* __restrict__ rho, const double* __restrict__ vloc, const double* __restrict__ vH,
                  const double* __restrict__ exc, const double* __restrict__ vxc4, double Bx, double By, double Bz,
                  double* part) {
  __shared__ double sh[8];
  double acc[10];
  for (int i = 0; i < 10; ++i) acc[i] = 0.0;
  const size_t len = (N3 + kFieldBlocks - 1) / kFieldBlocks;
  const size_t lo = (size_t)blockIdx.x * len, hi = lo + len < N3 ? lo + len : N3;
  for (size_t r = lo + threadIdx.x; r < hi; r += 256) {
    const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
    const double n = r0 + r1, mx = 2.0 * r2, my = -2.0 * r3, mz = r0 - r1;
    acc[0] += vloc[r] * n;
    acc[1] += vH[r] * n;
    acc[2] += exc[r];
    acc[3] += mx; acc[4] += my; acc[5] += mz;
    acc[6] += n;
    acc[7] += Bx * mx + By * my + Bz * mz;
    acc[8] += r0 * vxc4[r] + r1 * vxc4[N3 + r] + r2 * vxc4[2 * N3 + r] + r3 * vxc4[3 * N3 + r];
    acc[9] += (isfinite(r0) && isfinite(r1) && isfinite(r2) && isfinite(r3)) ? 0.0 : 1.0;
  }
  for (int i = 0; i < 10; ++i) {
    const double t = block_sum<256>(acc[i], sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 10 + i] = t;
  }
}
__global__ void k_field_sums_total(const double* __restrict__ part, double* out) {
  const int i = threadIdx.x;
  if (i >= 10) return;
  double s = 0.0;
  for (int b = 0; b < kFieldBlocks; ++b) s += part[(size_t)b * 10 + i];
  out[i] = s;
}
cudaError_t launch_field_sums(cudaStream_t st, size_t N3, const double* rho, const double* vloc, const double* vH,
                              const double* exc, const double* vxc4, const double* /*V*/, const double* B, double* out,
                              double* part) {
  k_field_sums_part<<<kFieldBlocks, 256, 0, st>>>(N3, rho, vloc, vH, exc, vxc4, B[0], B[1], B[2], part);
  k_field_sums_total<<<1, 32, 0, st>>>(part, out);
  return cudaGetLastError();
}
size_t field_sums_part_doubles() { return (size_t)kFieldBlocks * 10; }

__global__ void __launch_bounds__(1024) k_max_abs_diff(size_t n, const double* a, const double* b, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (size_t i = threadIdx.x; i < n; i += 1024) m = fmax(m, fabs(a[i] - b[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t = fmax(t, sh[w]);
    *out = t;
  }
}
cudaError_t launch_max_abs_diff(cudaStream_t st, size_t n, const double* a, const double* b, double* out) {
  k_max_abs_diff<<<1, 1024, 0, st>>>(n, a, b, out);
  return cudaGetLastError();
}

// Sets *flag when the local potential leaves [lo, hi] given the kinetic maximum and projector bound.
__global__ void k_check_window(size_t N3, const double* __restrict__ V, double lo, double hi, double kin_max,
                               double nl_bound, int* flag) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  const double v = 0.5 * (V[r] + V[N3 + r]);
  const double bz = 0.5 * (V[r] - V[N3 + r]), bx = 0.5 * V[2 * N3 + r], by = 0.5 * V[3 * N3 + r];
  const double b = sqrt(bx * bx + by * by + bz * bz);
  const bool bad = !(v - b - nl_bound >= lo) || !(v + b + nl_bound + kin_max <= hi);
  if (bad) atomicOr(flag, 1);
}
cudaError_t launch_check_window(cudaStream_t st, size_t N3, const double* V, double lo, double hi, double kin_max,
                                double nl_bound, int* flag) {
  k_check_window<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, V, lo, hi, kin_max, nl_bound, flag);
  return cudaGetLastError();
}

// n = rho_uu + rho_dd and m = (2 Re rho_ud, -2 Im rho_ud, rho_uu - rho_dd) from rho_v, into
// nm[0 .. N3) (n) and nm[N3 .. 4 N3) (m_x, m_y, m_z).
__global__ void k_nm_from_rho(size_t N3, const double* __restrict__ rho, double* __restrict__ nm) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
  nm[r] = r0 + r1;
  nm[N3 + r] = 2.0 * r2;
  nm[2 * N3 + r] = -2.0 * r3;
  nm[3 * N3 + r] = r0 - r1;
}
cudaError_t launch_nm_from_rho(cudaStream_t st, size_t N3, const double* rho, double* nm) {
  k_nm_from_rho<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, rho, nm);
  return cudaGetLastError();
}

// Extrema of the local potential for the automatic spectral window: min and max of
// v = (V_0 + V_1)/2 and max of |b| = |(V_2, V_3, V_0 - V_1)|/2 over the grid.  Products and sums
// are rounded one by one (no fused multiply-add), as in a plain IEEE evaluation; min and max do
// not depend on the order, so the result is exact.  Partials per block, then one block.
__global__ void __launch_bounds__(256) k_window_part(size_t N3, const double* __restrict__ V, double* part) {
  __shared__ double sh[3][8];
  double vmin = 1e300, vmax = -1e300, bmax = 0.0;
  for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < N3; r += (size_t)gridDim.x * blockDim.x) {
    const double v = __dmul_rn(0.5, __dadd_rn(V[r], V[N3 + r]));
    const double bz = __dmul_rn(0.5, __dsub_rn(V[r], V[N3 + r]));
    const double bx = __dmul_rn(0.5, V[2 * N3 + r]), by = __dmul_rn(0.5, V[3 * N3 + r]);
    const double b = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz)));
    vmin = fmin(vmin, v);
    vmax = fmax(vmax, v);
    bmax = fmax(bmax, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[0][warp] = vmin; sh[1][warp] = vmax; sh[2][warp] = bmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      vmin = fmin(vmin, sh[0][w]);
      vmax = fmax(vmax, sh[1][w]);
      bmax = fmax(bmax, sh[2][w]);
    }
    part[3 * blockIdx.x] = vmin;
    part[3 * blockIdx.x + 1] = vmax;
    part[3 * blockIdx.x + 2] = bmax;
  }
}
__global__ void k_window_total(int nparts, const double* __restrict__ part, double* out) {
  if (threadIdx.x != 0) return;
  double vmin = 1e300, vmax = -1e300, bmax = 0.0;
  for (int i = 0; i < nparts; ++i) {
    vmin = fmin(vmin, part[3 * i]);
    vmax = fmax(vmax, part[3 * i + 1]);
    bmax = fmax(bmax, part[3 * i + 2]);
  }
  out[0] = vmin;
  out[1] = vmax;
  out[2] = bmax;
}
cudaError_t launch_window_extrema(cudaStream_t st, size_t N3, const double* V, double* part, double* out3) {
  k_window_part<<<kFieldBlocks, 256, 0, st>>>(N3, V, part);
  k_window_total<<<1, 32, 0, st>>>(kFieldBlocks, part, out3);
  return cudaGetLastError();
}

// ============================================================================ per-atom moments
// Nearest atom of every grid point (minimum image), Algorithm 1's NearestAtom rule; equal
// distances go to the lowest atom index.  Every operation is explicitly rounded (no fused
// multiply-add) so that ties resolve the same way as in a plain IEEE evaluation of
// d = x h - R, d -= L rint(d / L), |d|^2 = (dx^2 + dy^2) + dz^2.
__global__ void k_voronoi_owner(int N, double hx, double hy, double hz, double Lx, double Ly, double Lz, int natoms,
                                const double* __restrict__ pos, int* __restrict__ owner) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N3 = (size_t)N * N * N;
  if (i >= N3) return;
  const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
  const double rx = __dmul_rn((double)x, hx), ry = __dmul_rn((double)y, hy), rz = __dmul_rn((double)z, hz);
  double best = 1e300;
  int own = 0;
  for (int a = 0; a < natoms; ++a) {
    double dx = __dsub_rn(rx, pos[3 * a]), dy = __dsub_rn(ry, pos[3 * a + 1]), dz = __dsub_rn(rz, pos[3 * a + 2]);
    dx = __dsub_rn(dx, __dmul_rn(Lx, rint(__ddiv_rn(dx, Lx))));
    dy = __dsub_rn(dy, __dmul_rn(Ly, rint(__ddiv_rn(dy, Ly))));
    dz = __dsub_rn(dz, __dmul_rn(Lz, rint(__ddiv_rn(dz, Lz))));
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < best) {
      best = d2;
      own = a;
    }
  }
  owner[i] = own;
}
cudaError_t launch_voronoi_owner(cudaStream_t st, int N, const double* L, int natoms, const double* pos, int* owner) {
  const size_t N3 = (size_t)N * N * N;
  k_voronoi_owner<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N, L[0] / N, L[1] / N, L[2] / N, L[0], L[1], L[2],
                                                               natoms, pos, owner);
  return cudaGetLastError();
}

// out[a] = {sum m_x, sum m_y, sum m_z, sum n} over the points owned by atom a (one CTA per atom,
// fixed order; multiply by dV on the host).
__global__ void __launch_bounds__(256) k_atom_sums(size_t N3, const double* __restrict__ rho,
                                                   const int* __restrict__ owner, double* __restrict__ out) {
  __shared__ double sh[8];
  const int a = blockIdx.x;
  double acc[4] = {0, 0, 0, 0};
  for (size_t r = threadIdx.x; r < N3; r += 256) {
    if (owner[r] != a) continue;
    const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
    acc[0] += 2.0 * r2;
    acc[1] += -2.0 * r3;
    acc[2] += r0 - r1;
    acc[3] += r0 + r1;
  }
  for (int c = 0; c < 4; ++c) {
    const double t = block_sum<256>(acc[c], sh);
    if (threadIdx.x == 0) out[4 * a + c] = t;
    __syncthreads();
  }
}
cudaError_t launch_atom_sums(cudaStream_t st, size_t N3, int natoms, const double* rho, const int* owner, double* out) {
  k_atom_sums<<<natoms, 256, 0, st>>>(N3, rho, owner, out);
  return cudaGetLastError();
}

// ============================================================================ instantiations
#define TDDFT_INST(R)                                                                                           \
  template cudaError_t launch_fft_xy<R>(cudaStream_t, int, const void*, void*, int, const void*, bool);                       \
  template cudaError_t launch_fft_z<R>(cudaStream_t, int, void*, int, const void*, int, const ZParams&);          \
  template cudaError_t launch_proj_gather<R>(cudaStream_t, int, const void*, int, const ProjTables<R>&, double,  \
                                             const EpiParams&, void*, void*);                                   \
  template cudaError_t launch_density<R>(cudaStream_t, size_t, const void*, int, const double*, double*,         \
                                         double*);                                                                \
  template cudaError_t launch_convert_in<R>(cudaStream_t, size_t, const double2*, void*);                        \
  template cudaError_t launch_convert_out<R>(cudaStream_t, size_t, const void*, double2*);                       \
  template cudaError_t launch_band_dot<R>(cudaStream_t, size_t, int, const void*, const void*, double*, double*); \
  template cudaError_t launch_nl_energy<R>(cudaStream_t, int, int, const void*, const void*, double*);          \
  template cudaError_t launch_soc_torque<R>(cudaStream_t, int, int, int, const void*, const double2*, double*);

TDDFT_INST(float)
TDDFT_INST(double)

}  // namespace tddft
