// Kernels of the discrete adjoint (reverse mode) of the ETRS propagation step.
//
// Cotangent convention: for a real loss L and complex arrays, psibar = dL/dRe psi + i dL/dIm psi,
// so dL = Re sum conj(psibar) dpsi over the array (no dV).
//
//   k_grad_v          dRe<S, dV T>/dV_v(r) summed over spinors (4-vector potential gradient)
//   k_fft_z_current   z pass on the xy transforms of S and T: accumulates the kinetic current
//                     Re sum_G conj(S^) (G + k + A)_a T^ and applies the kinetic multiply to S
//   k_nl_agrad_fused  projector-phase part of dRe<S, dV_NL T>/dA in one pass over the entries
//   k_xc_adjoint      locally collinear LSDA Jacobian-transpose (analytic second derivatives of
//                     Slater exchange and PW92 correlation), the B-field and Hartree inputs
//   k_density_adjoint psibar += d rho_v / d psi ^T rhobar  (Eqs. rho1-rho3, density4)
//   k_seed            out = a y1 + b y2 (complex coefficients)
#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"
#include "kepi.cuh"

namespace tddft {

// ------------------------------------------------------------------ potential gradient
// Band group g = blockIdx.y sums spinors [kb0, kb1) for two neighbouring points per thread (the
// density kernel's layout); FP32 spinors sum up to 8 spinors in FP32 before each FP64 addition.
// With one group the result goes straight into gV (+= f x), else the groups' partials are added
// in a fixed order by k_grad_v_reduce.
template <typename R>
__global__ void __launch_bounds__(256)
k_grad_v(const typename CT<R>::type* __restrict__ S, const typename CT<R>::type* __restrict__ T, size_t N3, int nkb,
         int ngroups, double f, double* __restrict__ gV, double* __restrict__ part) {
  using C = typename CT<R>::type;
  const size_t r = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (r >= N3) return;
  const int g = blockIdx.y;
  const int kb0 = (int)(((long long)nkb * g) / ngroups), kb1 = (int)(((long long)nkb * (g + 1)) / ngroups);
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  constexpr int CH = sizeof(R) == 4 ? 8 : 1;
  for (int kc = kb0; kc < kb1; kc += CH) {
    R p[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const int kend = min(kb1, kc + CH);
#pragma unroll 1
    for (int kb = kc; kb < kend; ++kb) {
      const size_t ou = (size_t)(2 * kb) * N3 + r, od = ou + N3;
      const Pair<C> su = ld2(S + ou), sd = ld2(S + od), tu = ld2(T + ou), td = ld2(T + od);
      const C sus[2] = {su.a, su.b}, sds[2] = {sd.a, sd.b}, tus[2] = {tu.a, tu.b}, tds[2] = {td.a, td.b};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R sux = sus[j].x, suy = sus[j].y, sdx = sds[j].x, sdy = sds[j].y;
        const R tux = tus[j].x, tuy = tus[j].y, tdx = tds[j].x, tdy = tds[j].y;
        p[j][0] += sux * tux + suy * tuy;  // Re(conj(su) tu)
        p[j][1] += sdx * tdx + sdy * tdy;  // Re(conj(sd) td)
        p[j][2] += (R)0.5 * ((sux * tdx + suy * tdy) + (sdx * tux + sdy * tuy));
        // 1/2 [Re(i conj(su) td) - Re(i conj(sd) tu)] = 1/2 [-Im(conj(su) td) + Im(conj(sd) tu)]
        p[j][3] += (R)0.5 * (-(sux * tdy - suy * tdx) + (sdx * tuy - sdy * tux));
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[j][c] += (double)p[j][c];
  }
  if (ngroups == 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gV[c * N3 + r] += f * acc[0][c];
      gV[c * N3 + r + 1] += f * acc[1][c];
    }
    return;
  }
  double* o = part + (size_t)g * 4 * N3;
#pragma unroll
  for (int c = 0; c < 4; ++c) *reinterpret_cast<double2*>(o + c * N3 + r) = make_double2(acc[0][c], acc[1][c]);
}

__global__ void k_grad_v_reduce(size_t n, int ngroups, const double* __restrict__ part, double f, double* gV) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int g = 0; g < ngroups; ++g) t += part[(size_t)g * n + i];
  gV[i] += f * t;
}

template <typename R>
cudaError_t launch_grad_v(cudaStream_t st, size_t N3, int nkb, const void* S, const void* T, double f, double* gV,
                          double* part) {
  using C = typename CT<R>::type;
  const int G = part ? density_groups(N3, nkb) : 1;
  dim3 grid((unsigned)((N3 / 2 + 255) / 256), G);
  k_grad_v<R><<<grid, 256, 0, st>>>((const C*)S, (const C*)T, N3, nkb, G, f, gV, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || G == 1) return e;
  k_grad_v_reduce<<<(unsigned)((4 * N3 + 255) / 256), 256, 0, st>>>(4 * N3, G, part, f, gV);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ kinetic current
// One y-slab of one component: U holds the xy transform of S (overwritten by the z-inverse of
// the kinetic-multiplied transform), W the xy transform of T.  part[b][y][a] receives
// Re sum_{x,z} conj(U^) (G + s)_a W^ for this slab (unnormalised transforms).
template <typename R, int N>
__global__ void __launch_bounds__(256)
k_fft_z_current(typename CT<R>::type* __restrict__ U, const typename CT<R>::type* __restrict__ W,
                const typename CT<R>::type* __restrict__ twg, ZParams zp, double* __restrict__ part) {
  using C = typename CT<R>::type;
  constexpr int NT = 256;
  constexpr int RS = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* su = tw + N;
  C* sw = su + N * RS;
  double* red = reinterpret_cast<double*>(sw + N * RS);  // [8][3]
  const int y = blockIdx.x;
  const int b = blockIdx.y;
  const int k = b / zp.comps_per_k;
  const size_t base = (size_t)b * N * N * N + (size_t)y * N;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  slab_load<N, NT, RS>(su, U + base, (size_t)N * N);
  slab_load<N, NT, RS>(sw, W + base, (size_t)N * N);
  __syncthreads();
  fft_pass<C, N, NT, false, 2>(su, 1, RS, tw, N * RS);  // z transforms of both slabs
  const double qy = zp.gs[1] * freq<N>(y) + zp.shift[k][1];
  double ax = 0, ay = 0, az = 0;
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int z = i / N, x = i - z * N;
    const C u = su[z * RS + x], w = sw[z * RS + x];
    const double re = (double)u.x * w.x + (double)u.y * w.y;  // Re(conj(u) w)
    const double qx = zp.gs[0] * freq<N>(x) + zp.shift[k][0];
    const double qz = zp.gs[2] * freq<N>(z) + zp.shift[k][2];
    ax += re * qx;
    ay += re * qy;
    az += re * qz;
    const R m = (R)(0.5 * (qx * qx + qy * qy + qz * qz) * zp.scale);
    su[z * RS + x] = cscale(u, m);
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  az = warp_sum(az);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[3 * warp] = ax;
    red[3 * warp + 1] = ay;
    red[3 * warp + 2] = az;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w8 = 0; w8 < NT / 32; ++w8) t += red[3 * w8 + threadIdx.x];
    part[((size_t)b * N + y) * 3 + threadIdx.x] = t;
  }
  fft_pass<C, N, NT, true>(su, 1, RS, tw);
  slab_store<N, NT, RS>(U + base, su, (size_t)N * N);
}

// Two-factor form of the same pass (n = R1 R2, see k_fft_z2_kin): A side (x, n0) reads both
// slabs along z, B side (x, K0) holds U^ and W^ at kz = K0 + R2 K1 in registers, adds
// Re(conj(U^) W^) (G + s)_a over its K1 in the working precision before the FP64 sums, then
// multiplies U^ by the kinetic factor and transforms it back.
template <typename R, int N>
__global__ void __launch_bounds__(256)
k_fft_z2_current(typename CT<R>::type* __restrict__ U, const typename CT<R>::type* __restrict__ W,
                 const typename CT<R>::type* __restrict__ twg, ZParams zp, double* __restrict__ part) {
  using C = typename CT<R>::type;
  using TFW = TF<C, N, false>;
  using TIN = TF<C, N, true>;
  constexpr int NT = 256;
  constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  constexpr int IA = N * R1, IB = N * R2;
  constexpr int PA = (IA + NT - 1) / NT, PB = (IB + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* su = tw + N;            // [K0 R1 + n0][x]
  C* sw = su + N * N;
  R* kx = reinterpret_cast<R*>(sw + N * N);  // kinetic factors 1/2 q^2 scale per axis
  R* kz = kx + N;
  R* vx = kz + N;                            // velocities q_a = g_a f(i) + s_a
  R* vz = vx + N;
  double* red = reinterpret_cast<double*>(vz + N + (N & 1));  // [8][3], 8-byte aligned
  const int y = blockIdx.x;
  const int b = blockIdx.y;
  const int k = b / zp.comps_per_k;
  const size_t base = (size_t)b * N * N * N + (size_t)y * N;
  constexpr size_t ZS = (size_t)N * N;
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = twg[i];
    const double qx = zp.gs[0] * freq<N>(i) + zp.shift[k][0];
    const double qz = zp.gs[2] * freq<N>(i) + zp.shift[k][2];
    kx[i] = (R)(0.5 * qx * qx * zp.scale);
    kz[i] = (R)(0.5 * qz * qz * zp.scale);
    vx[i] = (R)qx;
    vz[i] = (R)qz;
  }
  const double qyd = zp.gs[1] * freq<N>(y) + zp.shift[k][1];
  const R qy = (R)qyd, ky = (R)(0.5 * qyd * qyd * zp.scale);
  C vu[PA][R2], vw[PA][R2];
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
#pragma unroll
      for (int q = 0; q < R2; ++q) {
        vu[p][q] = U[base + (size_t)(n0 + R1 * q) * ZS + x];
        vw[p][q] = W[base + (size_t)(n0 + R1 * q) * ZS + x];
      }
    }
  }
  __syncthreads();  // tables
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
      TFW::a_side(vu[p], n0, tw);
      TFW::a_side(vw[p], n0, tw);
#pragma unroll
      for (int k0 = 0; k0 < R2; ++k0) {
        su[(k0 * R1 + n0) * N + x] = vu[p][k0];
        sw[(k0 * R1 + n0) * N + x] = vw[p][k0];
      }
    }
  }
  __syncthreads();
  double ax = 0, ay = 0, az = 0;
#pragma unroll
  for (int p = 0; p < PB; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IB % NT == 0 || i < IB) {
      const int k0 = i / N, x = i - k0 * N;
      C a[R1], w[R1];
#pragma unroll
      for (int n0 = 0; n0 < R1; ++n0) {
        a[n0] = su[(k0 * R1 + n0) * N + x];
        w[n0] = sw[(k0 * R1 + n0) * N + x];
      }
      TFW::b_side(a, k0, tw);
      TFW::b_side(w, k0, tw);
      R cx = 0, cz = 0, cs = 0;
      const R kxy = kx[x] + ky;
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int kzi = k0 + R2 * k1;
        const R re = a[k1].x * w[k1].x + a[k1].y * w[k1].y;  // Re(conj(U^) W^)
        cs += re;
        cz += re * vz[kzi];
        a[k1] = cscale(a[k1], kxy + kz[kzi]);
      }
      cx = cs * vx[x];
      ax += (double)cx;
      ay += (double)cs * (double)qy;
      az += (double)cz;
      TIN::b_side(a, k0, tw);
#pragma unroll
      for (int n0 = 0; n0 < R1; ++n0) su[(k0 * R1 + n0) * N + x] = a[n0];
    }
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  az = warp_sum(az);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[3 * warp] = ax;
    red[3 * warp + 1] = ay;
    red[3 * warp + 2] = az;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w8 = 0; w8 < NT / 32; ++w8) t += red[3 * w8 + threadIdx.x];
    part[((size_t)b * N + y) * 3 + threadIdx.x] = t;
  }
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    const int i = threadIdx.x + p * NT;
    if (IA % NT == 0 || i < IA) {
      const int n0 = i / N, x = i - n0 * N;
#pragma unroll
      for (int k0 = 0; k0 < R2; ++k0) vu[p][k0] = su[(k0 * R1 + n0) * N + x];
      TIN::a_side(vu[p], n0, tw);
#pragma unroll
      for (int n1 = 0; n1 < R2; ++n1) U[base + (size_t)(n0 + R1 * n1) * ZS + x] = vu[p][n1];
    }
  }
}

template <typename R, int N>
static cudaError_t z_current_n(cudaStream_t st, void* U, const void* W, int nbatch, const void* tw, const ZParams& zp,
                               double* part) {
  using C = typename CT<R>::type;
  if constexpr (TwoFactor<N>::ok) {
    const size_t smem2 = (size_t)(N + 2 * N * N) * sizeof(C) + (size_t)(4 * N + 2) * sizeof(R) + 24 * sizeof(double);
    auto kf2 = k_fft_z2_current<R, N>;
    cudaFuncSetAttribute(kf2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    kf2<<<dim3(N, nbatch), 256, smem2, st>>>((C*)U, (const C*)W, (const C*)tw, zp, part);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)(N + 2 * N * (N + 1)) * sizeof(C) + 24 * sizeof(double);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  auto kf = k_fft_z_current<R, N>;
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kf<<<dim3(N, nbatch), 256, smem, st>>>((C*)U, (const C*)W, (const C*)tw, zp, part);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_z_current(cudaStream_t st, int N, void* U, const void* W, int nbatch, const void* tw,
                                 const ZParams& zp, double* part) {
  TDDFT_DISPATCH_N(N, (z_current_n<R, NN>(st, U, W, nbatch, tw, zp, part)));
}

// out3[a] += f * sum_i part[3 i + a] over count rows (single CTA, fixed order).
__global__ void __launch_bounds__(256) k_accum_parts(size_t count, const double* __restrict__ part, double f,
                                                      double* __restrict__ out3) {
  __shared__ double sh[8 * 3];
  double acc[3] = {0, 0, 0};
  for (size_t i = threadIdx.x; i < count; i += 256)
    for (int a = 0; a < 3; ++a) acc[a] += part[3 * i + a];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = 0; a < 3; ++a) {
    const double v = warp_sum(acc[a]);
    if (lane == 0) sh[3 * warp + a] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[3 * w + threadIdx.x];
    out3[threadIdx.x] += f * t;
  }
}
cudaError_t launch_accum_parts(cudaStream_t st, size_t count, const double* part, double f, double* out3) {
  k_accum_parts<<<1, 256, 0, st>>>(count, part, f, out3);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ projector-phase gradient
// d Re<S, V_NL T> / dA_alpha through the projector phases exp(-i (k + A).d): with the moment
// projections m^alpha_p[X] = sum_e d_alpha beta_p e^{i phi} X(e) dV (phi = (k + A).d) it is
//   sum_{p, sigma} [ Im(conj(m^alpha_p[S]) (D c_T)_p) + Im(conj(m^alpha_p[T]) (D c_S)_p) ],
// and since beta is real this equals, per atom and spinor, one pass over the sphere entries:
//   sum_e d_alpha Im( e^{-i phi} [conj(S) w_T + conj(T) w_S] ) dV,  w_X = sum_p beta_p (D c_X)_p,
// summed over both spin components.  The caller's 1/dV cancels the dV.  Partials per (spinor,
// atom) are added over atoms in a fixed order by k_nl_agrad_sum.
template <typename R, int NLM>
__global__ void __launch_bounds__(256)
k_nl_agrad_fused(const typename CT<R>::type* __restrict__ S, const typename CT<R>::type* __restrict__ T, size_t N3,
                 ProjTables<R> pt, EpiParams ep, const typename CT<R>::type* __restrict__ dcS,
                 const typename CT<R>::type* __restrict__ dcT, double* __restrict__ part) {
  using C = typename CT<R>::type;
  const int a = blockIdx.x;
  const int kb = blockIdx.y;
  const int k = kb / ep.nstates;
  const R sx = (R)ep.shift[k][0], sy = (R)ep.shift[k][1], sz = (R)ep.shift[k][2];
  __shared__ C dS[2 * NLM], dT[2 * NLM];
  __shared__ double red[8][3];
  const size_t cof = ((size_t)kb * pt.natoms + a) * 2 * NLM;
  if (threadIdx.x < 2 * NLM) {
    dS[threadIdx.x] = dcS[cof + threadIdx.x];
    dT[threadIdx.x] = dcT[cof + threadIdx.x];
  }
  __syncthreads();
  R nl[4];
  load_row<R, 4>(pt.nrm + (size_t)a * 4, nl);
  const C* su_ = S + (size_t)(2 * kb) * N3;
  const C* sd_ = su_ + N3;
  const C* tu_ = T + (size_t)(2 * kb) * N3;
  const C* td_ = tu_ + N3;
  double acc[3] = {0.0, 0.0, 0.0};
  const int e0 = pt.g_ptr[a], e1 = pt.g_ptr[a + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += 256) {
    const int r = pt.g_idx[e];
    R t[4], bt[NLM];
    load_row<R, 4>(pt.g_row + (size_t)e * 4, t);
    beta_values<R, NLM>(t[0], t[1], t[2], t[3], nl, pt.yc, bt);
    R sn, cs;
    sincos_r<R>(sx * t[0] + sy * t[1] + sz * t[2], &sn, &cs);
    const C su = su_[r], sd = sd_[r], tu = tu_[r], td = td_[r];
    R wtu_x = 0, wtu_y = 0, wtd_x = 0, wtd_y = 0, wsu_x = 0, wsu_y = 0, wsd_x = 0, wsd_y = 0;
#pragma unroll
    for (int p = 0; p < NLM; ++p) {
      const R bp = bt[p];
      wtu_x += bp * dT[2 * p].x; wtu_y += bp * dT[2 * p].y;
      wtd_x += bp * dT[2 * p + 1].x; wtd_y += bp * dT[2 * p + 1].y;
      wsu_x += bp * dS[2 * p].x; wsu_y += bp * dS[2 * p].y;
      wsd_x += bp * dS[2 * p + 1].x; wsd_y += bp * dS[2 * p + 1].y;
    }
    // X = conj(su) wTu + conj(sd) wTd + conj(tu) wSu + conj(td) wSd
    const R xr = su.x * wtu_x + su.y * wtu_y + sd.x * wtd_x + sd.y * wtd_y + tu.x * wsu_x + tu.y * wsu_y +
                 td.x * wsd_x + td.y * wsd_y;
    const R xi = su.x * wtu_y - su.y * wtu_x + sd.x * wtd_y - sd.y * wtd_x + tu.x * wsu_y - tu.y * wsu_x +
                 td.x * wsd_y - td.y * wsd_x;
    const double im = (double)(cs * xi - sn * xr);  // Im(e^{-i phi} X)
    acc[0] += (double)t[0] * im;
    acc[1] += (double)t[1] * im;
    acc[2] += (double)t[2] * im;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double tsum = 0.0;
    for (int w = 0; w < 8; ++w) tsum += red[w][threadIdx.x];
    part[((size_t)kb * pt.natoms + a) * 3 + threadIdx.x] = tsum;
  }
}

// out[3 kb + i] += f sum_a part[kb][a][i], atoms in order.
__global__ void k_nl_agrad_sum(int nkb, int natoms, const double* __restrict__ part, double f, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 3 * nkb) return;
  const int kb = j / 3, i = j - 3 * kb;
  double t = 0.0;
  for (int a = 0; a < natoms; ++a) t += part[((size_t)kb * natoms + a) * 3 + i];
  out[j] += f * t;
}

template <typename R>
cudaError_t launch_nl_agrad_fused(cudaStream_t st, int N, const void* S, const void* T, int nkb,
                                  const ProjTables<R>& pt, const EpiParams& ep, const void* dcS, const void* dcT,
                                  double f, double* part, double* out) {
  using C = typename CT<R>::type;
  const size_t N3 = (size_t)N * N * N;
  dim3 grid(pt.natoms, nkb);
#define NLA_ARGS (const C*)S, (const C*)T, N3, pt, ep, (const C*)dcS, (const C*)dcT, part
  switch (pt.nlm) {
    case 1: k_nl_agrad_fused<R, 1><<<grid, 256, 0, st>>>(NLA_ARGS); break;
    case 4: k_nl_agrad_fused<R, 4><<<grid, 256, 0, st>>>(NLA_ARGS); break;
    case 9: k_nl_agrad_fused<R, 9><<<grid, 256, 0, st>>>(NLA_ARGS); break;
    default: return cudaErrorInvalidValue;
  }
#undef NLA_ARGS
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nl_agrad_sum<<<(3 * nkb + 127) / 128, 128, 0, st>>>(nkb, pt.natoms, part, f, out);
  return cudaGetLastError();
}



// ------------------------------------------------------------------ XC adjoint
// PW92 G(rs) with first and second derivatives.
__device__ __forceinline__ void pw92_g2(double rs, double A, double a1, double b1, double b2, double b3, double b4,
                                        double* g, double* dg, double* d2g) {
  const double sr = sqrt(rs);
  const double q0 = -2.0 * A * (1.0 + a1 * rs);
  const double q1 = 2.0 * A * sr * (b1 + sr * (b2 + sr * (b3 + sr * b4)));
  const double q1p = A * (b1 / sr + 2.0 * b2 + 3.0 * b3 * sr + 4.0 * b4 * rs);
  const double q1pp = A * (-0.5 * b1 / (rs * sr) + 1.5 * b3 / sr + 4.0 * b4);
  const double den = q1 * (q1 + 1.0);
  const double lg = log1p(1.0 / q1);
  *g = q0 * lg;
  *dg = -2.0 * A * a1 * lg - q0 * q1p / den;
  *d2g = 4.0 * A * a1 * q1p / den - q0 * q1pp / den + q0 * q1p * q1p * (2.0 * q1 + 1.0) / (den * den);
}

// LSDA potentials and Hessian d v_sigma / d n_sigma' (Slater exchange + PW92 correlation).
__device__ void lsda_hessian_point(double nu, double nd, double* vu, double* vd, double* huu, double* hud,
                                   double* hdd) {
  const double kPi = 3.14159265358979323846;
  const double c6 = cbrt(6.0 / kPi);
  const double cbu = cbrt(nu), cbd = cbrt(nd);
  double vxu = -c6 * cbu, vxd = -c6 * cbd;
  double hxu = nu > 0.0 ? -c6 / (3.0 * cbu * cbu) : 0.0;
  double hxd = nd > 0.0 ? -c6 / (3.0 * cbd * cbd) : 0.0;
  const double n = nu + nd;
  const double rs = cbrt(3.0 / (4.0 * kPi * n));
  double z = (nu - nd) / n;
  z = fmin(1.0, fmax(-1.0, z));
  double ec0, d0, dd0, ec1, d1, dd1, mac, dmac, ddmac;
  pw92_g2(rs, 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294, &ec0, &d0, &dd0);
  pw92_g2(rs, 0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517, &ec1, &d1, &dd1);
  pw92_g2(rs, 0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671, &mac, &dmac, &ddmac);
  const double ac = -mac, dac = -dmac, ddac = -ddmac;
  const double fden = 1.0 / (cbrt(16.0) - 2.0);
  const double opz = 1.0 + z, omz = 1.0 - z;
  const double cpz = cbrt(opz), cmz = cbrt(omz);
  const double f = (opz * cpz + omz * cmz - 2.0) * fden;
  const double fp = (4.0 / 3.0) * (cpz - cmz) * fden;
  const double fpp = (4.0 / 9.0) * ((opz > 0.0 ? 1.0 / (cpz * cpz) : 0.0) + (omz > 0.0 ? 1.0 / (cmz * cmz) : 0.0)) * fden;
  const double fpp0 = 1.709921;
  const double z2 = z * z, z3 = z2 * z, z4 = z3 * z;
  const double de = ec1 - ec0, dde = d1 - d0, ddde = dd1 - dd0;
  const double ec = ec0 + ac * f * (1.0 - z4) / fpp0 + de * f * z4;
  const double e_r = d0 + dac * f * (1.0 - z4) / fpp0 + dde * f * z4;
  const double e_rr = dd0 + ddac * f * (1.0 - z4) / fpp0 + ddde * f * z4;
  const double pa = fp * (1.0 - z4) - 4.0 * z3 * f, pb = fp * z4 + 4.0 * z3 * f;
  const double e_z = ac / fpp0 * pa + de * pb;
  const double e_rz = dac / fpp0 * pa + dde * pb;
  const double e_zz = ac / fpp0 * (fpp * (1.0 - z4) - 8.0 * z3 * fp - 12.0 * z2 * f) +
                      de * (fpp * z4 + 8.0 * z3 * fp + 12.0 * z2 * f);
  const double common = ec - rs / 3.0 * e_r;
  *vu = vxu + common - (z - 1.0) * e_z;
  *vd = vxd + common - (z + 1.0) * e_z;
  // v_c,sigma = Q_sigma(rs, z); dQ/drs and dQ/dz, with drs/dn_s' = -rs/(3n), dz/dn_s' = (s' - z)/n
  const double drs = -rs / (3.0 * n);
  const double qr_u = (2.0 / 3.0) * e_r - rs / 3.0 * e_rr - (z - 1.0) * e_rz;
  const double qr_d = (2.0 / 3.0) * e_r - rs / 3.0 * e_rr - (z + 1.0) * e_rz;
  const double qz_u = -rs / 3.0 * e_rz - (z - 1.0) * e_zz;
  const double qz_d = -rs / 3.0 * e_rz - (z + 1.0) * e_zz;
  const double dzu = (1.0 - z) / n, dzd = (-1.0 - z) / n;
  *huu = hxu + qr_u * drs + qz_u * dzu;
  *hud = qr_u * drs + qz_u * dzd;  // d v_u / d n_d (symmetric)
  *hdd = hxd + qr_d * drs + qz_d * dzd;
}

// Per point: from gV (cotangent of V_v) and rho_v, produce the XC part of rhobar, the scalar
// field gv = gV0 + gV1 (input of the Hartree adjoint) and per-point b-cotangents for dL/dB.
__global__ void k_xc_adjoint(size_t N3, const double* __restrict__ rho, const double* __restrict__ gV, int xc,
                             double* __restrict__ rbar, double* __restrict__ gvf, double* __restrict__ gbf) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  const double gv = gV[r] + gV[N3 + r];
  const double gbx = 2.0 * gV[2 * N3 + r], gby = -2.0 * gV[3 * N3 + r], gbz = gV[r] - gV[N3 + r];
  gvf[r] = gv;
  gbf[r] = gbx;
  gbf[N3 + r] = gby;
  gbf[2 * N3 + r] = gbz;
  double nbar = 0.0, mbx = 0.0, mby = 0.0, mbz = 0.0;
  const double r0 = rho[r], r1 = rho[N3 + r], r2 = rho[2 * N3 + r], r3 = rho[3 * N3 + r];
  const double n = r0 + r1, mx = 2.0 * r2, my = -2.0 * r3, mz = r0 - r1;
  if (xc && n >= 1e-14) {
    const double mag = sqrt(mx * mx + my * my + mz * mz);
    const bool clamp = mag > n;
    const double s = fmin(mag, n);
    double vu, vd, huu, hud, hdd;
    lsda_hessian_point(0.5 * (n + s), 0.5 * (n - s), &vu, &vd, &huu, &hud, &hdd);
    const double u_n = 0.5 * (huu + hud), u_s = 0.5 * (huu - hud);
    const double d_n = 0.5 * (hud + hdd), d_s = 0.5 * (hud - hdd);
    const double vbar_n = 0.5 * (u_n + d_n), vbar_s = 0.5 * (u_s + d_s);
    const double beta_n = 0.5 * (u_n - d_n), beta_s = 0.5 * (u_s - d_s);
    const double beta = 0.5 * (vu - vd);
    const bool dirok = mag > 1e-14;
    double mhx = 0.0, mhy = 0.0, mhz = 0.0, mg = 0.0;
    if (dirok) {
      mhx = mx / mag; mhy = my / mag; mhz = mz / mag;
      mg = mhx * gbx + mhy * gby + mhz * gbz;
    }
    const double gs = vbar_s * gv + (dirok ? beta_s * mg : 0.0);
    nbar = vbar_n * gv + (dirok ? beta_n * mg : 0.0) + (clamp ? gs : 0.0);
    if (!clamp) {
      mbx = gs * mhx; mby = gs * mhy; mbz = gs * mhz;
    }
    if (dirok) {
      const double q = beta / mag;
      mbx += q * (gbx - mg * mhx);
      mby += q * (gby - mg * mhy);
      mbz += q * (gbz - mg * mhz);
    }
  }
  // (n, m) -> rho_v: n = r0 + r1, m_x = 2 r2, m_y = -2 r3, m_z = r0 - r1
  rbar[r] = nbar + mbz;
  rbar[N3 + r] = nbar - mbz;
  rbar[2 * N3 + r] = 2.0 * mbx;
  rbar[3 * N3 + r] = -2.0 * mby;
}

cudaError_t launch_xc_adjoint(cudaStream_t st, size_t N3, const double* rho, const double* gV, int xc, double* rbar,
                              double* gvf, double* gbf) {
  k_xc_adjoint<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, rho, gV, xc, rbar, gvf, gbf);
  return cudaGetLastError();
}

// rbar[0], rbar[1] += vH-adjoint field (real part of the Hartree-transformed gv).
__global__ void k_add_hartree_adjoint(size_t N3, const double2* __restrict__ h, double* __restrict__ rbar) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  rbar[r] += h[r].x;
  rbar[N3 + r] += h[r].x;
}
cudaError_t launch_add_hartree_adjoint(cudaStream_t st, size_t N3, const double2* h, double* rbar) {
  k_add_hartree_adjoint<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, h, rbar);
  return cudaGetLastError();
}

__global__ void k_real_field_to_complex(size_t n, const double* in, double2* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(in[i], 0.0);
}
cudaError_t launch_real_field_to_complex(cudaStream_t st, size_t N3, const double* in, double2* out) {
  k_real_field_to_complex<<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, in, out);
  return cudaGetLastError();
}

// Deterministic single-CTA sums of the three b-cotangent fields.
__global__ void __launch_bounds__(1024) k_sum3(size_t N3, const double* __restrict__ g, double* out) {
  __shared__ double sh[32];
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
    for (size_t r = threadIdx.x; r < N3; r += 1024) s += g[a * N3 + r];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 32; ++w) t += sh[w];
      out[a] = t;
    }
    __syncthreads();
  }
}
cudaError_t launch_sum3(cudaStream_t st, size_t N3, const double* g, double* out) {
  k_sum3<<<1, 1024, 0, st>>>(N3, g, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ density adjoint
// out = add + w [ 2 r0 u + (r2 + i r3) d ,  2 r1 d + (r2 - i r3) u ]   (add may alias out)
template <typename R>
__global__ void __launch_bounds__(256)
k_density_adjoint(const typename CT<R>::type* __restrict__ psi, const double* __restrict__ rbar,
                  const double* __restrict__ wf, size_t N3, const typename CT<R>::type* add,
                  typename CT<R>::type* out) {
  using C = typename CT<R>::type;
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N3) return;
  const int kb = blockIdx.y;
  const size_t ou = (size_t)(2 * kb) * N3 + r, od = ou + N3;
  // in the working precision R (the output's; FP64 arithmetic is scarce on this part)
  const R w = (R)wf[kb];
  const R r0 = (R)rbar[r], r1 = (R)rbar[N3 + r], r2 = (R)rbar[2 * N3 + r], r3 = (R)rbar[3 * N3 + r];
  const C u = psi[ou], d = psi[od];
  R bux = w * ((R)2 * r0 * u.x + r2 * d.x - r3 * d.y);
  R buy = w * ((R)2 * r0 * u.y + r2 * d.y + r3 * d.x);
  R bdx = w * ((R)2 * r1 * d.x + r2 * u.x + r3 * u.y);
  R bdy = w * ((R)2 * r1 * d.y + r2 * u.y - r3 * u.x);
  if (add) {
    const C au = add[ou], ad = add[od];
    bux += au.x; buy += au.y; bdx += ad.x; bdy += ad.y;
  }
  out[ou] = cmake<C>(bux, buy);
  out[od] = cmake<C>(bdx, bdy);
}
template <typename R>
cudaError_t launch_density_adjoint(cudaStream_t st, size_t N3, int nkb, const void* psi, const double* rbar,
                                   const double* wf, const void* add, void* out) {
  using C = typename CT<R>::type;
  k_density_adjoint<R><<<dim3((unsigned)((N3 + 255) / 256), nkb), 256, 0, st>>>((const C*)psi, rbar, wf, N3,
                                                                                (const C*)add, (C*)out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ seeds
template <typename R>
__global__ void k_seed(size_t n, const typename CT<R>::type* __restrict__ y1, double ar, double ai,
                       const typename CT<R>::type* __restrict__ y2, double br, double bi,
                       typename CT<R>::type* __restrict__ out) {
  using C = typename CT<R>::type;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // in the working precision R (the output's; FP64 arithmetic is scarce on this part)
  R x = 0, y = 0;
  if (y1) {
    const C v = y1[i];
    x += (R)ar * v.x - (R)ai * v.y;
    y += (R)ar * v.y + (R)ai * v.x;
  }
  if (y2) {
    const C v = y2[i];
    x += (R)br * v.x - (R)bi * v.y;
    y += (R)br * v.y + (R)bi * v.x;
  }
  out[i] = cmake<C>(x, y);
}
template <typename R>
cudaError_t launch_seed(cudaStream_t st, size_t n, const void* y1, const double a[2], const void* y2,
                        const double b[2], void* out) {
  using C = typename CT<R>::type;
  k_seed<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (const C*)y1, a[0], a[1], (const C*)y2, b[0], b[1],
                                                          (C*)out);
  return cudaGetLastError();
}

#define TDDFT_ADJ_INST(R)                                                                                        \
  template cudaError_t launch_grad_v<R>(cudaStream_t, size_t, int, const void*, const void*, double, double*,       \
                                       double*);                                                                 \
  template cudaError_t launch_fft_z_current<R>(cudaStream_t, int, void*, const void*, int, const void*,            \
                                               const ZParams&, double*);                                         \
  template cudaError_t launch_density_adjoint<R>(cudaStream_t, size_t, int, const void*, const double*,           \
                                                 const double*, const void*, void*);                             \
  template cudaError_t launch_seed<R>(cudaStream_t, size_t, const void*, const double*, const void*,              \
                                      const double*, void*);                                                     \
  template cudaError_t launch_nl_agrad_fused<R>(cudaStream_t, int, const void*, const void*, int,                 \
                                                const ProjTables<R>&, const EpiParams&, const void*, const void*,  \
                                                double, double*, double*);

TDDFT_ADJ_INST(float)
TDDFT_ADJ_INST(double)

}  // namespace tddft
