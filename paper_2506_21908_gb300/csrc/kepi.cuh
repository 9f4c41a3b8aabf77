// Point-wise Hamiltonian helpers shared by the epilogue kernels: the 2x2 spin-matrix local
// potential [[v + b_z, b_x - i b_y], [b_x + i b_y, v - b_z]] from the 4-vector
// V_v = [v + b_z, v - b_z, 2 b_x, -2 b_y] (Eq. potential4) and the projector scatter
// sum_a sum_p beta_p(d) exp(-i (k+A).d) (D c)_p (Eq. Vps with the L.S blocks).
#pragma once
#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"

namespace tddft {

template <typename C> struct Pair { C a, b; };
__device__ __forceinline__ Pair<float2> ld2(const float2* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st2(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ Pair<double2> ld2(const double2* p) { return {p[0], p[1]}; }
__device__ __forceinline__ void st2(double2* p, double2 a, double2 b) { p[0] = a; p[1] = b; }

// One row of a projector table (3 + NLM values: d, beta).  Rows whose size is a multiple of
// 16 bytes start on 16-byte boundaries (the table is one allocation) and are read as vectors.
template <typename R, int TAB>
__device__ __forceinline__ void load_row(const R* __restrict__ t, R* v) {
  if constexpr (sizeof(R) == 4 && TAB % 4 == 0) {
    const float4* t4 = reinterpret_cast<const float4*>(t);
#pragma unroll
    for (int i = 0; i < TAB / 4; ++i) {
      const float4 q = __ldg(t4 + i);
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else if constexpr (sizeof(R) == 8 && TAB % 2 == 0) {
    const double2* t2 = reinterpret_cast<const double2*>(t);
#pragma unroll
    for (int i = 0; i < TAB / 2; ++i) {
      const double2 q = __ldg(t2 + i);
      v[2 * i] = q.x; v[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < TAB; ++i) v[i] = __ldg(t + i);
  }
}

// Projector values beta_p(d) = N_l g S_lm(d), p = l^2 + l + mu, from a compact row (d, g): the
// real solid harmonics r^l Y_lm for l <= 2 in the order of the tables (1; y, z, x; xy, yz,
// 3z^2 - r^2, xz, x^2 - y^2), nl = N_0, N_1, N_2 of the atom, yc the harmonic constants.
template <typename R, int NLM>
__device__ __forceinline__ void beta_values(R x, R y, R z, R g, const R* nl, const R* yc, R* b) {
  b[0] = nl[0] * g * yc[0];
  if constexpr (NLM > 1) {
    const R s1 = nl[1] * g * yc[1];
    b[1] = s1 * y; b[2] = s1 * z; b[3] = s1 * x;
  }
  if constexpr (NLM > 4) {
    const R s2 = nl[2] * g * yc[2], s0 = nl[2] * g * yc[3];
    b[4] = s2 * (x * y); b[5] = s2 * (y * z);
    b[6] = s0 * ((R)2 * z * z - x * x - y * y);
    b[7] = s2 * (x * z); b[8] = (R)0.5 * s2 * (x * x - y * y);
  }
}

// phase exp(-i arg): FP32 reduces the argument to [-pi, pi] and uses the fast intrinsic
__device__ __forceinline__ void phase_sincos(float x, float* sn, float* cs) {
  const float r = x - 6.28318530717958647692f * rintf(x * 0.15915494309189533577f);
  __sincosf(r, sn, cs);
}
__device__ __forceinline__ void phase_sincos(double x, double* sn, double* cs) { sincos(x, sn, cs); }

// Hamiltonian at one point for both spinor components: (hu, hd) holds the kinetic part on
// entry; the 2x2 local potential and the projector scatter are added.
template <typename R, int NLM>
__device__ __forceinline__ void h_point(typename CT<R>::type& hu, typename CT<R>::type& hd, typename CT<R>::type pu,
                                        typename CT<R>::type pd, R V0, R V1, R hx, R hy, size_t r,
                                        const ProjTables<R>& pt, const typename CT<R>::type* dcb, R sx, R sy, R sz) {
  using C = typename CT<R>::type;
  hu = cmake<C>(hu.x + V0 * pu.x + hx * pd.x - hy * pd.y, hu.y + V0 * pu.y + hx * pd.y + hy * pd.x);
  hd = cmake<C>(hd.x + V1 * pd.x + hx * pu.x + hy * pu.y, hd.y + V1 * pd.y + hx * pu.y - hy * pu.x);
  if constexpr (NLM > 0) {
    const int e0 = pt.s_ptr[r], e1 = pt.s_ptr[r + 1];
    for (int e = e0; e < e1; ++e) {
      const int a = pt.s_atom[e];
      R t[4], nl[4], bt[NLM];
      load_row<R, 4>(pt.s_row + (size_t)e * 4, t);
      load_row<R, 4>(pt.nrm + (size_t)a * 4, nl);
      beta_values<R, NLM>(t[0], t[1], t[2], t[3], nl, pt.yc, bt);
      const C* dca = dcb + (size_t)a * 2 * NLM;  // this spinor's D c of atom a, (up, dn) per p
      R vux = 0, vuy = 0, vdx = 0, vdy = 0;
#pragma unroll
      for (int p = 0; p < NLM; ++p) {
        const R bp = bt[p];
        const Pair<C> cc = ld2(dca + 2 * p);
        vux += bp * cc.a.x; vuy += bp * cc.a.y;
        vdx += bp * cc.b.x; vdy += bp * cc.b.y;
      }
      R sn, cs;
      phase_sincos(sx * t[0] + sy * t[1] + sz * t[2], &sn, &cs);
      hu.x += vux * cs + vuy * sn; hu.y += vuy * cs - vux * sn;
      hd.x += vdx * cs + vdy * sn; hd.y += vdy * cs - vdx * sn;
    }
  }
}


// The same for one point of two spinors of one k-point (index g = 0, 1): the projector entries
// of the point, their beta values and phases are evaluated once for both spinors.
template <typename R, int NLM>
__device__ __forceinline__ void h_point_2sp(typename CT<R>::type (&hu)[2], typename CT<R>::type (&hd)[2],
                                            const typename CT<R>::type (&pu)[2], const typename CT<R>::type (&pd)[2],
                                            R V0, R V1, R hx, R hy, size_t r, const ProjTables<R>& pt,
                                            const typename CT<R>::type* dcb0, const typename CT<R>::type* dcb1, R sx,
                                            R sy, R sz) {
  using C = typename CT<R>::type;
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    hu[g] = cmake<C>(hu[g].x + V0 * pu[g].x + hx * pd[g].x - hy * pd[g].y,
                     hu[g].y + V0 * pu[g].y + hx * pd[g].y + hy * pd[g].x);
    hd[g] = cmake<C>(hd[g].x + V1 * pd[g].x + hx * pu[g].x + hy * pu[g].y,
                     hd[g].y + V1 * pd[g].y + hx * pu[g].y - hy * pu[g].x);
  }
  if constexpr (NLM > 0) {
    const int e0 = pt.s_ptr[r], e1 = pt.s_ptr[r + 1];
    for (int e = e0; e < e1; ++e) {
      const int a = pt.s_atom[e];
      R t[4], nl[4], bt[NLM];
      load_row<R, 4>(pt.s_row + (size_t)e * 4, t);
      load_row<R, 4>(pt.nrm + (size_t)a * 4, nl);
      beta_values<R, NLM>(t[0], t[1], t[2], t[3], nl, pt.yc, bt);
      R sn, cs;
      phase_sincos(sx * t[0] + sy * t[1] + sz * t[2], &sn, &cs);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const C* dca = (g ? dcb1 : dcb0) + (size_t)a * 2 * NLM;
        R vux = 0, vuy = 0, vdx = 0, vdy = 0;
#pragma unroll
        for (int p = 0; p < NLM; ++p) {
          const R bp = bt[p];
          const Pair<C> cc = ld2(dca + 2 * p);
          vux += bp * cc.a.x; vuy += bp * cc.a.y;
          vdx += bp * cc.b.x; vdy += bp * cc.b.y;
        }
        hu[g].x += vux * cs + vuy * sn; hu[g].y += vuy * cs - vux * sn;
        hd[g].x += vdx * cs + vdy * sn; hd[g].y += vdy * cs - vdx * sn;
      }
    }
  }
}

}  // namespace tddft
