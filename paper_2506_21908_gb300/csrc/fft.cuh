// Shared-memory batched FFT building blocks (sm_103a).
//
// A plane or slab of N x N complex values lives in shared memory with a padded row
// stride; each pass transforms N rows of length N in place.  Every stage of a
// mixed-radix Stockham decomposition reads its butterflies into registers,
// synchronises the CTA, and writes them back in sorted order, so no second buffer is
// needed and the output is in natural order.  Radices 2, 3, 4 and 8 are available.
//
// Stage algebra (decimation in time).  After the stages with radices r_1..r_s the array
// holds Y[j, k] = sum_t x[k + m t] w_L^{j t} at position j*m + k, L = r_1 ... r_s,
// m = N / L.  A radix-r stage maps Y to Y' with L' = L r, m' = m / r:
//     Y'[j + L p, k'] = sum_q w_r^{p q} ( w_{L'}^{j q} Y[j, k' + m' q] ).
// The twiddle w_{L'}^{j q} equals w_N^{j q m'}; tw[] holds w_N^t = exp(-2 pi i t / N).
#pragma once
#include <cuda_runtime.h>

template <typename R> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) { return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a * conj(b)
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return cmake<C>(a.x * s, a.y * s); }

// Small DFTs in registers; INV selects exp(+2 pi i pq / r).
template <typename C, int RAD, bool INV> struct SmallDFT;

template <typename C, bool INV> struct SmallDFT<C, 2, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C, bool INV> struct SmallDFT<C, 3, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.8660254037844386467637;  // sin(pi/3)
    C a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C base = cmake<C>(a.x - (R)0.5 * s.x, a.y - (R)0.5 * s.y);
    // forward: out1 = base - i h d, out2 = base + i h d
    R sg = INV ? (R)-1 : (R)1;
    v[0] = cadd(a, s);
    v[1] = cmake<C>(base.x + sg * h * d.y, base.y - sg * h * d.x);
    v[2] = cmake<C>(base.x - sg * h * d.y, base.y + sg * h * d.x);
  }
};

template <typename C, bool INV> struct SmallDFT<C, 4, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    // forward: out1 = t1 - i t3, out3 = t1 + i t3
    C mi = INV ? cmake<C>(-t3.y, t3.x) : cmake<C>(t3.y, -t3.x);  // (+/- i) t3
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, mi);
    v[3] = csub(t1, mi);
  }
};

template <typename C, bool INV> struct SmallDFT<C, 8, INV> {
  // radix-2 split into two 4-point DFTs; w8^p = exp(-+ 2 pi i p / 8)
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R r = (R)0.70710678118654752440;  // 1/sqrt(2)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    SmallDFT<C, 4, INV>::run(e);
    SmallDFT<C, 4, INV>::run(o);
    C o1, o2, o3;
    if (!INV) {
      o1 = cmake<C>((o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r);   // (1 - i)/sqrt2
      o2 = cmake<C>(o[2].y, -o[2].x);                                  // -i
      o3 = cmake<C>((o[3].y - o[3].x) * r, -(o[3].x + o[3].y) * r);  // (-1 - i)/sqrt2
    } else {
      o1 = cmake<C>((o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r);   // (1 + i)/sqrt2
      o2 = cmake<C>(-o[2].y, o[2].x);                                  // +i
      o3 = cmake<C>(-(o[3].x + o[3].y) * r, (o[3].x - o[3].y) * r);  // (-1 + i)/sqrt2
    }
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};

template <int... Rs> struct RadixList {};
template <int N> struct FFTPlan;
template <> struct FFTPlan<8> { using type = RadixList<8>; };
template <> struct FFTPlan<12> { using type = RadixList<4, 3>; };
template <> struct FFTPlan<16> { using type = RadixList<4, 4>; };
template <> struct FFTPlan<24> { using type = RadixList<8, 3>; };
template <> struct FFTPlan<32> { using type = RadixList<8, 4>; };
template <> struct FFTPlan<48> { using type = RadixList<8, 2, 3>; };
template <> struct FFTPlan<64> { using type = RadixList<8, 8>; };
template <> struct FFTPlan<96> { using type = RadixList<8, 4, 3>; };

// One in-place radix-RAD stage over NP planes of N rows of length N.  Element (row, i) of
// plane p sits at s[p * ps + row * rs + i * es].  NT threads cooperate; all must call this.
template <typename C, int N, int RAD, int LSPAN, int NT, bool INV, int NP>
__device__ __forceinline__ void fft_stage(C* s, int rs, int es, int ps, const C* tw) {
  constexpr int MP = N / (LSPAN * RAD);
  constexpr int NBR = N / RAD;            // butterflies per row
  constexpr int NBF = NP * N * NBR;       // butterflies in the pass
  constexpr int PER = (NBF + NT - 1) / NT;
  C v[PER][RAD];
  int offv[PER], jv[PER], kv[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int b = threadIdx.x + u * NT;
    offv[u] = -1;
    if ((NBF % NT) == 0 || b < NBF) {
      // rows vary fastest across threads: a warp touches 32 different rows at the same
      // position, which with the odd row pitch is free of shared-memory bank conflicts
      const int bb = b / (NP * N), rowp = b - bb * (NP * N);
      const int plane = rowp / N, row = rowp - plane * N;
      const int j = bb / MP, kp = bb - j * MP;
      offv[u] = plane * ps + row * rs;
      jv[u] = j; kv[u] = kp;
      const C* base = s + offv[u];
#pragma unroll
      for (int q = 0; q < RAD; ++q) {
        C x = base[(j * MP * RAD + kp + MP * q) * es];
        if (LSPAN > 1 && q > 0) {
          C w = tw[j * q * MP];
          if (INV) w.y = -w.y;
          x = cmul(x, w);
        }
        v[u][q] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    if (offv[u] >= 0) {
      SmallDFT<C, RAD, INV>::run(v[u]);
      C* base = s + offv[u];
#pragma unroll
      for (int p = 0; p < RAD; ++p) base[((jv[u] + LSPAN * p) * MP + kv[u]) * es] = v[u][p];
    }
  }
  __syncthreads();
}

template <typename C, int N, int NT, bool INV, int NP, int LSPAN, int R0, int... Rest>
__device__ __forceinline__ void fft_stages(C* s, int rs, int es, int ps, const C* tw) {
  fft_stage<C, N, R0, LSPAN, NT, INV, NP>(s, rs, es, ps, tw);
  if constexpr (sizeof...(Rest) > 0) fft_stages<C, N, NT, INV, NP, LSPAN * R0, Rest...>(s, rs, es, ps, tw);
}

template <typename C, int N, int NT, bool INV, int NP, int... Rs>
__device__ __forceinline__ void fft_pass_impl(C* s, int rs, int es, int ps, const C* tw, RadixList<Rs...>) {
  fft_stages<C, N, NT, INV, NP, 1, Rs...>(s, rs, es, ps, tw);
}

// Unnormalised length-N transform of the N rows of NP planes held in shared memory.
template <typename C, int N, int NT, bool INV, int NP = 1>
__device__ __forceinline__ void fft_pass(C* s, int rs, int es, const C* tw, int ps = 0) {
  fft_pass_impl<C, N, NT, INV, NP>(s, rs, es, ps, tw, typename FFTPlan<N>::type{});
}

// Copy an N x N plane between global memory (dense rows) and shared memory (odd row stride RS).
// Consecutive lanes take consecutive elements (8-byte accesses): with the odd pitch a 16-byte
// access per lane would hit shared memory at a 2-element stride and conflict 4 ways.
template <int N, int NT, int RS>
__device__ __forceinline__ void plane_load(float2* s, const float2* __restrict__ g) {
#pragma unroll 8
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    s[row * RS + col] = g[i];
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void plane_store(float2* __restrict__ g, const float2* s) {
#pragma unroll 8
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    g[i] = s[row * RS + col];
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void plane_load(double2* s, const double2* __restrict__ g) {
#pragma unroll 4
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    s[row * RS + col] = g[i];
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void plane_store(double2* __restrict__ g, const double2* s) {
#pragma unroll 4
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    g[i] = s[row * RS + col];
  }
}
// Strided variant for z slabs: row z of the slab starts at g + z * gstride (elements).  With an
// even pitch (RS = N, used by the z pass, whose FFT accesses are conflict-free for any pitch)
// 16-byte accesses are used on both sides; otherwise 8-byte accesses as in plane_load.
template <int N, int NT, int RS>
__device__ __forceinline__ void slab_load(float2* s, const float2* __restrict__ g, size_t gstride) {
  if constexpr (RS % 2 == 0) {
#pragma unroll 4
    for (int i = threadIdx.x; i < N * N / 2; i += NT) {
      const int idx = 2 * i, row = idx / N, col = idx - row * N;
      *reinterpret_cast<float4*>(s + row * RS + col) = *reinterpret_cast<const float4*>(g + row * gstride + col);
    }
  } else {
#pragma unroll 8
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int row = i / N, col = i - row * N;
      s[row * RS + col] = g[row * gstride + col];
    }
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void slab_store(float2* __restrict__ g, const float2* s, size_t gstride) {
  if constexpr (RS % 2 == 0) {
#pragma unroll 4
    for (int i = threadIdx.x; i < N * N / 2; i += NT) {
      const int idx = 2 * i, row = idx / N, col = idx - row * N;
      *reinterpret_cast<float4*>(g + row * gstride + col) = *reinterpret_cast<const float4*>(s + row * RS + col);
    }
  } else {
#pragma unroll 8
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int row = i / N, col = i - row * N;
      g[row * gstride + col] = s[row * RS + col];
    }
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void slab_load(double2* s, const double2* __restrict__ g, size_t gstride) {
#pragma unroll 4
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    s[row * RS + col] = g[row * gstride + col];
  }
}
template <int N, int NT, int RS>
__device__ __forceinline__ void slab_store(double2* __restrict__ g, const double2* s, size_t gstride) {
#pragma unroll 4
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int row = i / N, col = i - row * N;
    g[row * gstride + col] = s[row * RS + col];
  }
}

// ---------------------------------------------------------------------------- two-factor form
//
// A length-N line with N = R1 R2 is transformed by two register DFTs and one exchange through
// shared memory (Cooley-Tukey with n = n0 + R1 n1, K = K0 + R2 K1):
//     X[K0 + R2 K1] = sum_{n0} w_{R1}^{n0 K1} ( w_N^{n0 K0} sum_{n1} x[n0 + R1 n1] w_{R2}^{n1 K0} ).
// "A side": one work item per (line, n0) holds the R2 values x[n0 + R1 n1]; a DFT of length R2
// and the twiddle w_N^{n0 K0} give the exchange values E[K0][n0].  "B side": one item per
// (line, K0) holds E[K0][0..R1) and a DFT of length R1 gives X[K0 + R2 K1].  The inverse runs
// the same two steps backwards (B side first, conjugate twiddle), so a forward and an inverse
// transform share the exchange layout.  The first and last steps can read and write global
// memory directly, leaving one shared-memory round trip per axis.

template <typename C, bool INV> struct SmallDFT<C, 6, INV> {
  // 6 = 2 x 3: three-point DFTs over n1 (n = n0 + 2 n1), twiddle w6^{n0 k0}, two-point DFTs over n0
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.8660254037844386467637;  // sin(pi/3)
    C a[3] = {v[0], v[2], v[4]};
    C b[3] = {v[1], v[3], v[5]};
    SmallDFT<C, 3, INV>::run(a);
    SmallDFT<C, 3, INV>::run(b);
    const R sg = INV ? (R)1 : (R)-1;  // w6 = 1/2 + sg i h, w6^2 = -1/2 + sg i h
    const C b1 = cmul(b[1], cmake<C>((R)0.5, sg * h));
    const C b2 = cmul(b[2], cmake<C>((R)-0.5, sg * h));
    v[0] = cadd(a[0], b[0]); v[3] = csub(a[0], b[0]);
    v[1] = cadd(a[1], b1);   v[4] = csub(a[1], b1);
    v[2] = cadd(a[2], b2);   v[5] = csub(a[2], b2);
  }
};

template <typename C, bool INV> struct SmallDFT<C, 12, INV> {
  // 12 = 3 x 4 (n = 4 n1 + n2, k = k1 + 3 k2): three-point DFTs over n1 for each n2, twiddle
  // w12^{n2 k1}, four-point DFTs over n2 for each k1.
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.8660254037844386467637;  // sin(pi/3) = cos(pi/6)
    const R sg = INV ? (R)1 : (R)-1;          // w12^m = exp(sg i pi m / 6)
    C y[4][3];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2];
      y[n2][1] = v[n2 + 4];
      y[n2][2] = v[n2 + 8];
      SmallDFT<C, 3, INV>::run(y[n2]);
    }
    // twiddles w12^{n2 k1}: m = 1 (h, sg/2), 2 (1/2, sg h), 3 (0, sg), 4 (-1/2, sg h), 6 (-1, 0)
    y[1][1] = cmul(y[1][1], cmake<C>(h, sg * (R)0.5));
    y[1][2] = cmul(y[1][2], cmake<C>((R)0.5, sg * h));
    y[2][1] = cmul(y[2][1], cmake<C>((R)0.5, sg * h));
    y[2][2] = cmul(y[2][2], cmake<C>((R)-0.5, sg * h));
    y[3][1] = cmake<C>(-sg * y[3][1].y, sg * y[3][1].x);  // times sg i
    y[3][2] = cmake<C>(-y[3][2].x, -y[3][2].y);           // times -1
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      C u[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      SmallDFT<C, 4, INV>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 3 * k2] = u[k2];
    }
  }
};

template <int N> struct TwoFactor { static constexpr bool ok = false; };
template <> struct TwoFactor<16> { static constexpr bool ok = true; static constexpr int R1 = 4, R2 = 4; };
template <> struct TwoFactor<24> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 3; };
template <> struct TwoFactor<32> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 4; };
template <> struct TwoFactor<48> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 6; };
template <> struct TwoFactor<64> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 8; };
template <> struct TwoFactor<96> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 12; };

// Row pitch of a two-factor xy plane in shared memory: congruent to 8 modulo 16 elements, so that
// the in-row exchange (8 lanes per row, columns rotated by K0) and the column accesses are both
// free of bank conflicts.
template <int N> struct TFPitch { static constexpr int value = (N % 16 == 8) ? N : (N % 16 == 0 ? N + 8 : N + 1); };

// A side, forward: v[n1] = x[n0 + R1 n1] -> v[K0] = E[K0][n0].
template <typename C, int N, bool INV> struct TF;
template <typename C, int N> struct TF<C, N, false> {
  static constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  __device__ __forceinline__ static void a_side(C* v, int n0, const C* tw) {
    SmallDFT<C, R2, false>::run(v);
#pragma unroll
    for (int k0 = 1; k0 < R2; ++k0) v[k0] = cmul(v[k0], tw[k0 * n0]);
  }
  // B side, forward: u[n0] = E[K0][n0] -> u[K1] = X[K0 + R2 K1].
  __device__ __forceinline__ static void b_side(C* u, int, const C*) { SmallDFT<C, R1, false>::run(u); }
};
template <typename C, int N> struct TF<C, N, true> {
  static constexpr int R1 = TwoFactor<N>::R1, R2 = TwoFactor<N>::R2;
  // B side, inverse: u[K1] = X[K0 + R2 K1] -> u[n0] = E[K0][n0] (conjugate twiddle).
  __device__ __forceinline__ static void b_side(C* u, int k0, const C* tw) {
    SmallDFT<C, R1, true>::run(u);
#pragma unroll
    for (int n0 = 1; n0 < R1; ++n0) u[n0] = cmulc(u[n0], tw[k0 * n0]);
  }
  // A side, inverse: v[K0] = E[K0][n0] -> v[n1] = x[n0 + R1 n1].
  __device__ __forceinline__ static void a_side(C* v, int, const C*) { SmallDFT<C, R2, true>::run(v); }
};
