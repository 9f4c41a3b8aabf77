// Shared-memory batched FFT building blocks (sm_103a).
//
// A plane or slab of N x N complex values lives in shared memory with a padded row
// stride; each pass transforms N rows of length N in place.  Every stage of a
// mixed-radix (2, 3, 4) Stockham decomposition reads its butterflies into registers,
// synchronises the CTA, and writes them back in sorted order, so no second buffer is
// needed and the output is in natural order.
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

template <int... Rs> struct RadixList {};
template <int N> struct FFTPlan;
template <> struct FFTPlan<8> { using type = RadixList<4, 2>; };
template <> struct FFTPlan<12> { using type = RadixList<4, 3>; };
template <> struct FFTPlan<16> { using type = RadixList<4, 4>; };
template <> struct FFTPlan<24> { using type = RadixList<4, 3, 2>; };
template <> struct FFTPlan<32> { using type = RadixList<4, 4, 2>; };
template <> struct FFTPlan<48> { using type = RadixList<4, 4, 3>; };
template <> struct FFTPlan<64> { using type = RadixList<4, 4, 4>; };
template <> struct FFTPlan<96> { using type = RadixList<4, 4, 3, 2>; };

// One in-place radix-RAD stage over N rows of length N.  Element (row, i) sits at
// s[row * rs + i * es].  NT threads cooperate; all of them must call this.
template <typename C, int N, int RAD, int LSPAN, int NT, bool INV>
__device__ __forceinline__ void fft_stage(C* s, int rs, int es, const C* tw) {
  constexpr int MP = N / (LSPAN * RAD);
  constexpr int NBR = N / RAD;            // butterflies per row
  constexpr int NBF = N * NBR;            // butterflies in the pass
  constexpr int PER = (NBF + NT - 1) / NT;
  C v[PER][RAD];
  int rowv[PER], jv[PER], kv[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int b = threadIdx.x + u * NT;
    rowv[u] = -1;
    if ((NBF % NT) == 0 || b < NBF) {
      const int row = b / NBR, bb = b - row * NBR;
      const int j = bb / MP, kp = bb - j * MP;
      rowv[u] = row; jv[u] = j; kv[u] = kp;
      const C* base = s + row * rs;
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
    if (rowv[u] >= 0) {
      SmallDFT<C, RAD, INV>::run(v[u]);
      C* base = s + rowv[u] * rs;
#pragma unroll
      for (int p = 0; p < RAD; ++p) base[((jv[u] + LSPAN * p) * MP + kv[u]) * es] = v[u][p];
    }
  }
  __syncthreads();
}

template <typename C, int N, int NT, bool INV, int LSPAN, int R0, int... Rest>
__device__ __forceinline__ void fft_stages(C* s, int rs, int es, const C* tw) {
  fft_stage<C, N, R0, LSPAN, NT, INV>(s, rs, es, tw);
  if constexpr (sizeof...(Rest) > 0) fft_stages<C, N, NT, INV, LSPAN * R0, Rest...>(s, rs, es, tw);
}

template <typename C, int N, int NT, bool INV, int... Rs>
__device__ __forceinline__ void fft_pass_impl(C* s, int rs, int es, const C* tw, RadixList<Rs...>) {
  fft_stages<C, N, NT, INV, 1, Rs...>(s, rs, es, tw);
}

// Unnormalised length-N transform of N rows held in shared memory.
template <typename C, int N, int NT, bool INV>
__device__ __forceinline__ void fft_pass(C* s, int rs, int es, const C* tw) {
  fft_pass_impl<C, N, NT, INV>(s, rs, es, tw, typename FFTPlan<N>::type{});
}
