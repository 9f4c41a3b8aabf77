// Fused Chebyshev term kernel (sm_103a): inverse xy FFT of the kinetic part, the pointwise
// Hamiltonian (2x2 spin potential of Eq. potential4 and projector scatter of Eq. Vps) with the
// Chebyshev update, and the forward xy FFT of the new term, for one z-plane of one spinor.
#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"
#include "kepi.cuh"

namespace tddft {

// ============================================================================ fused term

template <int N> struct FusedThreads { static constexpr int value = (N >= 48) ? 512 : 256; };

// One z-plane of one spinor (both components) per CTA:
//   tmp (kinetic part, x/y still transformed) --inverse xy FFT--> T psi in shared memory,
//   + V psi + V_NL psi --> T_{k+1} = (2) (H - c)/Delta T_k (- T_{k-1}), accumulators updated,
//   T_{k+1} --forward xy FFT--> tmp, ready for the next term's z pass.
template <typename R, int N, int NLM>
__global__ void __launch_bounds__(FusedThreads<N>::value, FusedMinBlocks<R, N>::value)
k_fused_term(typename CT<R>::type* tmp, const typename CT<R>::type* Tk, const typename CT<R>::type* Tkm1,
             typename CT<R>::type* Tout, typename CT<R>::type* acc1, typename CT<R>::type* acc2,
             const R* __restrict__ V, size_t N3, ProjTables<R> pt, const typename CT<R>::type* __restrict__ dc,
             const typename CT<R>::type* __restrict__ twg, EpiParams ep, int do_fwd) {
  using C = typename CT<R>::type;
  constexpr int NT = FusedThreads<N>::value;
  constexpr int RS = N + 1;
  constexpr int PS = N * RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;  // planes: up at s, down at s + PS
  C* dcs = s + 2 * PS;  // this spinor's D c for every atom (when staged)
  const int z = blockIdx.x;
  const int kb = blockIdx.y;
  const int k = kb / ep.nstates;
  const size_t pu0 = (size_t)(2 * kb) * N3 + (size_t)z * N * N;  // up-plane offset
  const size_t pd0 = pu0 + N3;
  const int ncoef = pt.natoms * 2 * NLM;
  const C* dcg = dc + (size_t)kb * ncoef;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  if (ep.dc_staged)
    for (int i = threadIdx.x; i < ncoef; i += NT) dcs[i] = dcg[i];
  const C* dcb = ep.dc_staged ? dcs : dcg;
  plane_load<N, NT, RS>(s, tmp + pu0);
  plane_load<N, NT, RS>(s + PS, tmp + pd0);
  __syncthreads();
  fft_pass<C, N, NT, true, 2>(s, RS, 1, tw, PS);  // along x, both planes
  fft_pass<C, N, NT, true, 2>(s, 1, RS, tw, PS);  // along y, both planes
  const R sx = (R)ep.shift[k][0], sy = (R)ep.shift[k][1], sz = (R)ep.shift[k][2];
  const R cc = (R)ep.c, id = (R)ep.inv_delta;
  const bool first = ep.mode == EPI_FIRST;
  const R a0r = (R)ep.a0[0], a0i = (R)ep.a0[1], a1r = (R)ep.a1[0], a1i = (R)ep.a1[1];
  const R b0r = (R)ep.b0[0], b0i = (R)ep.b0[1], b1r = (R)ep.b1[0], b1i = (R)ep.b1[1];
  for (int i2 = threadIdx.x; i2 < N * N / 2; i2 += NT) {
    const int i = 2 * i2;
    const int y = i / N, x = i - y * N;
    const size_t r = (size_t)z * N * N + i;
    const Pair<C> pu = ld2(Tk + pu0 + i), pd = ld2(Tk + pd0 + i);
    C hu[2] = {s[y * RS + x], s[y * RS + x + 1]};
    C hd[2] = {s[PS + y * RS + x], s[PS + y * RS + x + 1]};
    const C pus[2] = {pu.a, pu.b}, pds[2] = {pd.a, pd.b};
    const C v0 = *reinterpret_cast<const C*>(V + r), v1 = *reinterpret_cast<const C*>(V + N3 + r);
    const C v2 = *reinterpret_cast<const C*>(V + 2 * N3 + r), v3 = *reinterpret_cast<const C*>(V + 3 * N3 + r);
    h_point<R, NLM>(hu[0], hd[0], pus[0], pds[0], v0.x, v1.x, (R)0.5 * v2.x, (R)0.5 * v3.x, r, pt, dcb, sx, sy, sz);
    h_point<R, NLM>(hu[1], hd[1], pus[1], pds[1], v0.y, v1.y, (R)0.5 * v2.y, (R)0.5 * v3.y, r + 1, pt, dcb, sx, sy,
                    sz);
    C tu[2], td[2];
    if (first) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        tu[j] = cmake<C>((hu[j].x - cc * pus[j].x) * id, (hu[j].y - cc * pus[j].y) * id);
        td[j] = cmake<C>((hd[j].x - cc * pds[j].x) * id, (hd[j].y - cc * pds[j].y) * id);
      }
    } else {
      const Pair<C> qu = ld2(Tkm1 + pu0 + i), qd = ld2(Tkm1 + pd0 + i);
      const C qus[2] = {qu.a, qu.b}, qds[2] = {qd.a, qd.b};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        tu[j] = cmake<C>((R)2 * (hu[j].x - cc * pus[j].x) * id - qus[j].x, (R)2 * (hu[j].y - cc * pus[j].y) * id - qus[j].y);
        td[j] = cmake<C>((R)2 * (hd[j].x - cc * pds[j].x) * id - qds[j].x, (R)2 * (hd[j].y - cc * pds[j].y) * id - qds[j].y);
      }
    }
    st2(Tout + pu0 + i, tu[0], tu[1]);
    st2(Tout + pd0 + i, td[0], td[1]);
    s[y * RS + x] = tu[0]; s[y * RS + x + 1] = tu[1];
    s[PS + y * RS + x] = td[0]; s[PS + y * RS + x + 1] = td[1];
    auto upd = [&](C* acc, R c0r, R c0i, R c1r, R c1i) {
      C nu[2], nd[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        nu[j] = cmake<C>(c1r * tu[j].x - c1i * tu[j].y, c1r * tu[j].y + c1i * tu[j].x);
        nd[j] = cmake<C>(c1r * td[j].x - c1i * td[j].y, c1r * td[j].y + c1i * td[j].x);
        if (first) {
          nu[j] = cadd(nu[j], cmake<C>(c0r * pus[j].x - c0i * pus[j].y, c0r * pus[j].y + c0i * pus[j].x));
          nd[j] = cadd(nd[j], cmake<C>(c0r * pds[j].x - c0i * pds[j].y, c0r * pds[j].y + c0i * pds[j].x));
        }
      }
      if (!first) {
        const Pair<C> au = ld2(acc + pu0 + i), ad = ld2(acc + pd0 + i);
        nu[0] = cadd(nu[0], au.a); nu[1] = cadd(nu[1], au.b);
        nd[0] = cadd(nd[0], ad.a); nd[1] = cadd(nd[1], ad.b);
      }
      st2(acc + pu0 + i, nu[0], nu[1]);
      st2(acc + pd0 + i, nd[0], nd[1]);
    };
    if (ep.use_acc1) upd(acc1, a0r, a0i, a1r, a1i);
    if (ep.use_acc2) upd(acc2, b0r, b0i, b1r, b1i);
  }
  if (!do_fwd) return;
  __syncthreads();
  fft_pass<C, N, NT, false, 2>(s, RS, 1, tw, PS);
  fft_pass<C, N, NT, false, 2>(s, 1, RS, tw, PS);
  plane_store<N, NT, RS>(tmp + pu0, s);
  plane_store<N, NT, RS>(tmp + pd0, s + PS);
}

template <typename R, int N, int NLM>
static cudaError_t fused_nn(cudaStream_t st, void* tmp, const void* Tk, const void* Tkm1, void* Tout, void* acc1,
                            void* acc2, const R* V, const ProjTables<R>& pt, const void* dc, int nkb, const void* tw,
                            const EpiParams& ep, int do_fwd) {
  using C = typename CT<R>::type;
  size_t smem = (size_t)(N + 2 * N * (N + 1)) * sizeof(C);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  // stage D c of every atom in shared memory when it is small next to the two planes
  EpiParams epx = ep;
  const size_t dcb = (size_t)pt.natoms * 2 * NLM * sizeof(C);
  epx.dc_staged = (NLM > 0 && pt.natoms > 0 && dcb <= 24 * 1024 && smem + dcb <= 227 * 1024) ? 1 : 0;
  if (epx.dc_staged) smem += dcb;
  auto kf = k_fused_term<R, N, NLM>;
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  const size_t N3 = (size_t)N * N * N;
  kf<<<dim3(N, nkb), FusedThreads<N>::value, smem, st>>>((C*)tmp, (const C*)Tk, (const C*)Tkm1, (C*)Tout, (C*)acc1,
                                                         (C*)acc2, V, N3, pt, (const C*)dc, (const C*)tw, epx, do_fwd);
  return cudaGetLastError();
}

template <typename R, int N>
static cudaError_t fused_n(cudaStream_t st, void* tmp, const void* Tk, const void* Tkm1, void* Tout, void* acc1,
                           void* acc2, const R* V, const ProjTables<R>& pt, const void* dc, int nkb, const void* tw,
                           const EpiParams& ep, int do_fwd) {
  const int nlm = pt.natoms > 0 ? pt.nlm : 0;
  switch (nlm) {
    case 0: return fused_nn<R, N, 0>(st, tmp, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, tw, ep, do_fwd);
    case 1: return fused_nn<R, N, 1>(st, tmp, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, tw, ep, do_fwd);
    case 4: return fused_nn<R, N, 4>(st, tmp, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, tw, ep, do_fwd);
    case 9: return fused_nn<R, N, 9>(st, tmp, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, tw, ep, do_fwd);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R> bool fused_supported(int N) {
  const size_t smem = (size_t)(N + 2 * N * (N + 1)) * sizeof(typename CT<R>::type);
  return smem <= 227 * 1024;
}

template <typename R>
cudaError_t launch_fused_term(cudaStream_t st, int N, void* tmp, const void* Tk, const void* Tkm1, void* Tout,
                              void* acc1, void* acc2, const R* V, const ProjTables<R>& pt, const void* dc, int nkb,
                              const void* tw, const EpiParams& ep, int do_fwd) {
  if (!fused_supported<R>(N)) return cudaErrorInvalidConfiguration;
  TDDFT_DISPATCH_N(N, (fused_n<R, NN>(st, tmp, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, tw, ep, do_fwd)));
}


#define TDDFT_FUSED_INST(R)                                                                                    \
  template cudaError_t launch_fused_term<R>(cudaStream_t, int, void*, const void*, const void*, void*, void*,   \
                                            void*, const R*, const ProjTables<R>&, const void*, int, const void*, \
                                            const EpiParams&, int);                                            \
  template bool fused_supported<R>(int);

TDDFT_FUSED_INST(float)
TDDFT_FUSED_INST(double)

}  // namespace tddft
