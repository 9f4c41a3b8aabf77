// The pointwise epilogue of one Chebyshev (or Taylor) term, for every spinor and grid point:
// kinetic part (from the FFT passes) + 2x2 spin-matrix local potential (Eq. potential4,
// Eq. zeeman_potential) + separable projector scatter with the L.S blocks (Eq. Vps, Eq.
// Vps-soc), then T_{k+1} = 2 (H - c)/Delta T_k - T_{k-1} and the accumulator updates; also the
// plain H apply, the Taylor update and the adjoint (Clenshaw-type) recurrence.
#include <cstdint>

#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"
#include "kepi.cuh"

namespace tddft {

// ============================================================================ epilogue

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Each thread takes two items: two neighbouring grid points of one spinor (SP = 0, 16-byte
// accesses) or one grid point of two spinors of one k-point (SP = 1, 8-byte accesses), whose
// projector scatter then walks the point's entries once for both.  The D c of the CTA's
// spinor(s) for every atom is staged in shared memory when it is small.
// AK selects the accumulator code compiled in: 0 = Chebyshev term without accumulator update,
// 1 = Chebyshev term updating accumulator 1 only, 2 = every mode with run-time flags.  The
// Chebyshev recurrence touches its accumulators on every third term only, so most launches take
// the AK = 0 form, which carries the least code.  FP32 forms are held to 64 registers (four
// CTAs per SM; the few bytes of spill in the AK = 1, 2 forms cost less than the lost occupancy).
template <typename R, int AK> struct EpiMinBlocks { static constexpr int value = 1; };
template <int AK> struct EpiMinBlocks<float, AK> { static constexpr int value = 4; };

template <typename R, int NLM, int AK, int SP>
__global__ void __launch_bounds__(256, EpiMinBlocks<R, AK>::value)
k_epilogue(const typename CT<R>::type* __restrict__ kin, const typename CT<R>::type* __restrict__ kin2,
           const typename CT<R>::type* Tk,
           const typename CT<R>::type* Tkm1, typename CT<R>::type* Tout, typename CT<R>::type* acc1,
           typename CT<R>::type* acc2, const R* __restrict__ V, size_t N3, ProjTables<R> pt,
           const typename CT<R>::type* __restrict__ dc, EpiParams ep) {
  using C = typename CT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* dcs = reinterpret_cast<C*>(smem_raw);
  const int kb = SP ? 2 * blockIdx.y : blockIdx.y;  // the (first) spinor
  const int k = kb / ep.nstates;
  const int ncoef = pt.natoms * 2 * NLM;
  const C* dcg = dc + (size_t)kb * ncoef;
  if (NLM > 0 && ep.dc_staged) {
    for (int i = threadIdx.x; i < (SP + 1) * ncoef; i += blockDim.x) dcs[i] = dcg[i];
    __syncthreads();
  }
  const C* dcb = (NLM > 0 && ep.dc_staged) ? dcs : dcg;
  const size_t r = (SP ? 1 : 2) * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (r >= N3) return;
  const size_t ou = (size_t)(2 * kb) * N3 + r, od = ou + N3;
  // the thread's two items of an array at offset o (up) or o + N3 (down)
  const size_t step = 2 * N3;
  auto ld = [&](const C* b, size_t o) -> Pair<C> {
    if constexpr (SP) return Pair<C>{b[o], b[o + step]};
    else return ld2(b + o);
  };
  auto st = [&](C* b, size_t o, C x, C y) {
    if constexpr (SP) { b[o] = x; b[o + step] = y; }
    else st2(b + o, x, y);
  };
  auto pf = [&](const C* b, size_t o) {
    prefetch_l2(b + o);
    if constexpr (SP) prefetch_l2(b + o + step);
  };
  const Pair<C> pu2 = ld(Tk, ou), pd2 = ld(Tk, od);
  Pair<C> ku2 = ld(kin, ou), kd2 = ld(kin, od);
  if (kin2) {  // V_NL psi from the tensor-core scatter, added to the kinetic part
    const Pair<C> vu = ld(kin2, ou), vd = ld(kin2, od);
    ku2 = {cadd(ku2.a, vu.a), cadd(ku2.b, vu.b)};
    kd2 = {cadd(kd2.a, vd.a), cadd(kd2.b, vd.b)};
  }
  // Chebyshev terms: every input is requested before any arithmetic (more loads in flight)
  const bool cheb = AK < 2 || ep.mode == EPI_RECUR || ep.mode == EPI_FIRST;
  const bool rec = ep.mode == EPI_RECUR;
  const bool use1 = AK >= 1 && ep.use_acc1, use2 = AK >= 2 && ep.use_acc2;
  const C zc = cmake<C>((R)0, (R)0);
  Pair<C> qu0 = {zc, zc}, qd0 = {zc, zc}, au1 = {zc, zc}, ad1 = {zc, zc}, au2 = {zc, zc}, ad2 = {zc, zc};
  // T_{k-1} and the accumulators are not needed until after the projector scatter: their
  // lines are requested from HBM into L2 now and read into registers after the scatter, so they
  // hold no registers across its loop.
  const bool ld_acc1 = cheb && use1 && !ep.init1, ld_acc2 = cheb && use2 && !ep.init2;
  if (rec) { pf(Tkm1, ou); pf(Tkm1, od); }
  if (ld_acc1) { pf(acc1, ou); pf(acc1, od); }
  if (ld_acc2) { pf(acc2, ou); pf(acc2, od); }
  const C pu[2] = {pu2.a, pu2.b}, pd[2] = {pd2.a, pd2.b};
  C hu[2] = {ku2.a, ku2.b}, hd[2] = {kd2.a, kd2.b};
  {
    const R sx = (R)ep.shift[k][0], sy = (R)ep.shift[k][1], sz = (R)ep.shift[k][2];
    if constexpr (SP) {
      const R v0 = V[r], v1 = V[N3 + r], v2 = V[2 * N3 + r], v3 = V[3 * N3 + r];
      h_point_2sp<R, NLM>(hu, hd, pu, pd, v0, v1, (R)0.5 * v2, (R)0.5 * v3, r, pt, dcb, dcb + ncoef, sx, sy, sz);
    } else {
      const C v0 = *reinterpret_cast<const C*>(V + r), v1 = *reinterpret_cast<const C*>(V + N3 + r);
      const C v2 = *reinterpret_cast<const C*>(V + 2 * N3 + r), v3 = *reinterpret_cast<const C*>(V + 3 * N3 + r);
      h_point<R, NLM>(hu[0], hd[0], pu[0], pd[0], v0.x, v1.x, (R)0.5 * v2.x, (R)0.5 * v3.x, r, pt, dcb, sx, sy, sz);
      h_point<R, NLM>(hu[1], hd[1], pu[1], pd[1], v0.y, v1.y, (R)0.5 * v2.y, (R)0.5 * v3.y, r + 1, pt, dcb, sx, sy, sz);
    }
  }
  if (rec) { qu0 = ld(Tkm1, ou); qd0 = ld(Tkm1, od); }
  if (ld_acc1) { au1 = ld(acc1, ou); ad1 = ld(acc1, od); }
  if (ld_acc2) { au2 = ld(acc2, ou); ad2 = ld(acc2, od); }
  auto cmulr = [](C a, R cr, R ci) { return cmake<C>(cr * a.x - ci * a.y, cr * a.y + ci * a.x); };
  // (x - c p) / Delta, and a times a complex series coefficient z; FP32 applies every constant as
  // a float pair hi + lo (split_constants), FP64 as it is
  auto shf = [&](R x, R p) -> R {
    if constexpr (sizeof(R) == 4) return shifted_f(x, p, ep.f_c, ep.f_id);
    else return (x - (R)ep.c * p) * (R)ep.inv_delta;
  };
  auto ccoef = [&](C a, const double* z, const float* zf) -> C {
    if constexpr (sizeof(R) == 4) return cmul_split(a, zf);
    else return cmulr(a, (R)z[0], (R)z[1]);
  };
  if (AK == 2 && ep.mode == EPI_APPLY) {
    st(Tout, ou, hu[0], hu[1]);
    st(Tout, od, hd[0], hd[1]);
    return;
  }
  if (AK == 2 && ep.mode == EPI_TAYLOR) {
    C tu[2], td[2];
    for (int j = 0; j < 2; ++j) { tu[j] = ccoef(hu[j], ep.a1, ep.f_a1); td[j] = ccoef(hd[j], ep.a1, ep.f_a1); }
    st(Tout, ou, tu[0], tu[1]);
    st(Tout, od, td[0], td[1]);
    const Pair<C> au = ld(acc1, ou), ad = ld(acc1, od);
    st(acc1, ou, cadd(au.a, tu[0]), cadd(au.b, tu[1]));
    st(acc1, od, cadd(ad.a, td[0]), cadd(ad.b, td[1]));
    return;
  }
  if (AK == 2 && (ep.mode == EPI_ADJ || ep.mode == EPI_ADJ0)) {
    // Clenshaw-type adjoint recurrence: S_k = f (H - c)/Delta S_{k+1} - S_{k+2} + seeds,
    // f = 2 (k >= 1) or 1 (k = 0); Tk holds S_{k+1}, Tkm1 holds S_{k+2} (may be null),
    // acc1/acc2 hold the seed cotangents with coefficients a1, b1.
    const R fct = (ep.mode == EPI_ADJ) ? (R)2 : (R)1;
    C su[2], sd[2];
    for (int j = 0; j < 2; ++j) {
      su[j] = cmake<C>(fct * shf(hu[j].x, pu[j].x), fct * shf(hu[j].y, pu[j].y));
      sd[j] = cmake<C>(fct * shf(hd[j].x, pd[j].x), fct * shf(hd[j].y, pd[j].y));
    }
    if (Tkm1) {
      const Pair<C> qu = ld(Tkm1, ou), qd = ld(Tkm1, od);
      su[0] = csub(su[0], qu.a); su[1] = csub(su[1], qu.b);
      sd[0] = csub(sd[0], qd.a); sd[1] = csub(sd[1], qd.b);
    }
    if (ep.use_acc1) {
      const Pair<C> yu = ld(acc1, ou), yd = ld(acc1, od);
      su[0] = cadd(su[0], ccoef(yu.a, ep.a1, ep.f_a1)); su[1] = cadd(su[1], ccoef(yu.b, ep.a1, ep.f_a1));
      sd[0] = cadd(sd[0], ccoef(yd.a, ep.a1, ep.f_a1)); sd[1] = cadd(sd[1], ccoef(yd.b, ep.a1, ep.f_a1));
    }
    if (ep.use_acc2) {
      const Pair<C> yu = ld(acc2, ou), yd = ld(acc2, od);
      su[0] = cadd(su[0], ccoef(yu.a, ep.b1, ep.f_b1)); su[1] = cadd(su[1], ccoef(yu.b, ep.b1, ep.f_b1));
      sd[0] = cadd(sd[0], ccoef(yd.a, ep.b1, ep.f_b1)); sd[1] = cadd(sd[1], ccoef(yd.b, ep.b1, ep.f_b1));
    }
    st(Tout, ou, su[0], su[1]);
    st(Tout, od, sd[0], sd[1]);
    return;
  }
  const bool first = ep.mode == EPI_FIRST;
  C tu[2], td[2];
  if (first) {
    for (int j = 0; j < 2; ++j) {
      tu[j] = cmake<C>(shf(hu[j].x, pu[j].x), shf(hu[j].y, pu[j].y));
      td[j] = cmake<C>(shf(hd[j].x, pd[j].x), shf(hd[j].y, pd[j].y));
    }
  } else {
    const C qus[2] = {qu0.a, qu0.b}, qds[2] = {qd0.a, qd0.b};
    for (int j = 0; j < 2; ++j) {
      tu[j] = cmake<C>((R)2 * shf(hu[j].x, pu[j].x) - qus[j].x, (R)2 * shf(hu[j].y, pu[j].y) - qus[j].y);
      td[j] = cmake<C>((R)2 * shf(hd[j].x, pd[j].x) - qds[j].x, (R)2 * shf(hd[j].y, pd[j].y) - qds[j].y);
    }
  }
  st(Tout, ou, tu[0], tu[1]);
  st(Tout, od, td[0], td[1]);
  // Accumulators take up to three terms at once (T_{k-1}, T_k, T_{k+1}, all in registers here),
  // so the host updates each of them on every third term only.
  auto upd = [&](C* acc, int init, const Pair<C>& au, const Pair<C>& ad, const double* cm, const float* cmf,
                 const double* c0, const float* c0f, const double* c1, const float* c1f) {
    const C qus[2] = {qu0.a, qu0.b}, qds[2] = {qd0.a, qd0.b};
    C nu[2], nd[2];
    if constexpr (sizeof(R) == 4) {
      // float-float update, rounded once (ff_cmadd)
      const C aus[2] = {au.a, au.b}, ads[2] = {ad.a, ad.b};
      const C z2 = cmake<C>(0.f, 0.f);
      for (int j = 0; j < 2; ++j) {
        C hu2 = init ? z2 : aus[j], hd2 = init ? z2 : ads[j], lu = z2, ld = z2;
        ff_cmadd(hu2, lu, tu[j], c1f);
        ff_cmadd(hd2, ld, td[j], c1f);
        ff_cmadd(hu2, lu, pu[j], c0f);
        ff_cmadd(hd2, ld, pd[j], c0f);
        if (rec) {
          ff_cmadd(hu2, lu, qus[j], cmf);
          ff_cmadd(hd2, ld, qds[j], cmf);
        }
        nu[j] = cadd(hu2, lu);
        nd[j] = cadd(hd2, ld);
      }
    } else {
      for (int j = 0; j < 2; ++j) {
        nu[j] = cadd(ccoef(tu[j], c1, c1f), ccoef(pu[j], c0, c0f));
        nd[j] = cadd(ccoef(td[j], c1, c1f), ccoef(pd[j], c0, c0f));
        if (rec) {
          nu[j] = cadd(nu[j], ccoef(qus[j], cm, cmf));
          nd[j] = cadd(nd[j], ccoef(qds[j], cm, cmf));
        }
      }
      if (!init) {
        nu[0] = cadd(nu[0], au.a); nu[1] = cadd(nu[1], au.b);
        nd[0] = cadd(nd[0], ad.a); nd[1] = cadd(nd[1], ad.b);
      }
    }
    st(acc, ou, nu[0], nu[1]);
    st(acc, od, nd[0], nd[1]);
  };
  if (use1) upd(acc1, ep.init1, au1, ad1, ep.am, ep.f_am, ep.a0, ep.f_a0, ep.a1, ep.f_a1);
  if (use2) upd(acc2, ep.init2, au2, ad2, ep.bm, ep.f_bm, ep.b0, ep.f_b0, ep.b1, ep.f_b1);
}

template <typename R, int NLM, int SP, typename... A>
static void epi_ak(int ak, dim3 grid, size_t smem, cudaStream_t st, A... args) {
  if (ak == 0) k_epilogue<R, NLM, 0, SP><<<grid, 256, smem, st>>>(args...);
  else if (ak == 1) k_epilogue<R, NLM, 1, SP><<<grid, 256, smem, st>>>(args...);
  else k_epilogue<R, NLM, 2, SP><<<grid, 256, smem, st>>>(args...);
}
template <typename R, int NLM, typename... A>
static void epi_sp(bool sp, int ak, dim3 grid, size_t smem, cudaStream_t st, A... args) {
  if (sp) epi_ak<R, NLM, 1>(ak, grid, smem, st, args...);
  else epi_ak<R, NLM, 0>(ak, grid, smem, st, args...);
}

template <typename R>
cudaError_t launch_epilogue(cudaStream_t st, int N, const void* kin, const void* kin2, const void* Tk, const void* Tkm1,
                            void* Tout, void* acc1, void* acc2, const R* V, const ProjTables<R>& pt, const void* dc,
                            int nkb, const EpiParams& ep) {
  using C = typename CT<R>::type;
  const size_t N3 = (size_t)N * N * N;
  // spinor pairs need an even number of states, so that a pair shares its k-point
  const bool sp = ep.spinor_pairs && ep.nstates % 2 == 0 && nkb % 2 == 0;
  dim3 grid((unsigned)(sp ? (N3 + 255) / 256 : (N3 / 2 + 255) / 256), sp ? nkb / 2 : nkb);
  const int nlm = pt.natoms > 0 ? pt.nlm : 0;
  EpiParams epx = ep;
  split_constants(epx);
  const size_t dcb = (size_t)pt.natoms * 2 * nlm * sizeof(C) * (sp ? 2 : 1);
  epx.dc_staged = (nlm > 0 && dcb <= 32 * 1024) ? 1 : 0;
  const size_t smem = epx.dc_staged ? dcb : 0;
  const bool cheb = ep.mode == EPI_FIRST || ep.mode == EPI_RECUR;
  const int ak = !cheb ? 2 : (ep.use_acc2 ? 2 : (ep.use_acc1 ? 1 : 0));
#define EPI_ARGS (const C*)kin, (const C*)kin2, (const C*)Tk, (const C*)Tkm1, (C*)Tout, (C*)acc1, (C*)acc2, V, N3, pt, (const C*)dc, epx
  switch (nlm) {
    case 0: epi_sp<R, 0>(sp, ak, grid, smem, st, EPI_ARGS); break;
    case 1: epi_sp<R, 1>(sp, ak, grid, smem, st, EPI_ARGS); break;
    case 4: epi_sp<R, 4>(sp, ak, grid, smem, st, EPI_ARGS); break;
    case 9: epi_sp<R, 9>(sp, ak, grid, smem, st, EPI_ARGS); break;
    default: return cudaErrorInvalidValue;
  }
#undef EPI_ARGS
  return cudaGetLastError();
}


#define TDDFT_EPI_INST(R)                                                                                       \
  template cudaError_t launch_epilogue<R>(cudaStream_t, int, const void*, const void*, const void*, const void*,  \
                                          void*, void*, void*, const R*, const ProjTables<R>&, const void*, int, \
                                          const EpiParams&);

TDDFT_EPI_INST(float)
TDDFT_EPI_INST(double)

}  // namespace tddft
