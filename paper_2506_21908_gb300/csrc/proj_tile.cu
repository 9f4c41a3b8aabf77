// Tile-centric projector contraction on the tensor cores (tcgen05), FP32-mixed path.
//
// The grid is cut into bricks of BX x 8 x 8 points (BX = 32 or 16).  For one brick b, every atom
// image whose projector sphere reaches into the brick is a "slot" (at most 256 / nlm of them).
// With q = k + A(t) and the brick origin r_b, the projector phase of Eq. Vps in velocity gauge
// factorises as exp(i q.d) = exp(i q.(r - r_b)) exp(i q.delta), delta = r_b - R_image, so with the
// real projector values beta_{slot,p}(r) (zero outside the sphere):
//
//   gather   c[s,a,p] = dV sum_{b, slot of a} exp(i q.delta) sum_{r in b} beta_{slot,p}(r) psi'_s(r),
//            psi'_s(r) = exp(i q.(r - r_b)) psi_s(r);
//   scatter  (V_NL psi)_s(r) = exp(-i q.(r - r_b)) sum_{slot,p} beta_{slot,p}(r) X_s[slot,p],
//            X_s[slot,p] = exp(-i q.delta) (D c)[s, a_slot, p].
//
// Both inner sums are dense real products over one brick: the gather is [64 components x (re, im)]
// x [brick points] x [slots x nlm], read psi once per brick; the scatter is [128 points] x
// [slots x nlm] x [components x (re, im)].  The real projector values of every brick are built
// once at creation in FP64 and stored in the operand layout of the tensor cores (K-major, rows of
// 128 bytes with the 128-byte swizzle), as one rounded part (TF32) or as hi + lo parts (TF32 x3,
// BF16 x3, FP16 x3: hi*hi + hi*lo + lo*hi with FP32 accumulation, the split-precision product).
//
// Each CTA (320 threads): warps 0-7 stage psi (phase, split, swizzled stores) or X and drain the
// tensor memory, warp 8 issues the MMAs (one elected thread), warp 9 the bulk copies of the
// projector tables; two shared-memory stages between them, full / empty mbarriers.  Every
// mbarrier wait has an iteration limit: on expiry the CTA sets bit 1 of the error word, stops
// issuing work, waits (with a limit) for its copies and MMAs in flight and frees its tensor memory.
#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bulk.cuh"
#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"

namespace tddft {

namespace {

constexpr int PT_ROWB = 128;        // bytes per operand row
constexpr int PT_PART = 128 * PT_ROWB;  // one 128-row operand part (16 KB)
constexpr unsigned PT_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t sw128(uint32_t off) { return off ^ (((off >> 7) & 7u) << 4); }

// K-major operand, rows of 128 bytes with the 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (not used by swizzled K-major operands)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;            // descriptor version of this architecture family
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Element kinds: bytes per element, instruction descriptor type code.
template <int EK> struct Elt;
template <> struct Elt<TILE_TF32> { static constexpr int bytes = 4, code = 2; };
template <> struct Elt<TILE_BF16> { static constexpr int bytes = 2, code = 1; };
template <> struct Elt<TILE_F16> { static constexpr int bytes = 2, code = 0; };

// D = F32, A = B of kind EK, both K-major, M = 128, N.
template <int EK> __device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | ((uint32_t)Elt<EK>::code << 7) | ((uint32_t)Elt<EK>::code << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int EK>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  if constexpr (EK == TILE_TF32)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool pt_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < PT_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void pt_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// Split x into the rounded part(s) of kind EK (hi, and lo = x - hi for the split product).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <int EK> struct Split;
template <> struct Split<TILE_TF32> {
  __device__ __forceinline__ static void two(float x, uint32_t& hi, uint32_t& lo) {
    const float h = tf32_rna(x);
    hi = __float_as_uint(h);
    lo = __float_as_uint(tf32_rna(x - h));
  }
};
template <> struct Split<TILE_BF16> {
  __device__ __forceinline__ static void two(float x, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
};
template <> struct Split<TILE_F16> {
  __device__ __forceinline__ static void two(float x, uint32_t& hi, uint32_t& lo) {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
};

// Store element k of row `row` of a swizzled operand part (k within the 128-byte row).
template <int EK> __device__ __forceinline__ void put(unsigned char* part, int row, int k, uint32_t v) {
  const uint32_t off = sw128((uint32_t)row * PT_ROWB + (uint32_t)(k * Elt<EK>::bytes));
  if constexpr (Elt<EK>::bytes == 4) *reinterpret_cast<uint32_t*>(part + off) = v;
  else *reinterpret_cast<uint16_t*>(part + off) = (uint16_t)v;
}

// 16 consecutive columns of the thread's lane, without the wait for completion.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// After tmem_wait_ld: ties the loaded registers to a point after the wait, so that no use of them
// is scheduled before it.
__device__ __forceinline__ void tmem_regs_ready(uint32_t* r) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
               "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Per-axis phase tables exp(+i q_a l h_a) of one brick (l = 0 .. extent-1).
__device__ __forceinline__ void phase_tables(float2* px, float2* py, float2* pz, int BX, const TileDev& td,
                                             const double* q) {
  for (int i = threadIdx.x; i < BX + 16; i += blockDim.x) {
    float s, c;
    if (i < BX) {
      sincosf((float)(q[0] * td.h[0] * i), &s, &c);
      px[i] = make_float2(c, s);
    } else if (i < BX + 8) {
      sincosf((float)(q[1] * td.h[1] * (i - BX)), &s, &c);
      py[i - BX] = make_float2(c, s);
    } else {
      sincosf((float)(q[2] * td.h[2] * (i - BX - 8)), &s, &c);
      pz[i - BX - 8] = make_float2(c, s);
    }
  }
}

__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

}  // namespace

// Two neighbouring values a, b (elements k, k + 1) as packed 16-bit hi and lo pairs.
template <int EK> struct Split2;
template <> struct Split2<TILE_F16> {
  __device__ __forceinline__ static void two(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
};
template <> struct Split2<TILE_BF16> {
  __device__ __forceinline__ static void two(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
};

constexpr int PT_WARPS = 8;                   // worker warps
constexpr int PT_NT = 32 * (PT_WARPS + 2);    // + MMA warp + copy warp
constexpr int PT_MMA_WARP = PT_WARPS, PT_COPY_WARP = PT_WARPS + 1;

// ============================================================================ gather

// Chunks per accumulation group of the gather.  The tensor cores add each product into the FP32
// accumulator with a rounding that is biased toward zero, so one accumulator that takes every
// chunk of a brick (hundreds of MMAs) loses a relative 1e-5 of every partial sum, the same sign
// everywhere.  The accumulation therefore restarts from zero every CPG chunks: group 0 accumulates
// in the running sum R (tensor-memory columns 256..511), every later group in P (columns 0..255),
// and the worker warps add P into R on the CUDA cores (round to nearest) between groups; the bias
// falls with the length of a group.
template <int TERMS> struct GatherGroups { static constexpr int CPG = (TERMS == 3) ? 4 : 8; };

// CTA (kg, item): 64 components (group g of k-point k) against the slots of one brick.
template <int EK, int TERMS>
__global__ void __launch_bounds__(PT_NT, 1)
k_tile_gather(const float2* __restrict__ psi, int N, int comps_per_k, int groups, TileDev td, EpiParams ep,
              float* __restrict__ part, int* __restrict__ err) {
  constexpr int EPR = PT_ROWB / Elt<EK>::bytes;  // points per chunk (K elements per row)
  constexpr int NPART = (TERMS == 3) ? 2 : 1;
  constexpr int BPART = 256 * PT_ROWB;          // largest B part (N <= 256)
  constexpr int STAGE = NPART * (PT_PART + BPART);
  constexpr int CPW = 64 / PT_WARPS;            // components per worker warp
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int CPG = GatherGroups<TERMS>::CPG;
  __shared__ uint64_t bar_full[2], bar_empty[2], bar_acc, bar_grp, bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ float2 px[32], py[8], pz[8];

  // after a failed wait anywhere in the launch the remaining CTAs do nothing (the call reports it)
  if (*reinterpret_cast<volatile int*>(err) & 1) return;
  const int kg = blockIdx.x, it = blockIdx.y;
  const int k = kg / groups, comp0 = (kg % groups) * 64;
  const int nslot = td.it_nslot[it], npad = td.it_npad[it];
  if (nslot == 0) return;  // a brick no projector sphere reaches
  const int BX = td.BX;
  const int brick = td.it_brick[it];
  const int bx = brick % td.nbx, by = (brick / td.nbx) % td.nby, bz = brick / (td.nbx * td.nby);
  const int x0 = bx * BX, y0 = by * 8, z0 = bz * 8;
  const int nch = BX * 64 / EPR;
  const int ngrp = nch / CPG;  // nch is a multiple of 16 and of CPG, so ngrp >= 2
  const size_t N3 = (size_t)N * N * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto stageA = [&](int s, int q) { return smem + (size_t)s * STAGE + (size_t)q * PT_PART; };
  auto stageB = [&](int s, int q) { return smem + (size_t)s * STAGE + (size_t)NPART * PT_PART + (size_t)q * BPART; };

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < 2; ++s) {
      bar_init(sm_addr(&bar_full[s]), 32 * PT_WARPS + 1);
      bar_init(sm_addr(&bar_empty[s]), 1);
    }
    bar_init(sm_addr(&bar_acc), 1);
    bar_init(sm_addr(&bar_grp), 1);
    bar_init(sm_addr(&bar_drain), 32 * PT_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  phase_tables(px, py, pz, BX, td, ep.shift[k]);
  if (warp == PT_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t accP = tmem, accR = tmem + 256u;
  // worker warp: lane quarter of the accumulator, and which alternate blocks of 16 columns it takes
  const int quarter = warp & 3, half = (warp >> 2) & 1;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;

  if (warp < PT_WARPS) {
    // ---- psi' = exp(i q.(r - r_b)) psi, split, into rows cl (re) and 64 + cl (im) of stage A.
    constexpr int PPL = (EPR == 64) ? 2 : 1;  // points per lane
    using V = typename std::conditional<PPL == 2, float4, float2>::type;
    const int kk = lane * PPL;
    const float2* base0 = psi + ((size_t)k * comps_per_k + comp0 + warp * CPW) * N3;
    const int nvalid = min(CPW, comps_per_k - comp0 - warp * CPW);
    auto point = [&](int c, int& lx, int& ly, int& lz) -> size_t {
      const int p = c * EPR + kk;
      lx = p % BX;
      ly = (p / BX) & 7;
      lz = p / (BX * 8);
      return ((size_t)(z0 + lz) * N + (y0 + ly)) * N + (x0 + lx);
    };
    auto load = [&](int c, V* w) {
      int lx, ly, lz;
      const size_t idx = point(c, lx, ly, lz);
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        V v;
        if constexpr (PPL == 2) v = make_float4(0.f, 0.f, 0.f, 0.f);
        else v = make_float2(0.f, 0.f);
        if (j < nvalid) v = __ldg(reinterpret_cast<const V*>(base0 + (size_t)j * N3 + idx));
        w[j] = v;
      }
    };
    // loads run two chunks ahead of the conversion: chunk c + 2 is requested before chunk c is
    // converted (wa: chunk c, wb: c + 1, wc: c + 2)
    V wa[CPW], wb[CPW], wc[CPW];
    load(0, wa);
    if (nch > 1) load(1, wb);
    for (int c = 0; c < nch; ++c) {
      const int s = c & 1;
      if (c + 2 < nch) load(c + 2, wc);
      if (c >= 2 && !pt_wait(sm_addr(&bar_empty[s]), ((c >> 1) - 1) & 1)) abort_flag = 1;
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      int lx, ly, lz;
      point(c, lx, ly, lz);
      const float2 ph0 = cm(cm(px[lx], py[ly]), pz[lz]);
      const float2 ph1 = (PPL == 2) ? cm(cm(px[lx + 1], py[ly]), pz[lz]) : ph0;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int cl = warp * CPW + j;
        if constexpr (PPL == 2) {
          const float2 v0 = cm(make_float2(wa[j].x, wa[j].y), ph0);
          const float2 v1 = cm(make_float2(wa[j].z, wa[j].w), ph1);
          uint32_t rh, rl, ih, il;
          Split2<EK>::two(v0.x, v1.x, rh, rl);
          Split2<EK>::two(v0.y, v1.y, ih, il);
          const uint32_t ore = sw128((uint32_t)cl * PT_ROWB + (uint32_t)(kk * 2));
          const uint32_t oim = sw128((uint32_t)(64 + cl) * PT_ROWB + (uint32_t)(kk * 2));
          *reinterpret_cast<uint32_t*>(stageA(s, 0) + ore) = rh;
          *reinterpret_cast<uint32_t*>(stageA(s, 0) + oim) = ih;
          if constexpr (TERMS == 3) {
            *reinterpret_cast<uint32_t*>(stageA(s, 1) + ore) = rl;
            *reinterpret_cast<uint32_t*>(stageA(s, 1) + oim) = il;
          }
        } else {
          const float2 v0 = cm(make_float2(wa[j].x, wa[j].y), ph0);
          uint32_t rh, rl, ih, il;
          Split<EK>::two(v0.x, rh, rl);
          Split<EK>::two(v0.y, ih, il);
          put<EK>(stageA(s, 0), cl, kk, rh);
          put<EK>(stageA(s, 0), 64 + cl, kk, ih);
          if constexpr (TERMS == 3) {
            put<EK>(stageA(s, 1), cl, kk, rl);
            put<EK>(stageA(s, 1), 64 + cl, kk, il);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      pt_arrive(sm_addr(&bar_full[s]));
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        wa[j] = wb[j];
        wb[j] = wc[j];
      }
      // group g (1 <= g <= ngrp - 2) ended with chunk c - 2: add P into R before the next pass of
      // this loop waits for the MMAs of the first chunk of group g + 1, which reuse P (the votes keep
      // the warp together for the tensor-memory accesses)
      const int gd = (c - 1) / CPG;
      if ((c - 1) % CPG == 0 && gd >= 2 && gd <= ngrp - 1) {
        if (!pt_wait(sm_addr(&bar_grp), (gd - 2) & 1)) abort_flag = 1;
        if (__any_sync(0xffffffffu, abort_flag != 0)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int c0 = 16 * half; c0 < npad; c0 += 32) {
          uint32_t pv[16], rv[16];
          tmem_ld16_async(accP + lane_off + (uint32_t)c0, pv);
          tmem_ld16_async(accR + lane_off + (uint32_t)c0, rv);
          tmem_wait_ld();
          tmem_regs_ready(pv);
          tmem_regs_ready(rv);
          float sum[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[j] = __uint_as_float(rv[j]) + __uint_as_float(pv[j]);
          tmem_st16(accR + lane_off + (uint32_t)c0, sum);
        }
        tmem_wait_st();
        asm volatile("tcgen05.fence::before_thread_sync;");
        pt_arrive(sm_addr(&bar_drain));
      }
    }
  } else if (warp == PT_COPY_WARP) {
    if (lane == 0) {
      // ---- projector values of the brick, chunk by chunk
      const unsigned char* src = td.g_tab + td.it_goff[it];
      const uint32_t pbytes = (uint32_t)npad * PT_ROWB;
      int issued = 0;
      for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        if (c >= 2 && !pt_wait(sm_addr(&bar_empty[s]), ((c >> 1) - 1) & 1)) abort_flag = 1;
        if (abort_flag) break;
        bulk_expect(sm_addr(&bar_full[s]), NPART * pbytes);
        for (int q = 0; q < NPART; ++q)
          bulk_copy(stageB(s, q), src + ((size_t)c * NPART + q) * pbytes, pbytes, sm_addr(&bar_full[s]));
        issued = c + 1;
      }
      // every copy issued has landed before the CTA moves on
      for (int c = (issued > 2 ? issued - 2 : 0); c < issued; ++c)
        if (!pt_wait(sm_addr(&bar_full[c & 1]), (c >> 1) & 1)) atomicOr(err, 1);
    }
  } else {
    if (lane == 0) {
      const uint32_t id = idesc<EK>(npad);
      for (int c = 0; c < nch; ++c) {
        const int s = c & 1, g = c / CPG, cg = c % CPG;
        // the first wait may be shortened by the testing hook: on expiry the error bit is set and
        // the wait is retried with the full limit
        if (c == 0 && !bulk_first_try(sm_addr(&bar_full[s]), 0)) atomicOr(err, 1);
        // P holds group g - 1 until the worker warps have added it into R
        if (cg == 0 && g >= 2 && !pt_wait(sm_addr(&bar_drain), (g - 2) & 1)) abort_flag = 1;
        if (!abort_flag && !pt_wait(sm_addr(&bar_full[s]), (c >> 1) & 1)) abort_flag = 1;
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dst = (g == 0) ? accR : accP;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t off = (uint32_t)ks * 32;
          const uint64_t ah = desc_sw128(sm_addr(stageA(s, 0)) + off), bh = desc_sw128(sm_addr(stageB(s, 0)) + off);
          mma<EK>(dst, ah, bh, id, (cg | ks) ? 1u : 0u);
          if constexpr (TERMS == 3) {
            const uint64_t al = desc_sw128(sm_addr(stageA(s, 1)) + off), bl = desc_sw128(sm_addr(stageB(s, 1)) + off);
            mma<EK>(dst, ah, bl, id, 1u);
            mma<EK>(dst, al, bh, id, 1u);
          }
        }
        mma_commit(sm_addr(&bar_empty[s]));
        // groups 1 .. ngrp - 2 are added into R by the worker warps; the last one at the end
        if (cg == CPG - 1 && g >= 1 && g <= ngrp - 2) mma_commit(sm_addr(&bar_grp));
      }
      // also after an abort: every MMA issued completes before the accumulator is read or freed
      mma_commit(sm_addr(&bar_acc));
      if (!pt_wait(sm_addr(&bar_acc), 0)) atomicOr(err, 1);
    }
  }
  // ---- R + P (the last group) (rows: component re / im; columns: slot x nlm) -> partial sums;
  // the two warps of a lane quarter take alternate blocks of 16 columns
  if (warp < PT_WARPS) {
    const bool ok = __all_sync(0xffffffffu, pt_wait(sm_addr(&bar_acc), 0));
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok || __any_sync(0xffffffffu, abort_flag != 0)) {
      if (lane == 0) atomicOr(err, 1);
    } else {
      const int row = quarter * 32 + lane;
      const int ncol = td.nlm * nslot;
      float* dst = part + (size_t)kg * td.part_layer + td.it_poff[it];
      for (int c0 = 16 * half; c0 < npad; c0 += 32) {
        uint32_t pv[16], rv[16];
        tmem_ld16_async(accP + lane_off + (uint32_t)c0, pv);
        tmem_ld16_async(accR + lane_off + (uint32_t)c0, rv);
        tmem_wait_ld();
        tmem_regs_ready(pv);
        tmem_regs_ready(rv);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < ncol) dst[(size_t)(c0 + j) * 128 + row] = __uint_as_float(rv[j]) + __uint_as_float(pv[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == PT_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Sum the partial products of every (brick, slot) of atom a in a fixed order with the phase
// exp(i q.delta), times dV: c[kb][a][2p + sigma]; then D c with the atom's block.
__global__ void __launch_bounds__(64)
k_tile_reduce(const float* __restrict__ part, TileDev td, int groups, int comps_per_k, int nstates, int natoms,
              float dV, EpiParams ep, const float* __restrict__ Dmat, float2* __restrict__ c_out,
              float2* __restrict__ dc_out) {
  const int a = blockIdx.x, kg = blockIdx.y;
  const int k = kg / groups, comp0 = (kg % groups) * 64;
  const int nlm = td.nlm;
  const int t = threadIdx.x;
  __shared__ float2 cs[64][kMaxNLM];
  float2 acc[kMaxNLM];
#pragma unroll
  for (int p = 0; p < kMaxNLM; ++p) acc[p] = make_float2(0.f, 0.f);
  const double* q = ep.shift[k];
  for (int e = td.a_ptr[a]; e < td.a_ptr[a + 1]; ++e) {
    const int it = td.a_item[e], sl = td.a_slot[e];
    const float4 dl = td.slot_delta[(size_t)it * td.smax + sl];
    float sn, cs_;
    sincosf((float)(q[0] * dl.x + q[1] * dl.y + q[2] * dl.z), &sn, &cs_);
    const float* src = part + (size_t)kg * td.part_layer + td.it_poff[it] + (size_t)sl * nlm * 128;
#pragma unroll
    for (int p = 0; p < kMaxNLM; ++p) {
      if (p < nlm) {
        const float re = src[(size_t)p * 128 + t], im = src[(size_t)p * 128 + 64 + t];
        acc[p].x += re * cs_ - im * sn;
        acc[p].y += re * sn + im * cs_;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kMaxNLM; ++p) cs[t][p] = make_float2(acc[p].x * dV, acc[p].y * dV);
  __syncthreads();
  const int comp = comp0 + t;
  if (comp >= comps_per_k) return;
  const int sp = comp >> 1, sig = comp & 1;     // spinor within k, spin component
  const int pair = t & ~1;                      // the spinor's two components in cs
  const size_t kb = (size_t)k * nstates + sp;
  const int M = 2 * nlm;
  const float* D = Dmat + (size_t)a * M * M * 2;
  for (int p = 0; p < nlm; ++p) {
    const int row = 2 * p + sig;
    float re = 0.f, im = 0.f;
    for (int u = 0; u < M; ++u) {
      const float2 cu = cs[pair + (u & 1)][u >> 1];
      const float dr = D[(row * M + u) * 2], di = D[(row * M + u) * 2 + 1];
      re += dr * cu.x - di * cu.y;
      im += dr * cu.y + di * cu.x;
    }
    const size_t o = (kb * natoms + a) * M + row;
    c_out[o] = cs[t][p];
    dc_out[o] = make_float2(re, im);
  }
}

// ============================================================================ scatter

// CTA (kg, brick): SC components (X, the B operand, resident) against the brick's points in
// tiles of 128 (the A operand, streamed).  FUSED = 0: out = exp(-i q.(r - r_b)) (beta^T X) at every
// point of a brick with projectors (the points of other bricks are never written and keep their
// zeros).  FUSED = 1: the drain runs the Chebyshev epilogue of every point of the brick itself
// (kinetic part from io.kin, V_NL from the tensor memory, the 2x2 local potential, T_{k+1} and the
// accumulators) with the arithmetic of k_epilogue, so V_NL never crosses HBM; bricks without
// projectors take the same path with V_NL = 0.
template <int EK, int TERMS, int FUSED>
__global__ void __launch_bounds__(PT_NT, 1)
k_tile_scatter(float2* out, int N, int comps_per_k, int sgroups, int nstates, int natoms, TileDev td, EpiParams ep,
               const float2* __restrict__ dc, int* __restrict__ err, EpiIO io) {
  constexpr int EPR = PT_ROWB / Elt<EK>::bytes;    // projector indices per K chunk
  constexpr int SC = (Elt<EK>::bytes == 4) ? 32 : 64;  // components per CTA
  constexpr int NPART = (TERMS == 3) ? 2 : 1;
  constexpr int XPART = 2 * SC * PT_ROWB;          // one K chunk of X (2 SC rows)
  constexpr int STAGE = NPART * PT_PART;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_full[2], bar_empty[2], bar_accf[2], bar_acce[2], bar_fin;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ float2 px[32], py[8], pz[8];
  __shared__ float2 sph[256];  // exp(-i q.delta) per slot (at most 256 / nlm slots)

  if (*reinterpret_cast<volatile int*>(err) & 1) return;
  const int kg = blockIdx.x, it = blockIdx.y;
  const int k = kg / sgroups, comp0 = (kg % sgroups) * SC;
  const int nslot = td.it_nslot[it], kch = td.it_kch[it];
  if (!FUSED && nslot == 0) return;  // nothing to add at this brick
  const bool has_nl = nslot > 0;
  const int BX = td.BX;
  const int brick = td.it_brick[it];
  const int bx = brick % td.nbx, by = (brick / td.nbx) % td.nby, bz = brick / (td.nbx * td.nby);
  const int x0 = bx * BX, y0 = by * 8, z0 = bz * 8;
  const int ntile = BX * 64 / 128;
  const size_t N3 = (size_t)N * N * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nlm = td.nlm;
  unsigned char* X = smem;                                          // [kch][NPART][XPART]
  unsigned char* A = smem + (size_t)kch * NPART * XPART;             // [2][NPART][PT_PART]
  auto xpart = [&](int kc, int q) { return X + ((size_t)kc * NPART + q) * XPART; };
  auto apart = [&](int s, int q) { return A + (size_t)s * STAGE + (size_t)q * PT_PART; };

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < 2; ++s) {
      bar_init(sm_addr(&bar_full[s]), 1);
      bar_init(sm_addr(&bar_empty[s]), 1);
      bar_init(sm_addr(&bar_accf[s]), 1);
      bar_init(sm_addr(&bar_acce[s]), 32 * PT_WARPS);
    }
    bar_init(sm_addr(&bar_fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  phase_tables(px, py, pz, BX, td, ep.shift[k]);
  const double* q = ep.shift[k];
  for (int s = threadIdx.x; s < nslot; s += blockDim.x) {
    const float4 dl = td.slot_delta[(size_t)it * td.smax + s];
    float sn, c;
    sincosf((float)(q[0] * dl.x + q[1] * dl.y + q[2] * dl.z), &sn, &c);
    sph[s] = make_float2(c, -sn);
  }
  // tensor memory: two accumulators of 2 SC columns (tiles alternate); with three products the
  // hi x lo and lo x hi products go to a second pair at column 256, so the rounding of the tensor
  // cores' accumulation (biased toward zero) sees a third of the MMAs at full magnitude
  constexpr uint32_t TMEM_COLS = (TERMS == 3) ? 512u : 256u;
  if (warp == PT_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // ---- X: rows cl (re) and SC + cl (im), K element j = slot * nlm + p.  One 16-byte load of D c
  // gives both spin components of one spinor at one projector (index 2 p + sigma).
  if (warp < PT_WARPS) {
    const int tid = threadIdx.x;
    constexpr int SPG = SC / 2;                    // spinors per CTA
    const int total = nslot * SPG * nlm;
    const float4* dc4 = reinterpret_cast<const float4*>(dc);
    for (int b0 = 0; b0 < total; b0 += 4 * 32 * PT_WARPS) {
      float4 f[4];
      int ee[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = b0 + u * 32 * PT_WARPS + tid;
        ee[u] = e;
        f[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < total) {
          const int p = e % nlm, sp = (e / nlm) % SPG, sl = e / (nlm * SPG);
          const int comp = comp0 + 2 * sp;
          if (comp < comps_per_k) {
            const int a = td.slot_atom[(size_t)it * td.smax + sl];
            const size_t kb = (size_t)k * nstates + (comp >> 1);
            f[u] = __ldg(dc4 + (kb * natoms + a) * nlm + p);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = ee[u];
        if (e >= total) continue;
        const int p = e % nlm, sp = (e / nlm) % SPG, sl = e / (nlm * SPG);
        const int j = sl * nlm + p, kc = j / EPR, el = j % EPR;
        const float2 x0v = cm(make_float2(f[u].x, f[u].y), sph[sl]);
        const float2 x1v = cm(make_float2(f[u].z, f[u].w), sph[sl]);
        const float vals[4] = {x0v.x, x0v.y, x1v.x, x1v.y};
        const int rows[4] = {2 * sp, SC + 2 * sp, 2 * sp + 1, SC + 2 * sp + 1};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          uint32_t hi, lo;
          Split<EK>::two(vals[r], hi, lo);
          put<EK>(xpart(kc, 0), rows[r], el, hi);
          if constexpr (TERMS == 3) put<EK>(xpart(kc, 1), rows[r], el, lo);
        }
      }
    }
    // padding of the last K chunk
    const int j0 = nslot * nlm, pad = kch * EPR - j0;
    for (int i = tid; i < pad * 2 * SC; i += 32 * PT_WARPS) {
      const int row = i % (2 * SC), j = j0 + i / (2 * SC);
      put<EK>(xpart(j / EPR, 0), row, j % EPR, 0u);
      if constexpr (TERMS == 3) put<EK>(xpart(j / EPR, 1), row, j % EPR, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const int nchunk = ntile * kch;
  if (warp == PT_COPY_WARP) {
    if (lane == 0 && has_nl) {
      const unsigned char* src = td.s_tab + td.it_soff[it];
      int issued = 0;
      for (int j = 0; j < nchunk; ++j) {
        const int s = j & 1;
        if (j >= 2 && !pt_wait(sm_addr(&bar_empty[s]), ((j >> 1) - 1) & 1)) abort_flag = 1;
        if (abort_flag) break;
        bulk_expect(sm_addr(&bar_full[s]), NPART * PT_PART);
        for (int qq = 0; qq < NPART; ++qq)
          bulk_copy(apart(s, qq), src + ((size_t)j * NPART + qq) * PT_PART, PT_PART, sm_addr(&bar_full[s]));
        issued = j + 1;
      }
      for (int j = (issued > 2 ? issued - 2 : 0); j < issued; ++j)
        if (!pt_wait(sm_addr(&bar_full[j & 1]), (j >> 1) & 1)) atomicOr(err, 1);
    }
  } else if (warp == PT_MMA_WARP) {
    if (lane == 0 && has_nl) {
      const uint32_t id = idesc<EK>(2 * SC);
      for (int t = 0; t < ntile && !abort_flag; ++t) {
        const int acc = t & 1;
        if (t >= 2 && !pt_wait(sm_addr(&bar_acce[acc]), ((t >> 1) - 1) & 1)) { abort_flag = 1; break; }
        const uint32_t dtm = tmem + (uint32_t)(acc * 2 * SC), dlo = dtm + 256u;
        for (int kc = 0; kc < kch; ++kc) {
          const int j = t * kch + kc, s = j & 1;
          if (!pt_wait(sm_addr(&bar_full[s]), (j >> 1) & 1)) { abort_flag = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t off = (uint32_t)ks * 32;
            const uint64_t ah = desc_sw128(sm_addr(apart(s, 0)) + off), bh = desc_sw128(sm_addr(xpart(kc, 0)) + off);
            mma<EK>(dtm, ah, bh, id, (kc | ks) ? 1u : 0u);
            if constexpr (TERMS == 3) {
              const uint64_t al = desc_sw128(sm_addr(apart(s, 1)) + off), bl = desc_sw128(sm_addr(xpart(kc, 1)) + off);
              mma<EK>(dlo, ah, bl, id, (kc | ks) ? 1u : 0u);
              mma<EK>(dlo, al, bh, id, 1u);
            }
          }
          mma_commit(sm_addr(&bar_empty[s]));
        }
        if (abort_flag) break;
        mma_commit(sm_addr(&bar_accf[acc]));
      }
      // every MMA issued has completed before the tensor memory is released
      mma_commit(sm_addr(&bar_fin));
      if (!pt_wait(sm_addr(&bar_fin), 0)) atomicOr(err, 1);
    }
  } else {
    // ---- drain: thread = point of the tile (lane quarter of the warp); the two warps of a
    // quarter take one half of the components each; V_NL = exp(-i q.(r - r_b)) (re + i im)
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const int cbeg = half * (SC / 2), cend = (half + 1) * (SC / 2);
    // epilogue constants (Chebyshev term k: T_{k+1} = f (H - c) T_k / Delta - T_{k-1}, f = 1 or 2)
    const bool rec = ep.mode == EPI_RECUR;
    const bool use1 = ep.use_acc1, use2 = ep.use_acc2;
    const bool ld1 = use1 && !ep.init1, ld2 = use2 && !ep.init2;
    for (int t = 0; t < ntile; ++t) {
      const int acc = t & 1;
      if (has_nl) {
        if (!pt_wait(sm_addr(&bar_accf[acc]), (t >> 1) & 1)) abort_flag = 1;
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      const int p = t * 128 + row;
      const int lx = p % BX, ly = (p / BX) & 7, lz = p / (BX * 8);
      const size_t idx = ((size_t)(z0 + lz) * N + (y0 + ly)) * N + (x0 + lx);
      const float2 ph = cm(cm(px[lx], py[ly]), pz[lz]);
      const float2 phc = make_float2(ph.x, -ph.y);
      const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 2 * SC);
      const size_t base = ((size_t)k * comps_per_k + comp0) * N3 + idx;  // component comp0 at this point
      float V0 = 0.f, V1 = 0.f, hx = 0.f, hy = 0.f;
      if constexpr (FUSED) {
        V0 = io.V[idx];
        V1 = io.V[N3 + idx];
        hx = 0.5f * io.V[2 * N3 + idx];
        hy = 0.5f * io.V[3 * N3 + idx];
      }
      for (int c0 = cbeg; c0 < cend; c0 += 16) {
        float re[16], im[16];
        if (has_nl) {
          uint32_t hr[16], hi_[16];
          tmem_ld16_async(tb + (uint32_t)c0, hr);
          tmem_ld16_async(tb + (uint32_t)(SC + c0), hi_);
          if constexpr (TERMS == 3) {
            uint32_t lr[16], li[16];
            tmem_ld16_async(tb + 256u + (uint32_t)c0, lr);
            tmem_ld16_async(tb + 256u + (uint32_t)(SC + c0), li);
            tmem_wait_ld();
            tmem_regs_ready(hr);
            tmem_regs_ready(hi_);
            tmem_regs_ready(lr);
            tmem_regs_ready(li);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              re[j] = __uint_as_float(hr[j]) + __uint_as_float(lr[j]);
              im[j] = __uint_as_float(hi_[j]) + __uint_as_float(li[j]);
            }
          } else {
            tmem_wait_ld();
            tmem_regs_ready(hr);
            tmem_regs_ready(hi_);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              re[j] = __uint_as_float(hr[j]);
              im[j] = __uint_as_float(hi_[j]);
            }
          }
          if (c0 + 16 >= cend) {
            asm volatile("tcgen05.fence::before_thread_sync;");
            pt_arrive(sm_addr(&bar_acce[acc]));
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) re[j] = im[j] = 0.f;
        }
        if constexpr (!FUSED) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (comp0 + c0 + j < comps_per_k) out[base + (size_t)(c0 + j) * N3] = cm(make_float2(re[j], im[j]), phc);
        } else {
          // four spinors at a time: every input is requested before any arithmetic
#pragma unroll
          for (int b = 0; b < 16; b += 8) {
            float2 pu[4], pd[4], ku[4], kd[4], qu[4], qd[4], au[4], ad[4], bu[4], bd[4];
            const float2 z2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int cu = c0 + b + 2 * j;
              pu[j] = pd[j] = ku[j] = kd[j] = qu[j] = qd[j] = au[j] = ad[j] = bu[j] = bd[j] = z2;
              if (comp0 + cu < comps_per_k) {
                const size_t ou = base + (size_t)cu * N3, od = ou + N3;
                pu[j] = io.Tk[ou]; pd[j] = io.Tk[od];
                ku[j] = io.kin[ou]; kd[j] = io.kin[od];
                if (rec) { qu[j] = io.Tkm1[ou]; qd[j] = io.Tkm1[od]; }
                if (ld1) { au[j] = io.acc1[ou]; ad[j] = io.acc1[od]; }
                if (ld2) { bu[j] = io.acc2[ou]; bd[j] = io.acc2[od]; }
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int cu = c0 + b + 2 * j;
              if (comp0 + cu >= comps_per_k) continue;
              const size_t ou = base + (size_t)cu * N3, od = ou + N3;
              const float2 vu = cm(make_float2(re[b + 2 * j], im[b + 2 * j]), phc);
              const float2 vd = cm(make_float2(re[b + 2 * j + 1], im[b + 2 * j + 1]), phc);
              float2 hu = make_float2(ku[j].x + vu.x, ku[j].y + vu.y);
              float2 hd = make_float2(kd[j].x + vd.x, kd[j].y + vd.y);
              const float2 u = pu[j], d = pd[j];
              hu = make_float2(hu.x + V0 * u.x + hx * d.x - hy * d.y, hu.y + V0 * u.y + hx * d.y + hy * d.x);
              hd = make_float2(hd.x + V1 * d.x + hx * u.x + hy * u.y, hd.y + V1 * d.y + hx * u.y - hy * u.x);
              float2 tu, td;
              // the series constants as float pairs (split_constants)
              if (!rec) {
                tu = make_float2(shifted_f(hu.x, u.x, ep.f_c, ep.f_id), shifted_f(hu.y, u.y, ep.f_c, ep.f_id));
                td = make_float2(shifted_f(hd.x, d.x, ep.f_c, ep.f_id), shifted_f(hd.y, d.y, ep.f_c, ep.f_id));
              } else {
                tu = make_float2(2.f * shifted_f(hu.x, u.x, ep.f_c, ep.f_id) - qu[j].x,
                                 2.f * shifted_f(hu.y, u.y, ep.f_c, ep.f_id) - qu[j].y);
                td = make_float2(2.f * shifted_f(hd.x, d.x, ep.f_c, ep.f_id) - qd[j].x,
                                 2.f * shifted_f(hd.y, d.y, ep.f_c, ep.f_id) - qd[j].y);
              }
              io.Tout[ou] = tu;
              io.Tout[od] = td;
              // accumulators: up to three terms (T_{k-1}, T_k, T_{k+1}) at once
              // float-float update, rounded once (ff_cmadd), as in k_epilogue
              auto upd = [&](float2* accp, int init, float2 ou_old, float2 od_old, const float* cmf, const float* c0f,
                             const float* c1f) {
                const float2 z2 = make_float2(0.f, 0.f);
                float2 hu2 = init ? z2 : ou_old, hd2 = init ? z2 : od_old, lu = z2, ld = z2;
                ff_cmadd(hu2, lu, tu, c1f);
                ff_cmadd(hd2, ld, td, c1f);
                ff_cmadd(hu2, lu, u, c0f);
                ff_cmadd(hd2, ld, d, c0f);
                if (rec) {
                  ff_cmadd(hu2, lu, qu[j], cmf);
                  ff_cmadd(hd2, ld, qd[j], cmf);
                }
                accp[ou] = make_float2(hu2.x + lu.x, hu2.y + lu.y);
                accp[od] = make_float2(hd2.x + ld.x, hd2.y + ld.y);
              };
              if (use1) upd(io.acc1, ep.init1, au[j], ad[j], ep.f_am, ep.f_a0, ep.f_a1);
              if (use2) upd(io.acc2, ep.init2, bu[j], bd[j], ep.f_bm, ep.f_b0, ep.f_b1);
            }
          }
        }
      }
    }
    if (abort_flag && lane == 0) atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == PT_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ============================================================================ launchers

// At least 120 KB, so that one CTA (holding all 512 tensor-memory columns) runs per SM.
size_t tile_gather_smem(int terms) {
  const size_t need = (size_t)((terms == 3) ? 2 : 1) * (PT_PART + 256 * PT_ROWB) * 2 + 1024;
  return need > 120 * 1024 ? need : 120 * 1024;
}
// With three products, at least 120 KB, so that one CTA (holding all 512 tensor-memory columns)
// runs per SM.
size_t tile_scatter_smem(int ek, int terms, int kch_max) {
  const int sc = (ek == TILE_TF32) ? 32 : 64;
  const size_t np = (terms == 3) ? 2 : 1;
  const size_t need = (size_t)kch_max * np * 2 * sc * PT_ROWB + 2 * np * PT_PART + 1024;
  return (terms == 3 && need < 120 * 1024) ? 120 * 1024 : need;
}

template <int EK, int TERMS>
static cudaError_t gather_et(cudaStream_t st, int N, const void* psi, int nk, int nstates, const TileDev& td,
                             double dV, const EpiParams& ep, const float* Dmat, float* part, void* c_out,
                             void* dc_out, int* err) {
  const int comps_per_k = 2 * nstates;
  const int groups = (comps_per_k + 63) / 64;
  const size_t smem = tile_gather_smem(TERMS);
  auto kf = k_tile_gather<EK, TERMS>;
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kf<<<dim3(nk * groups, td.nitems), PT_NT, smem, st>>>((const float2*)psi, N, comps_per_k, groups, td, ep, part, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tile_reduce<<<dim3(td.natoms, nk * groups), 64, 0, st>>>(part, td, groups, comps_per_k, nstates, td.natoms,
                                                             (float)dV, ep, Dmat, (float2*)c_out, (float2*)dc_out);
  return cudaGetLastError();
}

template <int EK, int TERMS, int FUSED>
static cudaError_t scatter_et(cudaStream_t st, int N, void* out, int nk, int nstates, const TileDev& td,
                              const EpiParams& ep, const void* dc, int* err, const EpiIO& io) {
  constexpr int SC = (Elt<EK>::bytes == 4) ? 32 : 64;
  const int comps_per_k = 2 * nstates;
  const int sgroups = (comps_per_k + SC - 1) / SC;
  const size_t smem = tile_scatter_smem(EK, TERMS, td.kch_max);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  auto kf = k_tile_scatter<EK, TERMS, FUSED>;
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kf<<<dim3(nk * sgroups, td.nitems), PT_NT, smem, st>>>((float2*)out, N, comps_per_k, sgroups, nstates, td.natoms,
                                                         td, ep, (const float2*)dc, err, io);
  return cudaGetLastError();
}

template <int FUSED>
static cudaError_t scatter_dispatch(cudaStream_t st, int N, void* out, int nk, int nstates, const TileDev& td,
                                    const EpiParams& ep, const void* dc, int* err, const EpiIO& io) {
  switch (td.ek * 4 + td.terms) {
    case TILE_TF32 * 4 + 1: return scatter_et<TILE_TF32, 1, FUSED>(st, N, out, nk, nstates, td, ep, dc, err, io);
    case TILE_TF32 * 4 + 3: return scatter_et<TILE_TF32, 3, FUSED>(st, N, out, nk, nstates, td, ep, dc, err, io);
    case TILE_BF16 * 4 + 3: return scatter_et<TILE_BF16, 3, FUSED>(st, N, out, nk, nstates, td, ep, dc, err, io);
    case TILE_F16 * 4 + 3: return scatter_et<TILE_F16, 3, FUSED>(st, N, out, nk, nstates, td, ep, dc, err, io);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_gather(cudaStream_t st, int N, const void* psi, int nk, int nstates, const TileDev& td,
                               double dV, const EpiParams& ep, const float* Dmat, float* part, void* c_out,
                               void* dc_out, int* err) {
  if (td.nitems == 0) return cudaSuccess;
  switch (td.ek * 4 + td.terms) {
    case TILE_TF32 * 4 + 1: return gather_et<TILE_TF32, 1>(st, N, psi, nk, nstates, td, dV, ep, Dmat, part, c_out, dc_out, err);
    case TILE_TF32 * 4 + 3: return gather_et<TILE_TF32, 3>(st, N, psi, nk, nstates, td, dV, ep, Dmat, part, c_out, dc_out, err);
    case TILE_BF16 * 4 + 3: return gather_et<TILE_BF16, 3>(st, N, psi, nk, nstates, td, dV, ep, Dmat, part, c_out, dc_out, err);
    case TILE_F16 * 4 + 3: return gather_et<TILE_F16, 3>(st, N, psi, nk, nstates, td, dV, ep, Dmat, part, c_out, dc_out, err);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_scatter(cudaStream_t st, int N, void* out, int nk, int nstates, const TileDev& td,
                                const EpiParams& ep, const void* dc, int* err) {
  if (td.nitems == 0) return cudaSuccess;
  return scatter_dispatch<0>(st, N, out, nk, nstates, td, ep, dc, err, EpiIO{});
}

cudaError_t launch_tile_epilogue(cudaStream_t st, int N, int nk, int nstates, const TileDev& td, const EpiParams& ep,
                                 const void* dc, int* err, const EpiIO& io) {
  if (ep.mode != EPI_FIRST && ep.mode != EPI_RECUR) return cudaErrorInvalidValue;
  if (td.nitems == 0) return cudaSuccess;
  EpiParams epx = ep;
  split_constants(epx);
  return scatter_dispatch<1>(st, N, nullptr, nk, nstates, td, epx, dc, err, io);
}

cudaError_t set_first_wait_tile(unsigned polls) { return cudaMemcpyToSymbol(g_first_wait, &polls, sizeof(polls)); }

}  // namespace tddft
