// Tensor-core (tcgen05, kind::tf32) projector contraction for the FP32-mixed path.
//
// For one atom a and one k-point, the projections are a dense contraction over the atom's
// sphere points e:
//     c[comp][p] = sum_e psi_comp(r_e) B_p(e),   B_p(e) = beta_p(d_e) exp(+i (k+A).d_e) dV,
// with comp = (state, sigma).  In real arithmetic, with A rows = (Re psi | Im psi) of 64
// components and B columns = (Re B_p | Im B_p) of the 9 projectors, one 128 x 32 x K product
// gives every term: c_r = P[re][Br] - P[im][Bi], c_i = P[re][Bi] + P[im][Br].
//
// Each CTA (128 threads) handles one atom, one tile of 64 components of one k-point and one
// contiguous part of the sphere (the K dimension is split over CTAs for parallelism).  Per chunk
// of 32 sphere points the threads gather psi and evaluate B into shared memory in the canonical
// no-swizzle K-major layout (8 x 16-byte core matrices), one elected thread issues the MMAs
// (accumulator in tensor memory) and commits them to an mbarrier.  TF32x3 splits both operands
// into hi + lo TF32 parts and accumulates hi*hi + hi*lo + lo*hi.  Partial products are reduced
// over the K parts in a fixed order by a second kernel, which also applies the D blocks.
//
// Every mbarrier wait has an iteration limit; on expiry the CTA records an error flag, stops
// issuing work, and still frees its tensor memory.
#include <cstdint>

#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"

namespace tddft {

namespace {

constexpr int TC_M = 128;          // rows: 64 components x (re, im)
constexpr int TC_COMPS = 64;
constexpr int TC_N = 32;           // columns: 9 x (re, im) projectors, padded
constexpr int TC_KC = 32;          // sphere points per chunk
constexpr int TC_LBO = 128;        // bytes between core matrices adjacent in K
constexpr int TC_SBO = (TC_KC / 4) * 128;  // bytes between core matrices adjacent in M/N
constexpr int TC_A_BYTES = TC_M * TC_KC * 4;   // 16 KB
constexpr int TC_B_BYTES = TC_N * TC_KC * 4;   // 4 KB
constexpr unsigned TC_WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major no-swizzle operand tile
__device__ __forceinline__ int core_off(int row, int k) {
  return (row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for this architecture family; no swizzle
  return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 32.
__device__ __forceinline__ uint32_t tf32_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t phase) {
  for (unsigned it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace

// part[ks][k-tile][comp][32]: partial 128x32 products are folded to complex c here:
// out layout per (atom, k, comp): 18 reals = c_r[9], c_i[9].
template <int SPLIT3>
__global__ void __launch_bounds__(128)
k_proj_gather_tc(const float2* __restrict__ psi, size_t N3, ProjTables<float> pt, float dV, EpiParams ep,
                 int comps_per_k, int tiles_per_k, int kparts, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // stage layout: A_hi | A_lo | B_hi | B_lo | fold buffer
  unsigned char* sA = smem_raw;
  unsigned char* sAl = sA + TC_A_BYTES;
  unsigned char* sB = sAl + (SPLIT3 ? TC_A_BYTES : 0);
  unsigned char* sBl = sB + TC_B_BYTES;
  float* fold = reinterpret_cast<float*>(sBl + (SPLIT3 ? TC_B_BYTES : 0));  // [128][33]
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int a = blockIdx.x;
  const int tile = blockIdx.y;             // k * tiles_per_k + t
  const int kp = blockIdx.z;               // K part
  const int k = tile / tiles_per_k;
  const int comp0 = (tile % tiles_per_k) * TC_COMPS;  // within this k-point
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float sx = (float)ep.shift[k][0], sy = (float)ep.shift[k][1], sz = (float)ep.shift[k][2];
  constexpr int TAB = 3 + 9;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // zero the padding columns 18..31 of the B tiles once
  for (int i = threadIdx.x; i < (TC_N - 18) * TC_KC; i += 128) {
    const int n = 18 + i / TC_KC, kk = i % TC_KC;
    *reinterpret_cast<float*>(sB + core_off(n, kk)) = 0.0f;
    if (SPLIT3) *reinterpret_cast<float*>(sBl + core_off(n, kk)) = 0.0f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  const int e_begin = pt.g_ptr[a], e_end = pt.g_ptr[a + 1];
  const int ne = e_end - e_begin;
  const int per = (ne + kparts - 1) / kparts;
  const int my0 = e_begin + kp * per;
  const int my1 = min(e_end, my0 + per);
  const uint32_t idesc = tf32_idesc();
  const float2* base = psi + (size_t)k * comps_per_k * N3;
  uint32_t phase = 0;
  int issued = 0;
  for (int e0 = my0; e0 < my1; e0 += TC_KC) {
    // ---- gather psi: a warp covers 8 components x 4 sphere points per step (conflict-free stores)
    for (int pr = warp; pr < (TC_COMPS / 8) * (TC_KC / 4); pr += 4) {
      const int cg = pr % (TC_COMPS / 8), kg = pr / (TC_COMPS / 8);
      const int cl = cg * 8 + (lane >> 2);
      const int kk = kg * 4 + (lane & 3);
      const int e = e0 + kk;
      const int comp = comp0 + cl;
      float2 v = make_float2(0.0f, 0.0f);
      if (e < my1 && comp < comps_per_k) v = base[(size_t)comp * N3 + pt.g_idx[e]];
      const float hr = tf32_round(v.x), hi = tf32_round(v.y);
      *reinterpret_cast<float*>(sA + core_off(cl, kk)) = hr;
      *reinterpret_cast<float*>(sA + core_off(TC_COMPS + cl, kk)) = hi;
      if (SPLIT3) {
        *reinterpret_cast<float*>(sAl + core_off(cl, kk)) = tf32_round(v.x - hr);
        *reinterpret_cast<float*>(sAl + core_off(TC_COMPS + cl, kk)) = tf32_round(v.y - hi);
      }
    }
    // ---- B = beta_p exp(+i s.d) dV for 32 sphere points; warp w handles p = w, w + 4, w + 8
    {
      const int kk = lane;
      const int e = e0 + kk;
      float cs = 0.0f, sn = 0.0f;
      const float* t = nullptr;
      if (e < my1) {
        t = pt.g_tab + (size_t)e * TAB;
        sincosf(sx * t[0] + sy * t[1] + sz * t[2], &sn, &cs);
      }
      for (int p = warp; p < 9; p += 4) {
        const float bp = t ? t[3 + p] * dV : 0.0f;
        const float br = bp * cs, bi = bp * sn;
        const float hr = tf32_round(br), hi = tf32_round(bi);
        *reinterpret_cast<float*>(sB + core_off(p, kk)) = hr;
        *reinterpret_cast<float*>(sB + core_off(9 + p, kk)) = hi;
        if (SPLIT3) {
          *reinterpret_cast<float*>(sBl + core_off(p, kk)) = tf32_round(br - hr);
          *reinterpret_cast<float*>(sBl + core_off(9 + p, kk)) = tf32_round(bi - hi);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int ks = 0; ks < TC_KC / 8; ++ks) {
        const uint32_t off = (uint32_t)ks * 2 * TC_LBO;  // 8 TF32 along K = two core matrices
        const uint64_t ah = smem_desc(smem_addr(sA) + off), bh = smem_desc(smem_addr(sB) + off);
        mma_tf32(tmem, ah, bh, idesc, (issued | ks) ? 1u : 0u);
        if (SPLIT3) {
          const uint64_t al = smem_desc(smem_addr(sAl) + off), bl = smem_desc(smem_addr(sBl) + off);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar)));
    }
    issued = 1;
    // the tiles are rewritten next chunk: wait for the MMAs that read them
    if (!mbar_wait(smem_addr(&mbar), phase)) abort_flag = 1;
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  float* out = part + (((size_t)kp * gridDim.y + tile) * gridDim.x + a) * (size_t)TC_COMPS * 18;
  if (!abort_flag) {
    // ---- accumulator rows -> registers (warp w owns lanes 32w..32w+31) -> shared fold buffer
    uint32_t r[32];
    if (issued) {
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = 0u;
    }
    const int row = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) fold[row * 33 + j] = __uint_as_float(r[j]);
    __syncthreads();
    // c_r[p] = P[re][p] - P[im][9+p], c_i[p] = P[re][9+p] + P[im][p]
    for (int i = threadIdx.x; i < TC_COMPS * 9; i += 128) {
      const int cl = i / 9, p = i % 9;
      const float* re = fold + cl * 33;
      const float* im = fold + (TC_COMPS + cl) * 33;
      out[cl * 18 + p] = re[p] - im[9 + p];
      out[cl * 18 + 9 + p] = re[9 + p] + im[p];
    }
  } else if (threadIdx.x == 0) {
    atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

// Sum the K parts in a fixed order, write c[kb][a][2p + sigma] and dc = D c.
__global__ void k_proj_tc_reduce(const float* __restrict__ part, int natoms, int ntiles, int kparts, int comps_per_k,
                                 int tiles_per_k, int nstates, const float* __restrict__ Dmat, float2* __restrict__ c_out,
                                 float2* __restrict__ dc_out) {
  // one CTA per (atom, tile): 32 spinors x 18 outputs
  const int a = blockIdx.x, tile = blockIdx.y;
  const int k = tile / tiles_per_k;
  const int comp0 = (tile % tiles_per_k) * TC_COMPS;
  __shared__ float2 cs[TC_COMPS / 2][18];  // [spinor in tile][2p + sigma]
  for (int i = threadIdx.x; i < TC_COMPS * 9; i += blockDim.x) {
    const int cl = i / 9, p = i % 9;
    float re = 0.0f, im = 0.0f;
    for (int kp = 0; kp < kparts; ++kp) {
      const float* src = part + (((size_t)kp * ntiles + tile) * natoms + a) * (size_t)TC_COMPS * 18;
      re += src[cl * 18 + p];
      im += src[cl * 18 + 9 + p];
    }
    cs[cl >> 1][2 * p + (cl & 1)] = make_float2(re, im);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (TC_COMPS / 2) * 18; i += blockDim.x) {
    const int sl = i / 18, q = i % 18;
    const int comp = comp0 + 2 * sl;
    if (comp >= comps_per_k) continue;
    const int kb = k * nstates + comp / 2;
    const float* D = Dmat + ((size_t)a * 18 + q) * 18 * 2;
    float re = 0.0f, im = 0.0f;
    for (int u = 0; u < 18; ++u) {
      const float dr = D[2 * u], di = D[2 * u + 1];
      re += dr * cs[sl][u].x - di * cs[sl][u].y;
      im += dr * cs[sl][u].y + di * cs[sl][u].x;
    }
    const size_t o = ((size_t)kb * natoms + a) * 18 + q;
    c_out[o] = cs[sl][q];
    dc_out[o] = make_float2(re, im);
  }
}

int proj_tc_kparts(int natoms, int ntiles) {
  // enough CTAs to cover the SMs a few times over
  const int want = 4 * 152;
  int kp = (want + natoms * ntiles - 1) / (natoms * ntiles);
  return kp < 1 ? 1 : (kp > 64 ? 64 : kp);
}

cudaError_t launch_proj_gather_tc(cudaStream_t st, int N, const void* psi, int nk, int nstates,
                                  const ProjTables<float>& pt, double dV, const EpiParams& ep, int split3,
                                  float* part, void* c_out, void* dc_out, int* err) {
  if (pt.natoms == 0) return cudaSuccess;
  if (pt.nlm != 9) return cudaErrorInvalidValue;
  const size_t N3 = (size_t)N * N * N;
  const int comps_per_k = 2 * nstates;
  const int tiles_per_k = (comps_per_k + TC_COMPS - 1) / TC_COMPS;
  const int ntiles = nk * tiles_per_k;
  const int kparts = proj_tc_kparts(pt.natoms, ntiles);
  const size_t smem = (split3 ? 2 : 1) * (size_t)(TC_A_BYTES + TC_B_BYTES) + (size_t)TC_M * 33 * 4 + 1024;
  dim3 grid(pt.natoms, ntiles, kparts);
  if (split3) {
    cudaFuncSetAttribute(k_proj_gather_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_proj_gather_tc<1><<<grid, 128, smem, st>>>((const float2*)psi, N3, pt, (float)dV, ep, comps_per_k, tiles_per_k,
                                                 kparts, part, err);
  } else {
    cudaFuncSetAttribute(k_proj_gather_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_proj_gather_tc<0><<<grid, 128, smem, st>>>((const float2*)psi, N3, pt, (float)dV, ep, comps_per_k, tiles_per_k,
                                                 kparts, part, err);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_proj_tc_reduce<<<dim3(pt.natoms, ntiles), 128, 0, st>>>(part, pt.natoms, ntiles, kparts, comps_per_k, tiles_per_k,
                                                           nstates, pt.Dmat, (float2*)c_out, (float2*)dc_out);
  return cudaGetLastError();
}

size_t proj_tc_part_floats(int natoms, int nk, int nstates) {
  const int tiles_per_k = (2 * nstates + TC_COMPS - 1) / TC_COMPS;
  const int ntiles = nk * tiles_per_k;
  return (size_t)proj_tc_kparts(natoms, ntiles) * ntiles * natoms * TC_COMPS * 18;
}

}  // namespace tddft
