// Kinetic term of one spinor component in one kernel, using a 16-CTA thread-block cluster.
//
// The 16 CTAs of a cluster hold the whole n^3 component in their shared memory (CTA c keeps
// z-planes [c P, (c+1) P), P = n/16).  Each CTA transforms its planes along x and y, the
// cluster synchronises, then each CTA owns P y-values: it gathers the (z, x) slab of each of
// them from the 16 CTAs' shared memory (distributed shared memory), transforms along z,
// multiplies by 1/2 |G + k + A|^2 / n^3, transforms back and scatters the slab to its owners.
// After a second cluster barrier every CTA transforms its planes back along y and x and writes
// them out.  One read and one write of the component in HBM instead of three of each.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "impl.cuh"
#include "kcommon.cuh"

namespace cg = cooperative_groups;

namespace tddft {

constexpr int KC_CLUSTER = 16;

template <int N> struct KinClusterThreads { static constexpr int value = 512; };

template <int N>
__global__ void __cluster_dims__(KC_CLUSTER, 1, 1) __launch_bounds__(512, 1)
k_kinetic_cluster(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ twg, ZParams zp) {
  constexpr int NT = 512;
  constexpr int P = N / KC_CLUSTER;   // planes per CTA
  constexpr int RS = N + 1;
  constexpr int PS = N * RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* pl = tw + N;                 // [P][N][RS] my z-planes
  float2* sl = pl + P * PS;            // [N z][N x] one y-slab (dense)
  float* tx = reinterpret_cast<float*>(sl + N * N);
  float* tz = tx + N;
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int b = blockIdx.y;
  const int k = b / zp.comps_per_k;
  const size_t base = (size_t)b * N * N * N + (size_t)c * P * N * N;
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = twg[i];
    const double qx = zp.gs[0] * freq<N>(i) + zp.shift[k][0];
    const double qz = zp.gs[2] * freq<N>(i) + zp.shift[k][2];
    tx[i] = (float)(0.5 * qx * qx * zp.scale);
    tz[i] = (float)(0.5 * qz * qz * zp.scale);
  }
  for (int p = 0; p < P; ++p) plane_load<N, NT, RS>(pl + p * PS, in + base + (size_t)p * N * N);
  __syncthreads();
  fft_pass<float2, N, NT, false, P>(pl, RS, 1, tw, PS);  // along x, all my planes
  fft_pass<float2, N, NT, false, P>(pl, 1, RS, tw, PS);  // along y
  cluster.sync();
  for (int yl = 0; yl < P; ++yl) {
    const int y = c * P + yl;
    // gather the (z, x) slab at this y from the owners of every z-plane
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int z = i / N, x = i - z * N;
      const float2* src = cluster.map_shared_rank(pl, z / P);
      sl[i] = src[(z % P) * PS + y * RS + x];
    }
    __syncthreads();
    fft_pass<float2, N, NT, false>(sl, 1, N, tw);  // along z (rows: x)
    const double qy = zp.gs[1] * freq<N>(y) + zp.shift[k][1];
    const float ty = (float)(0.5 * qy * qy * zp.scale);
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int z = i / N, x = i - z * N;
      sl[i] = cscale(sl[i], tx[x] + ty + tz[z]);
    }
    __syncthreads();
    fft_pass<float2, N, NT, true>(sl, 1, N, tw);
    for (int i = threadIdx.x; i < N * N; i += NT) {
      const int z = i / N, x = i - z * N;
      float2* dst = cluster.map_shared_rank(pl, z / P);
      dst[(z % P) * PS + y * RS + x] = sl[i];
    }
    __syncthreads();
  }
  cluster.sync();
  fft_pass<float2, N, NT, true, P>(pl, 1, RS, tw, PS);  // along y
  fft_pass<float2, N, NT, true, P>(pl, RS, 1, tw, PS);  // along x
  for (int p = 0; p < P; ++p) plane_store<N, NT, RS>(out + base + (size_t)p * N * N, pl + p * PS);
}

template <int N>
static cudaError_t kin_cluster_n(cudaStream_t st, const void* in, void* out, int nbatch, const void* tw,
                                 const ZParams& zp) {
  constexpr int P = N / KC_CLUSTER;
  const size_t smem = (size_t)(N + P * N * (N + 1) + N * N) * sizeof(float2) + 2 * N * sizeof(float);
  auto kf = k_kinetic_cluster<N>;
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kf, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  kf<<<dim3(KC_CLUSTER, nbatch), 512, smem, st>>>((const float2*)in, (float2*)out, (const float2*)tw, zp);
  return cudaGetLastError();
}

bool kinetic_cluster_supported(int N) { return N == 32 || N == 48 || N == 64; }

cudaError_t launch_kinetic_cluster(cudaStream_t st, int N, const void* in, void* out, int nbatch, const void* tw,
                                   const ZParams& zp) {
  switch (N) {
    case 32: return kin_cluster_n<32>(st, in, out, nbatch, tw, zp);
    case 48: return kin_cluster_n<48>(st, in, out, nbatch, tw, zp);
    case 64: return kin_cluster_n<64>(st, in, out, nbatch, tw, zp);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tddft
