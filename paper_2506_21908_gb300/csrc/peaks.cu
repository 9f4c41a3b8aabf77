// Peak-rate microbenchmarks of this GPU, for the roofline denominators the copy bandwidth and the
// library GEMM do not give: FP64 and FP32 fused multiply-adds on the CUDA cores, and dense
// tcgen05 products of kind tf32 and f16 (FP16 and BF16 operands) with FP32 accumulation.
//
// FMA kernels: every thread runs 8 independent chains of dependent FMAs in registers (no memory
// traffic); 4 CTAs of 256 threads per SM.  MMA kernel: one CTA per SM; one elected thread issues
// back-to-back 128 x 256 x K products from shared-memory operands (contents irrelevant) into a
// 256-column tensor-memory accumulator, committing to an mbarrier every 64 products; every wait
// has an iteration limit.  Rates are FLOPs (2 per multiply-add) over the CUDA-event time.
#include <cstdint>

#include "bulk.cuh"
#include "impl.cuh"

namespace tddft {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains live
}

constexpr int PK_N = 256;

__device__ __forceinline__ uint64_t pk_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}

// kind code: 0 f16 (FP16), 1 f16 (BF16), 2 tf32
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int nmma, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  // A: 128 rows x 128 bytes, B: 256 rows x 128 bytes (one K chunk), zero-filled
  for (int i = threadIdx.x; i < (128 + PK_N) * 128 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&tmem_base)),
                 "r"(PK_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t code = KIND == 2 ? 2u : (uint32_t)KIND;
    const uint32_t id = (1u << 4) | (code << 7) | (code << 10) | ((uint32_t)(PK_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint64_t ad = pk_desc(sm_addr(smem)), bd = pk_desc(sm_addr(smem + 128 * 128));
    uint32_t phase = 0;
    for (int i = 0; i < nmma; ++i) {
      const uint32_t acc = i ? 1u : 0u;
      if constexpr (KIND == 2)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
      else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
      if ((i & 63) == 63 || i == nmma - 1) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_addr(&bar))
                     : "memory");
        if (!bulk_try_wait(sm_addr(&bar), phase)) atomicOr(err, 1);
        phase ^= 1u;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PK_N));
}

template <class F> double time_ms(F&& f) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  f();  // warm-up
  cudaEventRecord(a);
  f();
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)ms;
}

}  // namespace

// out[0..4]: FP64 FMA, FP32 FMA, TF32 MMA, FP16 MMA, BF16 MMA (TFLOP/s, dense).
cudaError_t measure_peaks(double* out, int nout) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* buf = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&buf, 256);
  if (e != cudaSuccess) return e;
  if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) { cudaFree(buf); return e; }
  cudaMemset(err, 0, sizeof(int));
  const int blocks = 4 * sms, threads = 256;
  double r[5] = {0, 0, 0, 0, 0};
  {
    const int it = 4096;
    const double flops = 2.0 * 16 * 8 * (double)it * blocks * threads;
    const double ms = time_ms([&] { k_peak_fma<double><<<blocks, threads>>>((double*)buf, it, 1.0000001, 1e-7); });
    r[0] = flops / (ms * 1e-3) / 1e12;
  }
  {
    const int it = 65536;
    const double flops = 2.0 * 16 * 8 * (double)it * blocks * threads;
    const double ms = time_ms([&] { k_peak_fma<float><<<blocks, threads>>>((float*)buf, it, 1.0000001f, 1e-7f); });
    r[1] = flops / (ms * 1e-3) / 1e12;
  }
  const size_t smem = (size_t)(128 + PK_N) * 128 + 1024;
  const int nmma = 65536;
  auto mma_rate = [&](auto kern, int K) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double flops = 2.0 * 128 * PK_N * K * (double)nmma * sms;
    const double ms = time_ms([&] { kern<<<sms, 128, smem>>>(nmma, err); });
    return flops / (ms * 1e-3) / 1e12;
  };
  r[2] = mma_rate(k_peak_mma<2>, 8);
  r[3] = mma_rate(k_peak_mma<0>, 16);
  r[4] = mma_rate(k_peak_mma<1>, 16);
  e = cudaDeviceSynchronize();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  cudaFree(err);
  if (e != cudaSuccess) return e;
  if (herr) return cudaErrorLaunchTimeout;
  for (int i = 0; i < nout && i < 5; ++i) out[i] = r[i];
  return cudaSuccess;
}

}  // namespace tddft

extern "C" tddft_status tddft_measure_peaks(double* out, int nout) {
  if (!out || nout < 1) return TDDFT_ERR_ARG;
  const cudaError_t e = tddft::measure_peaks(out, nout);
  return e == cudaSuccess ? TDDFT_OK : TDDFT_ERR_CUDA;
}
