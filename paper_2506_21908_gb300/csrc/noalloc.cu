// Allocation-free Hartree (Poisson) solve: tddft_hartree_noalloc.
//
// Some callers cannot call cudaMalloc: frameworks that reserve all device memory up front
// and forbid further allocations, and latency-critical loops where an allocation's implicit
// device synchronisation is not acceptable.  This entry point solves the same Poisson problem as
// the library's own potential pipeline, but its scratch (one complex FP64 field and the
// FFT twiddles) lives in a file-scope static device array instead of memory owned by a
// handle.  The array exists on every GPU that loads the library, for the life of the
// process.
#include <mutex>
#include <string>

#include "impl.cuh"

namespace {

constexpr int kNoAllocMaxN = 64;
constexpr size_t kFieldElems = (size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN;
constexpr size_t kScratchElems = kFieldElems + kNoAllocMaxN;  // field + twiddles

// Shared by every call on a device; its contents persist between calls.
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_prepare(size_t n3, int N, const double* __restrict__ dens, double2* __restrict__ field,
                                  double2* __restrict__ tw) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) field[i] = make_double2(dens[i], 0.0);
  if (i < (size_t)N) {
    double s, c;
    sincospi(-2.0 * (double)i / (double)N, &s, &c);  // exp(-2 pi i t / N)
    tw[i] = make_double2(c, s);
  }
}

}  // namespace

namespace tddft {
void set_global_error(const std::string& msg);
}

extern "C" tddft_status tddft_hartree_noalloc(const double* n_dev, double* vH_dev, int n, const double* L,
                                              void* stream) {
  using namespace tddft;
  if (!n_dev || !vH_dev || !L) {
    set_global_error("tddft_hartree_noalloc: null pointer");
    return TDDFT_ERR_ARG;
  }
  static const int ok[] = {8, 12, 16, 24, 32, 48, 64};
  bool supported = false;
  for (int v : ok) supported = supported || (v == n);
  if (!supported) {
    set_global_error("tddft_hartree_noalloc: n must be one of 8, 12, 16, 24, 32, 48, 64 (static scratch holds "
                     "at most 64^3 complex values)");
    return TDDFT_ERR_ARG;
  }
  if (!(L[0] > 0.0) || !(L[1] > 0.0) || !(L[2] > 0.0)) {
    set_global_error("tddft_hartree_noalloc: cell lengths must be positive");
    return TDDFT_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(std::string("tddft_hartree_noalloc: no usable device: ") + cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  double2* scratch = nullptr;
  {
    // First call on this device: resolve the device address of the static array (the
    // host-side symbol is only a stand-in and must never be passed to a kernel).
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error(std::string("tddft_hartree_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return TDDFT_ERR_CUDA;
      }
      g_scratch_ptr[dev] = (double2*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n3 = (size_t)n * n * n;
  double2* field = scratch;
  double2* tw = scratch + kFieldElems;
  // every field element and twiddle used below is written first, so stale contents of the
  // shared array from an earlier call never leak into the result
  k_noalloc_prepare<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(n3, n, n_dev, field, tw);
  if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  {
    ZParams zp{};
    const double pi = 3.14159265358979323846;
    for (int a = 0; a < 3; ++a) zp.gs[a] = 2.0 * pi / L[a];
    zp.scale = 1.0 / (double)n3;
    if ((e = launch_fft_xy<double>(st, n, field, field, 1, tw, false)) != cudaSuccess) goto fail;
    if ((e = launch_fft_z<double>(st, n, field, 1, tw, Z_POISSON, zp)) != cudaSuccess) goto fail;
    if ((e = launch_fft_xy<double>(st, n, field, field, 1, tw, true)) != cudaSuccess) goto fail;
    if ((e = launch_complex_real_part(st, n3, field, vH_dev, 1.0)) != cudaSuccess) goto fail;
  }
  return TDDFT_OK;
fail:
  set_global_error(std::string("tddft_hartree_noalloc: launch failed: ") + cudaGetErrorString(e));
  return TDDFT_ERR_CUDA;
}
