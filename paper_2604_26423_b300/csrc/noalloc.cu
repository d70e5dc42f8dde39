// noalloc.cu -- measurement sampling that never allocates device memory.
//
// qaoa_sample_state_noalloc draws shots from a state vector the caller already
// holds on the GPU, using the same rule as qaoa_sample, but keeps its scratch
// (per-block probability sums and their prefix) in one fixed file-scope device
// array instead of buffers obtained from cudaMalloc. It is meant for callers
// that must not allocate while they run: a plugin whose enqueue step runs
// inside a host framework that owns every device allocation, or a serving loop
// with a preallocated memory budget that a cudaMalloc would break.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "qaoa.h"
#include "aux_kernels.cuh"

using namespace qaoa;

namespace {

// Scratch for the sampler: block sums S_j (QAOA_NOALLOC_MAX_BLOCKS doubles)
// followed by their exclusive prefix (QAOA_NOALLOC_MAX_BLOCKS + 1 doubles),
// about 1 MiB. Every GPU that loads this library keeps it until the process
// exits. In host code this name is only a stand-in for the device symbol; the
// device address comes from cudaGetSymbolAddress.
constexpr long long kScratchDoubles = 2LL * QAOA_NOALLOC_MAX_BLOCKS + 1;
static __device__ __align__(256) double g_sample_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_dev[kMaxDevices] = {};

// Looks up (once per device, with that device current) the device address of
// the scratch array. The address is kept for the life of the process: after a
// device reset (cudaDeviceReset, or a reset of the primary context) it is
// stale, so a process that resets a device must not call this entry point on
// that device again.
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QAOA_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return QAOA_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sample_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QAOA_ECUDA;
    }
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return QAOA_OK;
}

}  // namespace

extern "C" int qaoa_sample_state_noalloc(const void* state_dev, int n, int precision, int shots,
                                         const double* uniforms_dev, uint64_t seed, uint64_t* out_dev,
                                         void* cuda_stream) {
  if (precision != QAOA_C64 && precision != QAOA_C128) return QAOA_EINVAL;
  if (n < 1 || n > QAOA_NOALLOC_MAX_QUBITS) return QAOA_EINVAL;
  if (shots < 0) return QAOA_EINVAL;
  if (shots == 0) return QAOA_OK;
  if (!state_dev || !out_dev) return QAOA_EINVAL;
  // blocks of 2^B amplitudes: 2^12 as in qaoa_sample while that keeps the
  // number of blocks within the scratch, larger blocks beyond
  int B = std::min(n, 12);
  while ((1LL << (n - B)) > QAOA_NOALLOC_MAX_BLOCKS) ++B;
  const long long nb = 1LL << (n - B);
  if (nb > QAOA_NOALLOC_MAX_BLOCKS) return QAOA_EINVAL;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  double* sums = scratch;
  double* pre = scratch + QAOA_NOALLOC_MAX_BLOCKS;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // every scratch entry read below is written earlier in the same call, so
  // nothing needs clearing between calls
  if (precision == QAOA_C128)
    block_sum_kernel<double><<<(unsigned)nb, 256, 0, st>>>(static_cast<const double2*>(state_dev), B, sums);
  else
    block_sum_kernel<float><<<(unsigned)nb, 256, 0, st>>>(static_cast<const float2*>(state_dev), B, sums);
  scan_kernel<<<1, 1024, 0, st>>>(sums, nb, pre);
  // one warp per shot, four per block: the search and in-block walk of
  // qaoa_sample (coalesced 32-amplitude steps, the same FP64 order)
  constexpr int kWarpsPerBlock = 4;
  const long long gb = ((long long)shots + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (gb > INT_MAX) return QAOA_EINVAL;
  if (precision == QAOA_C128)
    shot_warp_kernel<double><<<(unsigned)gb, 32 * kWarpsPerBlock, 0, st>>>(
        static_cast<const double2*>(state_dev), B, pre, nb, shots, uniforms_dev, seed,
        reinterpret_cast<unsigned long long*>(out_dev));
  else
    shot_warp_kernel<float><<<(unsigned)gb, 32 * kWarpsPerBlock, 0, st>>>(
        static_cast<const float2*>(state_dev), B, pre, nb, shots, uniforms_dev, seed,
        reinterpret_cast<unsigned long long*>(out_dev));
  return cudaGetLastError() == cudaSuccess ? QAOA_OK : QAOA_ECUDA;
}
