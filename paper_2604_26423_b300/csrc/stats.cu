// stats.cu -- context-free entry points of the sampling methodology (Sec.
// II-D): the mean of subsample means (device) and the regime classification
// (host). qaoa_sample_cuts, which needs a context's graph, is in api.cu.
#include <cuda_runtime.h>

#include <cmath>

#include "qaoa.h"
#include "stats_kernels.cuh"

using namespace qaoa;

extern "C" {

int qaoa_mean_of_means(const double* r_dev, int64_t m, int ns, int reps, uint64_t seed, double* means_dev,
                       double* stats_dev, void* cuda_stream) {
  if (!r_dev || !means_dev || !stats_dev) return QAOA_EINVAL;
  if (m < 1 || m >= (int64_t)0xffffffffLL) return QAOA_EINVAL;
  if (ns < 1 || ns > QAOA_MOM_MAX_NS || (int64_t)ns > m) return QAOA_EINVAL;
  if (reps < 1 || reps > 65535) return QAOA_EINVAL;
  // table of 2^log2cap slots, at least 2 ns + 1 (at most ns keys are inserted)
  int log2cap = 1;
  while ((1 << log2cap) < 2 * ns + 1) ++log2cap;
  MeanOfMeansArgs a;
  a.r = r_dev;
  a.m = (unsigned long long)m;
  a.ns = ns;
  a.reps = reps;
  a.log2cap = log2cap;
  a.seed = seed;
  a.means = means_dev;
  a.stats = stats_dev;
  const size_t smem = size_t(2) << log2cap << 2;  // keys and values, 4 bytes each
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaFuncSetAttribute(mean_of_means_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return QAOA_ECUDA;
  }
  mean_of_means_kernel<<<reps, 32, smem, st>>>(a);
  mean_of_means_final_kernel<<<1, 1, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? QAOA_OK : QAOA_ECUDA;
}

int qaoa_classify_regime(double r_obs, double rand_mean, double rand_sigma, int have_ideal, double ideal_mean,
                         double ideal_sigma) {
  if (std::isnan(rand_sigma) || rand_sigma < 0) return -1;
  if (have_ideal && (std::isnan(ideal_sigma) || ideal_sigma < 0)) return -1;
  if (!(r_obs > rand_mean + 3.0 * rand_sigma)) return QAOA_REGIME_RANDOM;
  if (!have_ideal) return QAOA_REGIME_ABOVE_RANDOM;
  return r_obs >= ideal_mean - 3.0 * ideal_sigma ? QAOA_REGIME_NOISE_TOLERANT : QAOA_REGIME_TRANSITION;
}

double qaoa_overlap_ratio(double r_noisy, double r_ideal, double r_random) {
  return (r_noisy - r_random) / (r_ideal - r_random);
}

double qaoa_fit_k0(int count, const double* eps_acc, const double* r_ovl) {
  if (count < 1 || !eps_acc || !r_ovl) return NAN;
  double num = 0.0, den = 0.0;
  for (int i = 0; i < count; ++i) {
    if (!(r_ovl[i] > 0.0)) continue;
    num += eps_acc[i] * std::log2(r_ovl[i]);
    den += eps_acc[i] * eps_acc[i];
  }
  return den > 0.0 ? -num / den : NAN;
}

}  // extern "C"
