// stats_kernels.cuh -- sampling methodology (Sec. II-D): cut values and
// approximation ratios of individual bitstrings (shots or the uniform random
// sampler), and the mean of subsample means drawn without replacement.
#pragma once
#include <cstdint>

#include "aux_kernels.cuh"

namespace qaoa {

// C(x) = sum_i x_i d_i - 2 sum_{i<j} w_ij x_i x_j (the Sec. II-B cut formula
// with d_i = sum_j w_ij), the pair sum taken by weight bit planes: for plane t
// of sign s, U_i = {j > i : w_ij has sign s and bit t of |w_ij| set}, and
// sum_{j>i} w_ij x_j = sum_planes coef * popcount(U_i & x), coef = +-2^t.
// Planes without any edge are left out.
constexpr int kMaxCutPlanes = 62;

struct SampleCutArgs {
  int n = 0, planes = 0;
  const unsigned long long* tab = nullptr;  // planes x n masks | planes coefs (int64) | n row sums (int64)
  long long count = 0;
  const unsigned long long* x = nullptr;    // bitstrings, or nullptr: draw i of stream `seed`, top n bits
  unsigned long long seed = 0;
  long long c_min = 0, c_max = 0;
  unsigned long long* x_out = nullptr;
  int32_t* c_out = nullptr;
  double* r_out = nullptr;
  int* bad = nullptr;                        // set to 1 when an input bitstring has bits >= n
};

// Dynamic shared memory: (planes * (n + 1) + n) * 8 bytes.
static __global__ void __launch_bounds__(256) sample_cut_kernel(const SampleCutArgs a) {
  extern __shared__ unsigned long long st[];
  const int n = a.n, P = a.planes;
  const int words = P * n + P + n;
  for (int k = threadIdx.x; k < words; k += blockDim.x) st[k] = a.tab[k];
  __syncthreads();
  const unsigned long long* masks = st;
  const long long* coef = reinterpret_cast<const long long*>(st + P * n);
  const long long* dsum = coef + P;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const double span = double(a.c_max - a.c_min);
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.count; s += stride) {
    unsigned long long x;
    if (a.x) {
      x = a.x[s];
      if (x >> n) {
        *a.bad = 1;
        x &= (1ull << n) - 1ull;
      }
    } else {
      x = splitmix_draw(a.seed, (unsigned long long)s) >> (64 - n);
    }
    // only the vertices with x_i = 1 contribute: walk the set bits of x
    long long c = 0, q = 0;
    for (unsigned long long b = x; b; b &= b - 1ull) {
      const int i = __ffsll((long long)b) - 1;
      c += dsum[i];
      for (int p = 0; p < P; ++p) q += coef[p] * __popcll(masks[p * n + i] & x);
    }
    c -= 2 * q;
    if (a.x_out) a.x_out[s] = x;
    if (a.c_out) a.c_out[s] = (int32_t)c;
    if (a.r_out) a.r_out[s] = a.c_max == a.c_min ? 1.0 : double(c - a.c_min) / span;
  }
}

// Mean of subsample means: one CTA per subsample. Its displaced positions
// (the partial Fisher-Yates shuffle leaves every other position holding its
// own index) live in an open-addressing table in shared memory: 2^log2cap
// uint32 keys (0xffffffff = empty) then 2^log2cap uint32 values, with
// 2^log2cap >= 2 ns + 1 so a probe always ends.
struct MeanOfMeansArgs {
  const double* r = nullptr;
  unsigned long long m = 0;
  int ns = 0, reps = 0, log2cap = 0;
  unsigned long long seed = 0;
  double* means = nullptr;
  double* stats = nullptr;
};

__device__ __forceinline__ unsigned mom_slot(const unsigned* keys, unsigned key, int log2cap) {
  const unsigned mask = (1u << log2cap) - 1u;
  unsigned h = (key * 2654435761u) >> (32 - log2cap);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const unsigned k = keys[h];
    if (k == key || k == 0xffffffffu) return h;
    h = (h + 1u) & mask;
  }
  return h;  // not reached: the table is never more than half full
}

static __global__ void __launch_bounds__(32) mean_of_means_kernel(const MeanOfMeansArgs a) {
  extern __shared__ unsigned tabw[];
  const unsigned cap = 1u << a.log2cap;
  unsigned* keys = tabw;
  unsigned* vals = tabw + cap;
  for (unsigned e = threadIdx.x; e < cap; e += 32) keys[e] = 0xffffffffu;
  __syncwarp();
  if (threadIdx.x != 0) return;
  const unsigned long long base = (unsigned long long)blockIdx.x * (unsigned long long)a.ns;
  double acc = 0.0;
  for (int j = 0; j < a.ns; ++j) {
    const unsigned long long z = splitmix_draw(a.seed, base + (unsigned long long)j);
    const unsigned k = (unsigned)j + (unsigned)__umul64hi(z, a.m - (unsigned long long)j);
    const unsigned hj = mom_slot(keys, (unsigned)j, a.log2cap);
    const unsigned vj = keys[hj] == (unsigned)j ? vals[hj] : (unsigned)j;
    const unsigned hk = mom_slot(keys, k, a.log2cap);
    const unsigned vk = keys[hk] == k ? vals[hk] : k;
    // position k now holds position j's entry; position j is never read again
    keys[hk] = k;
    vals[hk] = vj;
    acc = __dadd_rn(acc, a.r[vk]);
  }
  a.means[blockIdx.x] = acc / double(a.ns);
}

// Grand mean, sigma and threshold, summed in subsample order (one thread;
// explicit roundings so that no product is fused into a sum).
static __global__ void mean_of_means_final_kernel(const MeanOfMeansArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double g = 0.0;
  for (int i = 0; i < a.reps; ++i) g = __dadd_rn(g, a.means[i]);
  g = g / double(a.reps);
  double var = 0.0;
  for (int i = 0; i < a.reps; ++i) {
    const double d = __dsub_rn(a.means[i], g);
    var = __dadd_rn(var, __dmul_rn(d, d));
  }
  const double sigma = sqrt(var / double(a.reps));
  a.stats[0] = g;
  a.stats[1] = sigma;
  a.stats[2] = __dadd_rn(g, __dmul_rn(3.0, sigma));
}

}  // namespace qaoa
