// aux_kernels.cuh -- cost diagonal / exhaustive extremes, reductions, sampling.
#pragma once
#include <climits>
#include <cstdint>

#include "device.cuh"

namespace qaoa {

// ---------------------------------------------------------------------------
// C(x) = sum_{k<l} w_kl [x_k != x_l] (Eq. for C(x)) for a block of 2^LB
// consecutive x (LB = 15, 1024 threads x 32 values). The block's high bits
// (>= LB) are fixed: per block, delta_j = sum_{g >= LB} w[j][g] (1 - 2 f_g) and
// base = C over the high bits + sum_{j < LB, g >= LB} w[j][g] f_g. A thread
// owns bits 5..LB-1 (value t) and enumerates bits 0..4 (value j):
//   C = base + sum_{k in 5..LB-1} t_k delta_k + C_mid(t) + sum_{i<5} A_i(t)
//       + sum_{i<5} j_i (delta_i + D_i - 2 A_i(t)) + C_low(j)
// with A_i(t) = sum_k w[i][k] t_k, D_i = sum_k w[i][k] over k in 5..LB-1.
// Optionally writes the int32 diagonal; always reduces (min, argmin, max, argmax)
// with ties resolved to the smallest index.
// ---------------------------------------------------------------------------
struct Extreme {
  long long vmin, vmax;
  unsigned long long amin, amax;
};

__device__ __forceinline__ void ext_merge(Extreme& a, const Extreme& b) {
  if (b.vmin < a.vmin || (b.vmin == a.vmin && b.amin < a.amin)) { a.vmin = b.vmin; a.amin = b.amin; }
  if (b.vmax > a.vmax || (b.vmax == a.vmax && b.amax < a.amax)) { a.vmax = b.vmax; a.amax = b.amax; }
}

__device__ __forceinline__ void ext_warp_merge(Extreme& ex) {
  for (int o = 16; o > 0; o >>= 1) {
    Extreme b;
    b.vmin = __shfl_xor_sync(0xffffffffu, ex.vmin, o);
    b.vmax = __shfl_xor_sync(0xffffffffu, ex.vmax, o);
    b.amin = __shfl_xor_sync(0xffffffffu, ex.amin, o);
    b.amax = __shfl_xor_sync(0xffffffffu, ex.amax, o);
    ext_merge(ex, b);
  }
}

__device__ __forceinline__ Extreme ext_empty() {
  Extreme ex;
  ex.vmin = LLONG_MAX;
  ex.vmax = LLONG_MIN;
  ex.amin = ex.amax = ~0ull;
  return ex;
}

template <int LB>
__global__ void __launch_bounds__(1 << (LB - 5))
cost_block_kernel(int n, const int32_t* __restrict__ wmat, int32_t* __restrict__ diag, Extreme* __restrict__ out) {
  constexpr int NT = 1 << (LB - 5);
  __shared__ int w[kMaxBits * kMaxBits];
  __shared__ int delta[LB];
  __shared__ int base_s;
  __shared__ int clow[32];
  __shared__ int dsum[5];
  __shared__ Extreme red[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n * n; i += NT) w[i] = wmat[i];
  __syncthreads();
  const unsigned long long hi = (unsigned long long)blockIdx.x << LB;
  if (warp == 0) {
    int a = 0;
    if (lane < LB) {
      int d = 0;
      for (int g = LB; g < n; ++g) {
        const int fg = int(hi >> g & 1ull), wg = w[lane * n + g];
        d += fg ? -wg : wg;
        a += fg ? wg : 0;
      }
      delta[lane] = d;
    }
    int cf = 0;
    for (int g = LB + lane; g < n; g += 32) {
      const int fg = int(hi >> g & 1ull);
      for (int h = g + 1; h < n; ++h)
        if (fg != int(hi >> h & 1ull)) cf += w[g * n + h];
    }
    int tot = a + cf;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) base_s = tot;
    // C_low(j) over bits 0..4 and D_i
    int cl = 0;
    for (int i = 0; i < 5; ++i)
      for (int k = i + 1; k < 5; ++k)
        if ((lane >> i & 1) != (lane >> k & 1)) cl += w[i * n + k];
    clow[lane] = cl;
    if (lane < 5) {
      int d = 0;
      for (int k = 5; k < LB; ++k) d += w[lane * n + k];
      dsum[lane] = d;
    }
  }
  __syncthreads();
  const int t = tid;  // bits 5..LB-1
  int kappa = base_s;
  for (int k = 5; k < LB; ++k) {
    const int tk = t >> (k - 5) & 1;
    if (tk) kappa += delta[k];
    for (int l = k + 1; l < LB; ++l)
      if (tk != (t >> (l - 5) & 1)) kappa += w[k * n + l];
  }
  int e[5];
  for (int i = 0; i < 5; ++i) {
    int ai = 0;
    for (int k = 5; k < LB; ++k)
      if (t >> (k - 5) & 1) ai += w[i * n + k];
    kappa += ai;
    e[i] = delta[i] + dsum[i] - 2 * ai;
  }
  Extreme ex = ext_empty();
  const unsigned long long x0 = hi | ((unsigned long long)t << 5);
  int vals[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    int c = kappa + clow[j];
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (j >> i & 1) c += e[i];
    vals[j] = c;
    if (c < ex.vmin) { ex.vmin = c; ex.amin = x0 | j; }
    if (c > ex.vmax) { ex.vmax = c; ex.amax = x0 | j; }
  }
  if (diag) {
    int4* d4 = reinterpret_cast<int4*>(diag + x0);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      __stcg(d4 + j, make_int4(vals[4 * j], vals[4 * j + 1], vals[4 * j + 2], vals[4 * j + 3]));
  }
  ext_warp_merge(ex);
  if (lane == 0) red[warp] = ex;
  __syncthreads();
  if (tid == 0) {
    Extreme r = red[0];
    for (int i = 1; i < NT / 32; ++i) ext_merge(r, red[i]);
    out[blockIdx.x] = r;
  }
}

// Per-tile constants of the pass kernels' C(x) tables (the quantities of
// tile_consts in device.cuh) for every tile of one sub-pass, one thread per
// tile. Tile t (kernel order: unit = t >> ninner, inner index t & (2^ninner-1))
// has fixed index bits gbase = outer(unit) | inner(t); its row holds
//   delta_j = sum_{g fixed} w[pos_j][g] (1 - 2 f_g)      at [j], j < T
//   base    = sum_{g<h fixed} w_gh [f_g != f_h] + sum_j sum_{g fixed} w[pos_j][g] f_g   at [15]
// so that C(x) = base + sum_j t_j delta_j + C_tile(t) for tile index t.
struct TileConstArgs {
  int8_t pos[16];
  BitRuns outer, inner;
  int T, n, ninner;
  uint64_t ntiles;
  const int32_t* wmat;
  int32_t* out;
};

// Tiles per thread of tile_const_table_kernel: a thread visits the tiles
// t0 | gray(k), k < 2^kTileConstRunBits, so consecutive tiles differ in one
// index bit and the row is updated in O(n) instead of recomputed in O(n^2).
constexpr int kTileConstRunBits = 6;

static __global__ void __launch_bounds__(256) tile_const_table_kernel(const TileConstArgs a) {
  __shared__ int32_t w[kMaxBits * kMaxBits];
  const int n = a.n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) w[i] = a.wmat[i];
  __syncthreads();
  const uint64_t t0 = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) << kTileConstRunBits;
  if (t0 >= a.ntiles) return;
  auto gbase_of = [&](uint64_t t) {
    return a.outer.scatter(t >> a.ninner) | a.inner.scatter(t & ((1ull << a.ninner) - 1));
  };
  uint64_t tbits = 0;
  for (int j = 0; j < a.T; ++j) tbits |= 1ull << a.pos[j];
  // first tile of the run: the definitions
  uint64_t gbase = gbase_of(t0);
  int32_t row[kTileConstInts];
#pragma unroll
  for (int i = 0; i < kTileConstInts; ++i) row[i] = 0;
  int base = 0;
#pragma unroll
  for (int j = 0; j < kTileConstInts - 1; ++j) {
    if (j >= a.T) break;
    const int* wr = w + a.pos[j] * n;
    int d = 0;
    for (int g = 0; g < n; ++g) {
      if (tbits >> g & 1ull) continue;
      if (gbase >> g & 1ull) { d -= wr[g]; base += wr[g]; } else { d += wr[g]; }
    }
    row[j] = d;
  }
  for (int g = 0; g < n; ++g) {
    if (tbits >> g & 1ull) continue;
    const uint64_t fg = gbase >> g & 1ull;
    for (int h = g + 1; h < n; ++h) {
      if (tbits >> h & 1ull) continue;
      if (fg != (gbase >> h & 1ull)) base += w[g * n + h];
    }
  }
  for (int k = 0; k < (1 << kTileConstRunBits); ++k) {
    if (k) {
      // flip the fixed index bit g of tile-index bit ctz(k)
      const int b = __ffs(k) - 1;
      const uint64_t gm = gbase_of(t0 | (1ull << b)) ^ gbase_of(t0);
      const int g = __ffsll((long long)gm) - 1;
      const bool was = (gbase >> g & 1ull) != 0;
      // pairs of fixed bits (g, h): [f_g != f_h] toggles
      int dpair = 0;
      for (int h = 0; h < n; ++h) {
        if (h == g || (tbits >> h & 1ull)) continue;
        const bool fh = (gbase >> h & 1ull) != 0;
        dpair += (fh != was) ? -w[g * n + h] : w[g * n + h];
      }
      base += dpair;
#pragma unroll
      for (int j = 0; j < kTileConstInts - 1; ++j) {
        if (j >= a.T) break;
        const int wjg = w[a.pos[j] * n + g];
        // delta_j: w (1 - 2 f_g) changes sign; base: w f_g toggles
        row[j] += was ? 2 * wjg : -2 * wjg;
        base += was ? -wjg : wjg;
      }
      gbase ^= 1ull << g;
    }
    const uint64_t t = t0 | uint64_t(k ^ (k >> 1));
    if (t >= a.ntiles) continue;
    row[15] = base;
    int4* o = reinterpret_cast<int4*>(a.out + t * kTileConstInts);
#pragma unroll
    for (int i = 0; i < kTileConstInts / 4; ++i)
      o[i] = make_int4(row[4 * i], row[4 * i + 1], row[4 * i + 2], row[4 * i + 3]);
  }
}

// Small n (< 15): one CTA, one thread per x, direct sum over all index pairs.
static __global__ void cost_small_kernel(int n, const int32_t* __restrict__ wmat, int32_t* __restrict__ diag,
                                  Extreme* __restrict__ out) {
  __shared__ Extreme red[32];
  const unsigned long long N = 1ull << n;
  Extreme ex = ext_empty();
  for (unsigned long long x = threadIdx.x; x < N; x += blockDim.x) {
    int c = 0;
    for (int g = 0; g < n; ++g)
      for (int h = g + 1; h < n; ++h)
        if ((x >> g & 1ull) != (x >> h & 1ull)) c += wmat[g * n + h];
    if (diag) diag[x] = c;
    if (c < ex.vmin) { ex.vmin = c; ex.amin = x; }
    if (c > ex.vmax) { ex.vmax = c; ex.amax = x; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ext_warp_merge(ex);
  if (lane == 0) red[warp] = ex;
  __syncthreads();
  if (threadIdx.x == 0) {
    Extreme r = red[0];
    for (int i = 1; i < (int)(blockDim.x / 32); ++i) ext_merge(r, red[i]);
    out[0] = r;
  }
}

// Merges per-block extremes (deterministic: ties go to the smallest index).
static __global__ void extreme_finalize_kernel(const Extreme* __restrict__ in, long long count, Extreme* __restrict__ out) {
  __shared__ Extreme red[32];
  Extreme ex = ext_empty();
  for (long long i = threadIdx.x; i < count; i += blockDim.x) ext_merge(ex, in[i]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ext_warp_merge(ex);
  if (lane == 0) red[warp] = ex;
  __syncthreads();
  if (threadIdx.x == 0) {
    Extreme r = red[0];
    for (int i = 1; i < (int)(blockDim.x / 32); ++i) ext_merge(r, red[i]);
    *out = r;
  }
}

// Sums `count` interleaved partials (stride `stride` doubles) in a fixed order.
static __global__ void sum_partials_kernel(const double* __restrict__ in, int count, int stride, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c < stride) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += in[(size_t)i * stride + c];
    out[c] = s;
  }
}

// ---------------------------------------------------------------------------
// Sampling (Sec. II-B: repeated measurement of the final state).
// Block sums S_j of |psi|^2 over 2^B consecutive indices; exclusive prefix
// E_j = S_0 + ... + S_{j-1} (E_nb = total); per shot t = u * total, block j =
// smallest with E_{j+1} > t, then the smallest x in the block whose in-block
// running FP64 sum exceeds t - E_j (the last nonzero-probability index of the
// block if rounding leaves none).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) block_sum_kernel(const typename Cx<Real>::T* __restrict__ psi, int B,
                                                        double* __restrict__ sums) {
  __shared__ double red[8];
  const size_t base = (size_t)blockIdx.x << B;
  const int len = 1 << B;
  // |psi_x|^2 formed and summed in FP64 exactly as the shot kernels' in-block
  // walk forms it, so a block sum and the walk over the same block differ only
  // by FP64 summation order
  double d = 0.0;
  for (int i = threadIdx.x; i < len; i += 256) {
    const typename Cx<Real>::T a = __ldcg(psi + base + i);
    d += double(a.x) * double(a.x) + double(a.y) * double(a.y);
  }
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < 8; ++i) t += red[i];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of `count` doubles into pre[0..count] (pre[count] = total),
// one CTA of 1024 threads, fixed order: each thread scans a contiguous chunk.
static __global__ void __launch_bounds__(1024) scan_kernel(const double* __restrict__ s, long long count,
                                                    double* __restrict__ pre) {
  __shared__ double part[1024];
  const long long chunk = (count + 1023) / 1024;
  const long long lo = threadIdx.x * chunk;
  const long long hi = lo + chunk < count ? lo + chunk : count;
  double acc = 0.0;
  for (long long i = lo; i < hi; ++i) acc += s[i];
  // exclusive prefix of the 1024 chunk sums: warp scans, then a scan of the
  // 32 warp totals (fixed order)
  __shared__ double wtot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double x = acc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double w = wtot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wtot[lane] = w;  // inclusive
    if (lane == 31) pre[count] = w;
  }
  __syncthreads();
  part[threadIdx.x] = (warp ? wtot[warp - 1] : 0.0) + (x - acc);
  __syncthreads();
  double run = part[threadIdx.x];
  for (long long i = lo; i < hi; ++i) { pre[i] = run; run += s[i]; }
}

// Multi-CTA exclusive scan for long block-sum arrays. Level 1: CTA b takes
// s[b * 4096 ..) (each thread 8 consecutive values, then warp and block
// prefixes, a fixed order), writes the chunk-local exclusive prefix to pre and
// its total to tot[b]. Level 2 scans tot with scan_kernel; level 3 adds the
// chunk offsets and sets pre[count] = total.
constexpr int kScanChunk = 4096;
static __global__ void __launch_bounds__(512) scan_chunk_kernel(const double* __restrict__ s, long long count,
                                                                 double* __restrict__ pre, double* __restrict__ tot) {
  __shared__ double buf[kScanChunk + kScanChunk / 32];
  __shared__ double wsum[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long base = (long long)blockIdx.x * kScanChunk;
  auto slot = [](int i) { return i + (i >> 5); };  // padding: 8 consecutive values per thread without conflicts
  for (int k = 0; k < 8; ++k) {
    const int i = k * 512 + tid;
    buf[slot(i)] = base + i < count ? s[base + i] : 0.0;
  }
  __syncthreads();
  double v[8], run = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = run; run += buf[slot(tid * 8 + k)]; }
  double x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (tid == 0) {
    double r = 0.0;
    for (int w = 0; w < 16; ++w) { const double t = wsum[w]; wsum[w] = r; r += t; }
    tot[blockIdx.x] = r;
  }
  __syncthreads();
  const double off = wsum[warp] + (x - run);
#pragma unroll
  for (int k = 0; k < 8; ++k) buf[slot(tid * 8 + k)] = off + v[k];
  __syncthreads();
  for (int k = 0; k < 8; ++k) {
    const int i = k * 512 + tid;
    if (base + i < count) pre[base + i] = buf[slot(i)];
  }
}

static __global__ void scan_offset_kernel(double* __restrict__ pre, long long count, const double* __restrict__ pre2,
                                          long long nchunks) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) pre[i] += pre2[i / kScanChunk];
  if (i == 0) pre[count] = pre2[nchunks];
}

// Draw k of the SplitMix64 stream `seed` (Steele, Lea and Flood 2014):
// mix(seed + (k+1) * golden gamma).
__device__ __forceinline__ unsigned long long splitmix_draw(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The same draw as a double in [0, 1): its top 53 bits times 2^-53.
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long k) {
  return double(splitmix_draw(seed, k) >> 11) * 0x1.0p-53;
}

template <typename Real>
__global__ void shot_kernel(const typename Cx<Real>::T* __restrict__ psi, int B, const double* __restrict__ pre,
                            long long nb, int shots, const double* __restrict__ uni, unsigned long long seed,
                            unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= shots) return;
  const double u = uni ? uni[i] : splitmix_uniform(seed, (unsigned long long)i);
  const double total = pre[nb];
  const double t = u * total;
  // smallest j with pre[j + 1] > t
  long long lo = 0, hi = nb;
  while (lo < hi) {
    const long long mid = lo + (hi - lo) / 2;
    if (pre[mid + 1] > t) hi = mid; else lo = mid + 1;
  }
  long long j = lo;
  if (j >= nb) {  // rounding pushed t to the total: last block with mass
    j = nb - 1;
    while (j > 0 && !(pre[j + 1] > pre[j])) --j;
  }
  const double tr = t - pre[j];
  const size_t base = (size_t)j << B;
  const int len = 1 << B;
  double run = 0.0;
  long long pick = -1, last_nz = 0;
  for (int k = 0; k < len; ++k) {
    const typename Cx<Real>::T a = psi[base + k];
    const double pr = double(a.x) * double(a.x) + double(a.y) * double(a.y);
    run += pr;
    if (pr > 0.0) last_nz = k;
    if (run > tr) { pick = k; break; }
  }
  if (pick < 0) pick = last_nz;
  out[i] = (unsigned long long)(base + pick);
}

// One warp per shot: the same block and in-block rules as shot_kernel, with a
// 32-way search over the prefix array (identical answer: the predicate
// pre[j + 1] > t is monotone in j) and the in-block running sum taken 32
// amplitudes at a time (warp prefix sums; a different FP64 summation order
// inside the block than the sequential loop).
template <typename Real>
__global__ void __launch_bounds__(128) shot_warp_kernel(const typename Cx<Real>::T* __restrict__ psi, int B,
                                                        const double* __restrict__ pre, long long nb, int shots,
                                                        const double* __restrict__ uni, unsigned long long seed,
                                                        unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= shots) return;
  const double u = uni ? uni[i] : splitmix_uniform(seed, (unsigned long long)i);
  const double total = pre[nb];
  const double t = u * total;
  // smallest j in [lo, hi) with pre[j + 1] > t, or hi if none; the answer
  // stays in [lo, hi]. Pivot lane i tests "answer <= lo + i step", which holds
  // for every pivot at or beyond hi (the answer is at most hi), so the first
  // pivot that holds bounds the answer from above and its predecessor from
  // below, also when the last pivots fall beyond hi
  long long lo = 0, hi = nb;
  while (hi - lo > 32) {
    const long long step = (hi - lo + 31) / 32;
    const long long piv = lo + (long long)lane * step;  // lane 0's pivot is lo
    const bool f = piv >= hi || pre[piv + 1] > t;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int k = m ? __ffs(m) - 1 : 32;      // first pivot where the predicate holds
    const long long nlo = k == 0 ? lo : lo + (long long)(k - 1) * step + 1;
    const long long nhi = k == 32 ? hi : lo + (long long)k * step;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
  }
  {
    const long long piv = lo + lane;
    const bool f = piv < hi && pre[piv + 1] > t;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    lo = m ? lo + __ffs(m) - 1 : hi;
  }
  long long j = lo;
  if (j >= nb) {  // rounding pushed t to the total: last block with mass
    j = nb - 1;
    while (j > 0 && !(pre[j + 1] > pre[j])) --j;
  }
  const double tr = t - pre[j];
  const size_t base = (size_t)j << B;
  const int len = 1 << B;
  double carry = 0.0;
  long long pick = -1, last_nz = 0;
  for (int k0 = 0; k0 < len; k0 += 32) {
    const int k = k0 + lane;
    double pr = 0.0;
    if (k < len) {
      const typename Cx<Real>::T a = __ldcg(psi + base + k);
      pr = double(a.x) * double(a.x) + double(a.y) * double(a.y);
    }
    double x = pr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned nz = __ballot_sync(0xffffffffu, pr > 0.0);
    if (nz) last_nz = k0 + 31 - __clz(nz);
    const unsigned hit = __ballot_sync(0xffffffffu, carry + x > tr);
    if (hit) { pick = k0 + __ffs(hit) - 1; break; }
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (pick < 0) pick = last_nz;
  if (lane == 0) out[i] = (unsigned long long)(base + pick);
}

}  // namespace qaoa
