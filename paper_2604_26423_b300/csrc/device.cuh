// device.cuh -- device-side plan structures and helpers shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qaoa {

constexpr int kMaxRoundsDev = 8;
constexpr int kMaxSubDev = 4;
constexpr int kMaxBits = 40;

// One round of a sub-pass (see plan.h): register / lane / warp tile bits,
// ops, and the offset of its precomputed cost tables.
struct RoundDev {
  int8_t reg[5], lane[5], warp[4];
  int8_t greg[5], glane[5], gwarp[4];  // global index bits of reg / lane / warp tile bits
  uint8_t mixA, cost, mixB, reduce, src, dst;
  uint8_t lam;     // adjoint: load psi only and create lambda = C(x) psi first
  uint8_t layout;  // menu layout id (plan.h, menu_layout)
  int32_t ctab;  // offset (in ints) of this round's cost tables, -1 if none
  int32_t gtab;  // offset (in ints, even) of this round's per-thread geometry:
                 // padded shared-memory slot (NT ints; bit 31 holds the parity
                 // of the thread's global index offset), then the global index
                 // offset of the thread's lane and warp bits (NT 64-bit words)
};

// Contiguous runs of a sorted bit list: bits [src, src+len) of an index go to
// global bits [dst, dst+len).
struct BitRuns {
  int8_t src[6], dst[6], len[6];
  int8_t n;
  __device__ __forceinline__ uint64_t scatter(uint64_t idx) const {
    uint64_t g = 0;
    for (int i = 0; i < n; ++i) g |= ((idx >> src[i]) & ((1ull << len[i]) - 1)) << dst[i];
    return g;
  }
};

struct SubDev {
  int8_t pos[16];          // tile bit -> global index bit
  int8_t inner[kMaxBits];  // global bits enumerating tiles inside a super-tile
  BitRuns inner_runs;
  int32_t ninner;
  int32_t nrounds;
  double scale;            // product of butterfly normalisations applied here
  uint8_t init, needs_c, store, keep, pad[4];  // keep: a later sub-pass reads this one's output
  float fscale;            // scale rounded to fp32 (complex64 kernels)
  int32_t rescale;         // scale != 1
  // per-tile constants of the C(x) tables, one row of kTileConstInts ints per
  // tile in the kernel's order (unit * 2^ninner + tile): delta_j for tile bit
  // j at [j], the fixed-bit base at [15]; nullptr: computed in the kernel
  const int32_t* tct;
  // asynchronous tile copy (complex64 kernels, one tile per super-tile):
  // offset of the per-thread geometry table of the copy mapping (lanes on
  // tile bits 0..4, warps on the next WB bits, one amplitude per 8-byte
  // copy), -1 if the sub-pass is not copied asynchronously
  int32_t cgtab;
  // complex64 storage between passes (see swapped storage in pass_kernel.cuh):
  // the sub-pass reads plain (re, im) amplitudes (ld_plain: the adjoint's first
  // sub-pass) or writes them (st_plain: a forward run's last sub-pass)
  uint8_t ld_plain, st_plain, pad2[2];
  RoundDev rd[kMaxRoundsDev];
};

constexpr int kTileConstInts = 16;
// shared-memory ints reserved for the tile constants (two buffers of 32:
// delta[0..15], base at [16])
constexpr int kTconstSmemInts = 64;

struct PassDev {
  int32_t n, T, nsub, nouter;
  int8_t outer[kMaxBits];  // global bits enumerating super-tiles
  BitRuns outer_runs;
  uint64_t n_units;        // number of super-tiles
  double tauA, alphaA;     // mixer of layer a: a' = alpha a + i tau b
  double tauB, alphaB;     // mixer of layer b (after the cost phase)
  double amp0;             // 2^(-n/2)
  int32_t c_lo;            // smallest possible C(x) (phase-table origin)
  int32_t ncost;           // phase-table length
  int32_t wsum;            // W = sum of the weights (h(x) = W - 2 C(x))
  int32_t pad0;
  double cA, cB;           // cos(beta) of layers a / b (adjoint per-round rescaling)
  float ftauA, falphaA, ftauB, falphaB, fcA, fcB;  // the same rounded to fp32
  // cost phase of the pass's cost layer as 64-bit fixed-point turns:
  // exp(-i gamma s (W - 2c)) = exp(2 pi i (ph0 + (c - c_lo) ph1) / 2^64)
  uint64_t ph0, ph1;
  float famp0;             // amp0 rounded to fp32
  int32_t pad1;
  // register-pair part CP[j] of C(x) (see RoundCost) for the pass's cost round
  // (cpc) and reduction round (cpr), and cpt[j] = top 32 bits of CP[j] ph1 mod
  // 2^64 (the cost round's phase increment in 2^-32 turns); in the parameter
  // space, so the kernels take them as constant operands
  int32_t cpc[32], cpr[32];
  uint32_t cpt[32];
  SubDev sub[kMaxSubDev];
};

// Scatters the bits of `idx` onto the global bit positions `pos[0..k-1]`.
__device__ __forceinline__ uint64_t scatter_bits(uint64_t idx, const int8_t* pos, int k) {
  uint64_t g = 0;
  for (int i = 0; i < k; ++i) g |= ((idx >> i) & 1ull) << pos[i];
  return g;
}

// L2 eviction-priority hints (per access; no device setting is changed).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float2 ld_hint(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_hint(const double2* a, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(double2* a, double2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(a), "d"(v.x), "d"(v.y), "l"(pol) : "memory");
}

// Asynchronous global -> shared copies of 8 bytes (both addresses 8-byte
// aligned), committed as one group per tile; the consumer waits for all of them.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// fp32 kernels take the host-rounded fp32 copies of the pass coefficients (no
// fp64 conversions in the kernels); fp64 kernels the doubles.
template <typename Real> __device__ __forceinline__ Real pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

constexpr float kTurn32 = 1.46291807926715968e-9f;  // 2 pi / 2^32

// exp(2 pi i t / 2^32) for a 32-bit turn count t (the signed angle in [-pi,
// pi)); k = -kTurn32 gives the conjugate (the sine's sign flipped exactly).
__device__ __forceinline__ float2 phase_turns32(uint32_t t, float k = kTurn32) {
  const float ang = float(int32_t(t)) * k;
  float sn, cs;
  __sincosf(ang, &sn, &cs);
  return make_float2(cs, sn);
}

// exp(2 pi i t / 2^64) for the turn count t = ph0 + u ph1 (mod 2^64), u >= 0:
// the top 32 bits of t as a signed angle in [-pi, pi), then the hardware sine
// and cosine (absolute error about 4e-7, below the complex64 state's rounding
// over a layer). Only the top word of the product is formed.
__device__ __forceinline__ float2 phase_turns(uint64_t ph0, uint64_t ph1, uint32_t u, float k = kTurn32) {
  const uint64_t lo = (uint64_t)u * (uint32_t)ph1 + (uint32_t)ph0;
  const uint32_t hi = (uint32_t)(ph0 >> 32) + u * (uint32_t)(ph1 >> 32) + (uint32_t)(lo >> 32);
  return phase_turns32(hi, k);
}

// Scales both components of an amplitude (packed for complex64).
__device__ __forceinline__ void scale_amp(float2& v, float s) { v = __fmul2_rn(v, make_float2(s, s)); }
__device__ __forceinline__ void scale_amp(double2& v, double s) { v.x *= s; v.y *= s; }

template <typename Real> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// Padded shared-memory slot of tile index t. For 8-byte amplitudes a
// half-warp access is conflict-free when the 16 slots are distinct mod 16;
// padi adds t >> 4 and t >> 8, so tile bit j shifts the slot by 2^(j mod 4)
// mod 16 for j < 12. For 16-byte amplitudes a quarter-warp covers 8 slots and
// the fold is by 3 bits (class j mod 3). Lanes 0..3 (0..2) on bits of distinct
// classes therefore never share a bank. padi is additive over disjoint bit
// sets (no carries), so padi(a | b) = padi(a) + padi(b): register offsets are
// compile-time constants.
template <int AB>
__host__ __device__ constexpr uint32_t padi(uint32_t t) {
  return AB == 8 ? t + (t >> 4) + (t >> 8) : t + (t >> 3) + (t >> 6) + (t >> 9) + (t >> 12);
}
template <int AB>
__host__ __device__ constexpr uint32_t padded_size(int T) {
  return padi<AB>((1u << T) - 1) + 1;
}

// Per-tile constants over the fixed (non-tile) index bits F, computed by all
// warps of the CTA into tconst[0..T-1] (delta) and tconst[16] (base):
//   delta_j = sum_{g in F} w[pos_j][g] (1 - 2 f_g)
//   base    = C restricted to F + sum_j sum_{g in F} w[pos_j][g] f_g
// so that C(x) = base + sum_j t_j delta_j + C_tile(t) for tile index t.
// Warp k takes tile bits j = k, k + nwarps, ... and rows g = k, k + nwarps, ...
// of the fixed-bit pairs; lanes split the inner sums; base is accumulated with
// shared-memory atomics, so tconst[16] must be zero on entry and a barrier
// must separate this call from the first use.
template <int T>
__device__ __forceinline__ void tile_consts(const int8_t* pos, uint64_t gbase, const int* __restrict__ w, int n,
                                            int* tconst, int lane, int warp, int nwarps) {
  uint64_t tbits = 0;
  for (int j = 0; j < T; ++j) tbits |= 1ull << pos[j];
  int base = 0;
  for (int j = warp; j < T; j += nwarps) {
    const int pj = pos[j];
    int d = 0, a = 0;
    for (int g = lane; g < n; g += 32) {
      if (tbits >> g & 1ull) continue;
      const int wg = __ldg(w + pj * n + g);
      const int fg = int(gbase >> g & 1ull);
      d += fg ? -wg : wg;
      a += fg ? wg : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if (lane == 0) tconst[j] = d;
    base += a;  // identical in every lane after the reduction
  }
  int cf = 0;
  for (int g = warp; g < n; g += nwarps) {
    if (tbits >> g & 1ull) continue;
    const int fg = int(gbase >> g & 1ull);
    for (int h = g + 1 + lane; h < n; h += 32) {
      if (tbits >> h & 1ull) continue;
      if (fg != int(gbase >> h & 1ull)) cf += __ldg(w + g * n + h);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cf += __shfl_xor_sync(0xffffffffu, cf, o);
  if (lane == 0 && (base | cf)) atomicAdd(tconst + 16, base + cf);
}

// C(x) of the 2^R register amplitudes of a round from its host-built tables:
//   C(j) = kappa + CP[j] + sum_{i: j_i = 1} e_i
// with kappa and e_i depending on the thread's lane / warp bits (see api.cu).
template <int R, int WB>
struct RoundCost {
  int kappa;
  int e[R];
  const int* cp;
  __device__ __forceinline__ void setup(const int* tab, const int* tconst, const int8_t* lanebits,
                                        const int8_t* warpbits, const int8_t* regbits, int lane, int warp) {
    constexpr int QN = 1 << (5 + WB);
    const int q = lane | (warp << 5);
    kappa = tconst[16] + __ldg(tab + q);
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (lane >> i & 1) kappa += tconst[lanebits[i]];
#pragma unroll
    for (int i = 0; i < WB; ++i)
      if (warp >> i & 1) kappa += tconst[warpbits[i]];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int aj = __ldg(tab + QN + q * R + i);
      kappa += aj;
      e[i] = tconst[regbits[i]] + __ldg(tab + QN + QN * R + i) - 2 * aj;
    }
    cp = tab + QN + QN * R + R;
  }
  // Phase increments in 2^-32 turns for the cost layer with turn constants
  // (ph0, ph1) (see PassDev): returns t0 = top32(ph0 + (kappa - c_lo) ph1) and
  // E[i] = top32(e_i ph1) (products mod 2^64), so that the 32-bit turn count
  // of register amplitude j is t0 + sum_{i: j_i = 1} E[i] + cpt[j]. Against the
  // exact top32(ph0 + (C(j) - c_lo) ph1) it lacks the carries of the dropped
  // low words: 0 to 6 units of 2^-32 turns (below 1e-8 rad).
  __device__ __forceinline__ uint32_t turns(uint64_t ph0, uint64_t ph1, int c_lo, uint32_t* E) const {
#pragma unroll
    for (int i = 0; i < R; ++i) E[i] = uint32_t(((uint64_t)(int64_t)e[i] * ph1) >> 32);
    return uint32_t((ph0 + (uint64_t)(int64_t)(kappa - c_lo) * ph1) >> 32);
  }
  __device__ __forceinline__ int operator()(int j) const {
    int c = kappa + __ldg(cp + j);
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (j >> i & 1) c += e[i];
    return c;
  }
};

}  // namespace qaoa
