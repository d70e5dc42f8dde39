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
  uint8_t mixA, cost, mixB, reduce, src, dst;
  uint8_t lam;   // adjoint: load psi only and create lambda = C(x) psi first
  uint8_t pad;
  int32_t ctab;  // offset (in ints) of this round's cost tables, -1 if none
};

struct SubDev {
  int8_t pos[16];          // tile bit -> global index bit
  int8_t inner[kMaxBits];  // global bits enumerating tiles inside a super-tile
  int32_t ninner;
  int32_t nrounds;
  double scale;            // product of butterfly normalisations applied here
  uint8_t init, needs_c, store, pad[5];
  RoundDev rd[kMaxRoundsDev];
};

struct PassDev {
  int32_t n, T, nsub, nouter;
  int8_t outer[kMaxBits];  // global bits enumerating super-tiles
  uint64_t n_units;        // number of super-tiles
  double tauA, alphaA;     // mixer of layer a: a' = alpha a + i tau b
  double tauB, alphaB;     // mixer of layer b (after the cost phase)
  double amp0;             // 2^(-n/2)
  int32_t c_lo;            // smallest possible C(x) (phase-table origin)
  int32_t ncost;           // phase-table length
  int32_t wsum;            // W = sum of the weights (h(x) = W - 2 C(x))
  int32_t pad0;
  double cA, cB;           // cos(beta) of layers a / b (adjoint per-round rescaling)
  SubDev sub[kMaxSubDev];
};

// Scatters the bits of `idx` onto the global bit positions `pos[0..k-1]`.
__device__ __forceinline__ uint64_t scatter_bits(uint64_t idx, const int8_t* pos, int k) {
  uint64_t g = 0;
  for (int i = 0; i < k; ++i) g |= ((idx >> i) & 1ull) << pos[i];
  return g;
}

template <typename Real> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// Shared-memory XOR swizzle over tile indices. For 8-byte amplitudes the
// bank group of a half-warp access is (index mod 16); bits 4k..4k+3 are folded
// onto bits 0..3, so tile bit j lands in class j mod 4. For 16-byte
// amplitudes a quarter-warp covers 8 slots; bits are folded in groups of 3,
// giving class j mod 3. The map is linear over XOR, so
// swz(a | b) = swz(a) ^ swz(b) for disjoint a, b.
template <int AMP_BYTES>
__device__ __forceinline__ uint32_t swz(uint32_t t) {
  if (AMP_BYTES == 8) return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u);
  return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7u);
}

// Per-tile constants over the fixed (non-tile) index bits F, computed by one
// warp into tconst[0..T-1] (delta) and tconst[16] (base):
//   delta_j = sum_{g in F} w[pos_j][g] (1 - 2 f_g)
//   base    = C restricted to F + sum_j sum_{g in F} w[pos_j][g] f_g
// so that C(x) = base + sum_j t_j delta_j + C_tile(t) for tile index t.
template <int T>
__device__ __forceinline__ void tile_consts(const int8_t* pos, uint64_t gbase, const int* wsm, int n, int* tconst,
                                            int lane) {
  uint64_t tbits = 0;
  for (int j = 0; j < T; ++j) tbits |= 1ull << pos[j];
  int a = 0;
  if (lane < T) {
    const int pj = pos[lane];
    int d = 0;
    for (int g = 0; g < n; ++g) {
      if (tbits >> g & 1ull) continue;
      const int wg = wsm[pj * n + g];
      const int fg = int(gbase >> g & 1ull);
      d += fg ? -wg : wg;
      a += fg ? wg : 0;
    }
    tconst[lane] = d;
  }
  int cf = 0;
  for (int g = lane; g < n; g += 32) {
    if (tbits >> g & 1ull) continue;
    const int fg = int(gbase >> g & 1ull);
    for (int h = g + 1; h < n; ++h) {
      if (tbits >> h & 1ull) continue;
      if (fg != int(gbase >> h & 1ull)) cf += wsm[g * n + h];
    }
  }
  int tot = a + cf;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (lane == 0) tconst[16] = tot;
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
  __device__ __forceinline__ int operator()(int j) const {
    int c = kappa + __ldg(cp + j);
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (j >> i & 1) c += e[i];
    return c;
  }
};

}  // namespace qaoa
