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
  uint8_t pad[2];
  int32_t ctab;  // offset (in ints) of this round's cost tables, -1 if none
};

struct SubDev {
  int8_t pos[16];          // tile bit -> global index bit
  int8_t inner[kMaxBits];  // global bits enumerating tiles inside a super-tile
  int32_t ninner;
  int32_t nrounds;
  double scale;            // product of butterfly normalisations applied here
  uint8_t init, needs_c, pad[6];
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

}  // namespace qaoa
