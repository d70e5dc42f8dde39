// desc.h -- host-side construction of the device pass descriptors (PassDev)
// and of their per-round cost tables, shared by the single-instance API and the
// batched launcher.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "device.cuh"
#include "plan.h"

namespace qaoa {

// Per-round cost tables (recompute mode), deduplicated by (shape, tile bits,
// register / lane / warp split). Offsets are in ints from the start of `h`.
struct TableStore {
  std::vector<int32_t> h;
  std::map<std::pair<int, std::vector<int8_t>>, int32_t> index;
  bool dirty = false;
  // Offset of the tables for a round of shape `sh` over tile bits `pos`, built
  // from the n x n weight matrix `wmat` on first use.
  int32_t offset(const int32_t* wmat, int n, const TileShape& sh, const int8_t* pos, const RoundDev& rd);
  // Offset (even) of the per-thread geometry table of a round over tile bits
  // `pos`: NT padded shared-memory slots (bit 31: parity of the thread's
  // global index offset), then NT 64-bit global offsets.
  int32_t geom_offset(const TileShape& sh, const int8_t* pos, const RoundDev& rd);
  void clear() { h.clear(); index.clear(); dirty = false; }
};

// Validates a weighted graph (vertices in [0, n), no self loops or repeated
// edges, nonzero weights, sum |w| <= max_abs) and builds its n x n weight
// matrix, W = sum w, and the cut-value range [c_lo, c_hi] (sums of the
// negative and of the positive weights). Returns "" or the first violation.
std::string check_graph(int n, int m, const int32_t* u, const int32_t* v, const int32_t* w, long long max_abs,
                        std::vector<int32_t>& wmat, long long& W, long long& c_lo, long long& c_hi);

// Offset of the per-thread geometry table of the asynchronous tile copy
// (complex64): lanes on tile bits 0..4, warps on tile bits 5..4+WB (see
// tile_copy_async in pass_kernel.cuh).
int32_t copy_geom_offset(TableStore& tabs, const TileShape& sh, const int8_t* pos);

// Contiguous runs of a sorted bit list.
BitRuns make_runs(const std::vector<int>& bits);

// Mixer exp(+i beta X) as a' = alpha a + i tau b: (cos, sin), or the fast form
// (1, tan) with the cos^k rescaling applied once per sub-pass.
void mixer_coeffs(double beta, bool fast, double* tau, double* alpha);

// What a pass descriptor needs besides its plan.
struct PassInputs {
  int n = 0;
  const double* beta = nullptr;   // beta_k per layer
  const double* gamma = nullptr;  // gamma_k per layer (phase constants of the cost layer)
  double scale = 0.1;             // phase weight scale s
  long long c_lo = 0, ncost = 1;  // phase-table origin and length
  long long W = 0;                // sum of the weights
  const int32_t* wmat = nullptr;  // n x n weights (host)
  bool stream = false;            // int32 diagonal instead of cost tables
  bool adjoint = false;
  bool plain = false;             // never use the fast (tan) mixer form
};

// Fills `pd` for pass `pp` of a plan with tile shape `sh`; returns "" or the
// reason the pass does not fit the device descriptor. `fast` receives the
// mixer form chosen for the pass.
std::string fill_pass_dev(const PassPlan& pp, const TileShape& sh, const PassInputs& in, TableStore& tabs,
                          PassDev& pd, bool& fast);

}  // namespace qaoa
