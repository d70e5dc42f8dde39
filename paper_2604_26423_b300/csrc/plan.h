// plan.h -- host-side pass planner for the LR-QAOA state-vector kernels.
//
// A run of p layers (Sec. II-B: U_C(gamma_k) then U_B(beta_k) per layer) is
// executed as a sequence of HBM passes. Each pass streams the whole state once
// (one read and one write per amplitude) and applies, inside on-chip tiles,
// every gate that can be applied between that read and that write:
//   - the mixer exp(i beta X_q) of a layer on one group of qubits (the mixer is
//     a product over qubits of commuting 2x2 rotations, so any grouping works),
//   - the diagonal cost phase of the next layer, which needs the full index
//     of each amplitude but no neighbours,
//   - the mixer of that next layer on the same group (cross-layer fusion: the
//     group order is reversed on alternate layers so consecutive layers meet on
//     the same group).
// Inside a pass the state is processed in super-tiles (2^S amplitudes spanning
// S chosen index bits, small enough that all super-tiles in flight stay in L2).
// A super-tile is swept by one CTA in one or more sub-passes; a sub-pass moves
// shared-memory tiles of 2^T amplitudes (T = R + 5 + WB index bits: R bits in
// each thread's registers, 5 bits across lanes, WB bits across warps) between
// global memory and registers, and between rounds through shared memory.
// Bit q of an amplitude index is qubit q.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace qaoa {

constexpr int kMaxT = 14;
constexpr int kMaxRounds = 8;
constexpr int kMaxQubits = 40;

enum : uint8_t { SRC_SMEM = 0, SRC_GLOBAL = 1, SRC_INIT = 2 };
enum : uint8_t { DST_SMEM = 0, DST_GLOBAL = 1 };

// Kernel shape: R register bits, 5 lane bits, WB warp bits; amplitude bytes.
struct TileShape {
  int R = 5, WB = 3, amp_bytes = 8, nvec = 1;
  // the menu offers the paired global layout (id 4: register bit 0 on tile bit
  // 0, so each thread moves two adjacent 8-byte amplitudes per 16-byte access)
  bool paired = false;
  // among equally short round sequences, a paired storing last round counts
  // more than a paired loading first round (tiles that arrive by tensor
  // loads into shared memory: their first round issues no global loads)
  bool paired_store_first = false;
  int T() const { return R + 5 + WB; }
};

// One round: every thread holds 2^R amplitudes whose tile indices differ in the
// tile bits reg[0..R-1]; lanes and warps select the other bits.
struct RoundPlan {
  int8_t reg[5] = {0, 0, 0, 0, 0};
  int8_t lane[5] = {0, 0, 0, 0, 0};
  int8_t warp[4] = {0, 0, 0, 0};
  uint8_t mixA = 0;   // register-position mask: mixer of layer a on these bits
  uint8_t cost = 0;   // then the cost phase of layer b (all of layer a done)
  uint8_t mixB = 0;   // then the mixer of layer b on these register bits
  uint8_t reduce = 0; // then accumulate norm and <C> (final pass)
  uint8_t lam = 0;    // adjoint: load psi only and set lambda = C(x) psi first
  uint8_t src = SRC_SMEM, dst = DST_SMEM;
  uint8_t layout = 0; // menu layout id (see menu_layout)
  bool global_facing = false;
};

struct SubPassPlan {
  int T = 0;
  int8_t pos[kMaxT] = {};               // tile bit j -> global index bit pos[j]
  std::vector<RoundPlan> rounds;
  int nA = 0, nB = 0;                   // butterflies per amplitude of layer a / b here
  bool init = false;                    // first sub-pass of the first pass
  bool linit = false;                   // adjoint: first sub-pass creates lambda = C psi
  bool store = true;                    // the last round writes its tile back
  bool needs_c = false;                 // some round needs C(x) (cost, reduce, lambda)
};

struct PassPlan {
  std::vector<int> sb;                  // super-tile bits (ascending)
  std::vector<int> outer;               // bits enumerating super-tiles (ascending)
  std::vector<int> targets;             // qubits whose mixer this pass applies
  std::vector<SubPassPlan> subs;
  int layer_a = -1;                     // mixer layer applied before the cost phase
  int layer_c = -1;                     // layer of the cost phase
  int layer_b = -1;                     // mixer layer applied after it
  bool init = false, reduce = false;
  bool linit = false;                   // adjoint: creates lambda = C psi
  bool store = true;                    // false only for the adjoint's final pass
};

struct Plan {
  int n = 0, p = 0, S = 0;
  bool backward = false;
  TileShape shape;
  std::vector<std::vector<int>> groups; // qubit groups (one pass each per layer)
  int float_lanes = 0;                  // bits 0..float_lanes-1 float (PLAN_FLOAT_LANES)
  std::vector<PassPlan> passes;
  std::string describe() const;
};

// Group orders: the layers alternate between an order and its reverse, so the
// two ends of the order host the cross-layer fused passes (cost phase and two
// mixers) and the last layer ends on the order's first group.
//   ORDER_LOW_LAST: groups by bit position, the last layer ending on the low
//     group (its final pass sees index-contiguous tiles: sampling block sums);
//   ORDER_LOW_MIDDLE: the low group away from both ends when there are three or
//     more groups, so the fused passes fall on the smaller high groups.
enum GroupOrder { ORDER_LOW_LAST = 0, ORDER_LOW_MIDDLE = 1 };

// Flag or-ed into the order argument of plan_forward: the index bits that
// every tile carries for coalescing (bits 0..4, or 0..3) leave the low group,
// and each layer applies their mixer in one of its plain passes (no cost
// phase) on a high group, whose tile holds them anyway. The fused passes and
// the final pass then work on the low group's remaining bits only (fewer
// butterflies and shared-memory rounds where the pass is instruction-bound);
// the plain pass that takes them gains a round. Applies when every layer has
// a plain pass on a high group (three or more groups); otherwise ignored.
constexpr int PLAN_FLOAT_LANES = 4;

// Forward plan for n qubits and depth p (n >= shape.T()).
// s_max: largest super-tile bit count; min_units_log2: keep at least 2^x super-tiles.
Plan plan_forward(int n, int p, const TileShape& shape, int s_max, int min_units_log2, int order = ORDER_LOW_LAST);

// Adjoint plan: lambda = C psi, then for k = p-1..0 the inverse mixer of layer
// k on every group followed by the inverse cost phase of layer k, packed into
// passes like the forward plan (cross-layer fusion through alternating group
// order). Nothing is stored after the last inverse cost phase.
Plan plan_backward(int n, int p, const TileShape& shape, int s_max, int min_units_log2, int order = ORDER_LOW_LAST);

// Plans the rounds of one sub-pass with tile bits `tb` (tile bit order) for the
// op sequence [mixer A on a_bits] [cost] [mixer B on b_bits] [reduce].
// a_bits / b_bits are tile-bit masks. Throws std::runtime_error if impossible.
std::vector<RoundPlan> plan_rounds(const TileShape& shape, uint32_t a_bits, bool cost,
                                   uint32_t b_bits, bool reduce, uint8_t first_src, bool lam = false);

// Checks the structural invariants of a plan (each mixer bit applied once per
// op, cost after all of layer a, lanes/warps/registers a permutation of the tile
// bits, global rounds coalesced, shared-memory lanes conflict-free). Returns
// an empty string when valid, else a description of the first violation.
std::string validate(const Plan& plan);
std::string validate_rounds(const TileShape& shape, const std::vector<RoundPlan>& rounds,
                            uint32_t a_bits, bool cost, uint32_t b_bits, bool reduce);

// True when the adjoint plan `bwd` retraces the forward plan `fwd` pass by
// pass: equal pass counts, one sub-pass in every adjoint pass, and adjoint pass
// j applying the inverses of exactly the gates of forward pass P-1-j (the same
// mixer qubits of the same layers and the same cost layer). The state at the
// start of adjoint pass j is then the forward's output of pass P-1-j, so the
// adjoint can read it from a stored copy instead of uncomputing it.
bool plans_mirror(const Plan& fwd, const Plan& bwd);

// Compile-time signature of a round (the kernels' specialised instantiations,
// kSigValid set): bits 0-1 and 18 layout, 2-3 source, 4 stores to global
// memory, 5 cost phase, 6 reduction, 7 lambda creation, 8-12 mixer A mask,
// 13-17 mixer B mask. 0 is never a valid signature (it selects runtime
// decoding).
constexpr uint32_t kSigValid = 1u << 31;
uint32_t round_sig(const RoundPlan& rp);

// The fixed menu of round layouts for a tile shape (T = R + 5 + WB):
//   0 "G1": registers on bits 5..R+4, lanes on 0..4, warps on the rest
//   1 "G2": registers on the top R bits, lanes on 0..4, warps on the rest
//   2 "S":  registers on bits 0..R-1, lanes on R..R+4, warps on the rest
//   3 "G3": registers on bit 4 and the top R-1 bits, lanes on 0..3 and T-R
//   4 "GP" (shapes with `paired`): registers on bit 0 and the top R-1 bits,
//     lanes on 1..5, warps on the rest
// G1, G2 and G3 keep lanes 0..3 on tile bits 0..3 (coalesced global access);
// GP keeps register bit 0 and lanes 0..2 on tile bits 0..3 (each lane moves
// two adjacent amplitudes, eight lanes one 16-amplitude run); all keep lanes
// 0..3 (0..2 for 16-byte amplitudes) on bits of distinct residue classes, so
// shared-memory accesses are conflict-free. Kernels instantiate one code path
// per menu entry with compile-time offsets.
constexpr int kNumLayouts = 5;
bool menu_layout(const TileShape& sh, int id, RoundPlan& rp);

// Residue class of tile bit j in the shared-memory swizzle: rows of 16 c64 or 8
// c128 amplitudes, XOR-swizzled so that lanes on bits of distinct classes never
// share a bank.
inline int swizzle_class(int bit, int amp_bytes) { return amp_bytes == 8 ? bit % 4 : bit % 3; }

}  // namespace qaoa
