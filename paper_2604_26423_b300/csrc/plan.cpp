// plan.cpp -- pass / sub-pass / round planner (host only). See plan.h.
#include "plan.h"

#include <algorithm>
#include <cstdio>
#include <set>
#include <sstream>
#include <stdexcept>
#include <tuple>

namespace qaoa {
namespace {

int popc(uint32_t x) { return __builtin_popcount(x); }

std::vector<int> bits_of(uint32_t m) {
  std::vector<int> v;
  for (int i = 0; i < 32; ++i)
    if (m >> i & 1u) v.push_back(i);
  return v;
}

// Register-position mask of tile-bit mask `m` in round `rp`.
uint8_t regmask(const RoundPlan& rp, int R, uint32_t m) {
  uint8_t r = 0;
  for (int i = 0; i < R; ++i)
    if (m >> rp.reg[i] & 1u) r |= uint8_t(1u << i);
  return r;
}

}  // namespace

bool menu_layout(const TileShape& sh, int id, RoundPlan& rp) {
  const int T = sh.T(), R = sh.R, WB = sh.WB;
  std::vector<int> regs, lanes, warps;
  switch (id) {
    case 0:
      for (int i = 0; i < R; ++i) regs.push_back(5 + i);
      for (int i = 0; i < 5; ++i) lanes.push_back(i);
      for (int b = 5 + R; b < T; ++b) warps.push_back(b);
      break;
    case 1:
      for (int i = 0; i < R; ++i) regs.push_back(T - R + i);
      for (int i = 0; i < 5; ++i) lanes.push_back(i);
      for (int b = 5; b < T - R; ++b) warps.push_back(b);
      break;
    case 2:
      for (int i = 0; i < R; ++i) regs.push_back(i);
      for (int i = 0; i < 5; ++i) lanes.push_back(R + i);
      for (int b = R + 5; b < T; ++b) warps.push_back(b);
      break;
    case 3:
      regs.push_back(4);
      for (int i = 1; i < R; ++i) regs.push_back(T - R + i);
      for (int i = 0; i < 4; ++i) lanes.push_back(i);
      lanes.push_back(T - R);
      for (int b = 5; b < T - R; ++b) warps.push_back(b);
      break;
    case 4:
      if (!sh.paired || sh.amp_bytes != 8) return false;
      regs.push_back(0);
      for (int i = 1; i < R; ++i) regs.push_back(T - R + i);
      for (int i = 1; i <= 5; ++i) lanes.push_back(i);
      for (int b = 6; b <= T - R; ++b) warps.push_back(b);
      break;
    default:
      return false;
  }
  if ((int)regs.size() != R || (int)warps.size() != WB || (int)lanes.size() != 5) return false;
  for (int i = 0; i < 5; ++i) rp.reg[i] = i < R ? int8_t(regs[i]) : 0;
  for (int i = 0; i < 5; ++i) rp.lane[i] = int8_t(lanes[i]);
  for (int i = 0; i < 4; ++i) rp.warp[i] = i < WB ? int8_t(warps[i]) : 0;
  rp.layout = uint8_t(id);
  rp.global_facing = id != 2;
  return true;
}

uint32_t round_sig(const RoundPlan& rp) {
  return kSigValid | uint32_t(rp.layout & 3) | uint32_t(rp.layout >> 2 & 1) << 18 | uint32_t(rp.src & 3) << 2 |
         uint32_t(rp.dst == DST_GLOBAL) << 4 | uint32_t(rp.cost != 0) << 5 | uint32_t(rp.reduce != 0) << 6 |
         uint32_t(rp.lam != 0) << 7 | uint32_t(rp.mixA & 31) << 8 | uint32_t(rp.mixB & 31) << 13;
}

std::vector<RoundPlan> plan_rounds(const TileShape& sh, uint32_t a_bits, bool cost, uint32_t b_bits,
                                   bool reduce, uint8_t first_src, bool lam) {
  // Breadth-first search over (bits left for mixer A, bits left for mixer B,
  // cost applied) for the fewest rounds drawn from the layout menu. A round
  // applies mixer A on its register bits; once A is complete it applies the
  // cost phase (if pending) and mixer B on its register bits. The last round
  // must be global-facing (it stores the tile); so must the first when it
  // loads from global memory. Without a cost phase here, mixer B continues a
  // layer whose cost phase was applied in an earlier sub-pass.
  const int R = sh.R;
  struct Node { uint32_t remA, remB; bool cost_done; int parent; int layout; uint8_t mA, mB, c; };
  std::vector<Node> nodes;
  nodes.push_back({a_bits, b_bits, !cost, -1, -1, 0, 0, 0});
  std::set<std::tuple<uint32_t, uint32_t, bool>> seen;
  size_t head = 0;
  // among the shortest sequences, the one with the most paired global rounds
  // (16-byte accesses in the loading first round and the storing last round)
  std::vector<RoundPlan> best;
  int best_score = -1;
  for (int depth = 0; depth < kMaxRounds; ++depth) {
    const size_t level_end = nodes.size();
    for (size_t ni = head; ni < level_end; ++ni) {
      for (int k = 0; k < kNumLayouts; ++k) {
        // the paired layout first: among round sequences of equal length the
        // one with 16-byte global accesses is found first
        const int id = (k + kNumLayouts - 1) % kNumLayouts;
        RoundPlan rp;
        if (!menu_layout(sh, id, rp)) continue;
        if (depth == 0 && first_src == SRC_GLOBAL && !rp.global_facing) continue;
        Node nd = nodes[ni];
        uint32_t x = 0;
        for (int i = 0; i < R; ++i) x |= 1u << rp.reg[i];
        nd.mA = regmask(rp, R, x & nd.remA);
        nd.remA &= ~x;
        nd.c = 0;
        nd.mB = 0;
        if (nd.remA == 0) {
          if (!nd.cost_done) { nd.c = 1; nd.cost_done = true; }
          nd.mB = regmask(rp, R, x & nd.remB);
          nd.remB &= ~x;
        }
        nd.parent = (int)ni;
        nd.layout = id;
        const bool done = nd.remA == 0 && nd.remB == 0 && nd.cost_done;
        if (done && rp.global_facing) {
          nodes.push_back(nd);
          std::vector<int> chain;
          for (int k = (int)nodes.size() - 1; nodes[k].parent >= 0; k = nodes[k].parent) chain.push_back(k);
          std::reverse(chain.begin(), chain.end());
          std::vector<RoundPlan> out;
          for (size_t r = 0; r < chain.size(); ++r) {
            const Node& q = nodes[chain[r]];
            RoundPlan rr;
            menu_layout(sh, q.layout, rr);
            rr.mixA = q.mA;
            rr.cost = q.c;
            rr.mixB = q.mB;
            rr.src = r == 0 ? first_src : SRC_SMEM;
            rr.dst = r + 1 == chain.size() ? DST_GLOBAL : DST_SMEM;
            rr.reduce = (reduce && r + 1 == chain.size()) ? 1 : 0;
            rr.lam = (lam && r == 0) ? 1 : 0;
            out.push_back(rr);
          }
          const int score = (sh.paired_store_first ? 2 : 1) * int(out.back().layout == 4) +
                            int(first_src == SRC_GLOBAL && out[0].layout == 4);
          if (score > best_score) {
            best_score = score;
            best = out;
          }
          continue;
        }
        auto key = std::make_tuple(nd.remA, nd.remB, nd.cost_done);
        if (seen.count(key)) continue;
        seen.insert(key);
        nodes.push_back(nd);
      }
    }
    if (best_score >= 0) return best;
    head = level_end;
  }
  throw std::runtime_error("plan_rounds: no round sequence from the layout menu");
}

std::string validate_rounds(const TileShape& sh, const std::vector<RoundPlan>& rounds, uint32_t a_bits,
                            bool cost, uint32_t b_bits, bool reduce) {
  const int T = sh.T(), R = sh.R, WB = sh.WB;
  uint32_t doneA = 0, doneB = 0;
  bool cost_seen = false, reduce_seen = false;
  if (rounds.empty()) return "no rounds";
  for (size_t k = 0; k < rounds.size(); ++k) {
    const RoundPlan& rp = rounds[k];
    uint32_t seen = 0;
    for (int i = 0; i < R; ++i) seen |= 1u << rp.reg[i];
    for (int i = 0; i < 5; ++i) seen |= 1u << rp.lane[i];
    for (int i = 0; i < WB; ++i) seen |= 1u << rp.warp[i];
    if (seen != ((1u << T) - 1) || popc(seen) != T) return "round is not a permutation of tile bits";
    const bool is_last = k + 1 == rounds.size();
    if ((k == 0 && rp.src == SRC_GLOBAL) || is_last) {
      const bool paired = rp.reg[0] == 0 && rp.lane[0] == 1 && rp.lane[1] == 2 && rp.lane[2] == 3;
      for (int i = 0; i < 4; ++i)
        if (rp.lane[i] != i && !paired) return "global round without lanes 0..3 (or register 0 and lanes 0..2) on tile bits 0..3";
    }
    if (is_last != (rp.dst == DST_GLOBAL)) return "only the last round stores to global memory";
    if (k > 0 && rp.src != SRC_SMEM) return "only the first round reads global memory";
    if (!rp.global_facing || (k > 0 && !is_last)) {
      const int ncls = sh.amp_bytes == 8 ? 4 : 3;
      uint32_t cls = 0;
      for (int i = 0; i < ncls; ++i) cls |= 1u << swizzle_class(rp.lane[i], sh.amp_bytes);
      if (popc(cls) != ncls) return "shared-memory lanes share a swizzle class";
    }
    for (int i = 0; i < R; ++i) {
      const uint32_t b = 1u << rp.reg[i];
      if (rp.mixA >> i & 1u) {
        if (cost_seen) return "mixer A after the cost phase";
        if (doneA & b) return "mixer A bit applied twice";
        if (!(a_bits & b)) return "mixer A on a non-target bit";
        doneA |= b;
      }
    }
    if (rp.cost) {
      if (doneA != a_bits) return "cost phase before mixer A completed";
      if (!cost) return "unexpected cost phase";
      cost_seen = true;
    }
    for (int i = 0; i < R; ++i) {
      const uint32_t b = 1u << rp.reg[i];
      if (rp.mixB >> i & 1u) {
        if (cost && !cost_seen) return "mixer B before the cost phase";
        if (doneA != a_bits) return "mixer B before mixer A completed";
        if (doneB & b) return "mixer B bit applied twice";
        if (!(b_bits & b)) return "mixer B on a non-target bit";
        doneB |= b;
      }
    }
    if (rp.reduce) {
      if (!is_last) return "reduce before the last round";
      reduce_seen = true;
    }
  }
  if (doneA != a_bits) return "mixer A incomplete";
  if (doneB != b_bits) return "mixer B incomplete";
  if (cost != cost_seen) return "cost phase missing";
  if (reduce != reduce_seen) return "reduce missing";
  return "";
}

namespace {

struct Group {
  std::vector<int> sb;       // super-tile bits (ascending)
  std::vector<int> targets;  // qubits of the group (ascending)
};

// Splits a group's targets into sub-pass chunks and builds their tiles.
// Every tile holds global bits 0..3 (tile bits 0..3); the first tile also holds
// bit 4 when the super-tile has it as a non-target, so HBM reads come in
// 256-byte (c64) / 512-byte (c128) runs.
std::vector<std::pair<std::vector<int>, std::vector<int>>> chunk_group(const Group& g, int T) {
  std::vector<std::pair<std::vector<int>, std::vector<int>>> out;  // (tile bits in tile order, chunk)
  std::vector<int> rest = g.targets;
  bool first = true;
  auto in_sb = [&](int b) { return std::find(g.sb.begin(), g.sb.end(), b) != g.sb.end(); };
  auto is_target = [&](int b) { return std::find(g.targets.begin(), g.targets.end(), b) != g.targets.end(); };
  do {
    std::vector<int> tile = {0, 1, 2, 3};
    std::vector<int> chunk;
    for (int b = 0; b < 4; ++b) {
      auto it = std::find(rest.begin(), rest.end(), b);
      if (it != rest.end()) { chunk.push_back(b); rest.erase(it); }
    }
    const bool keep4 = first && in_sb(4) && !is_target(4);
    if (keep4) tile.push_back(4);
    while ((int)tile.size() < T && !rest.empty()) {
      tile.push_back(rest.front());
      chunk.push_back(rest.front());
      rest.erase(rest.begin());
    }
    // fillers: lowest super-tile bits not yet in the tile
    for (int b : g.sb)
      if ((int)tile.size() < T && std::find(tile.begin(), tile.end(), b) == tile.end()) tile.push_back(b);
    if ((int)tile.size() != T) throw std::runtime_error("chunk_group: super-tile smaller than a tile");
    std::vector<int> order(tile.begin() + 4, tile.end());
    std::sort(order.begin(), order.end());
    std::vector<int> t2 = {0, 1, 2, 3};
    t2.insert(t2.end(), order.begin(), order.end());
    std::sort(chunk.begin(), chunk.end());
    out.emplace_back(t2, chunk);
    first = false;
  } while (!rest.empty());
  return out;
}

uint32_t tile_mask(const std::vector<int>& tile, const std::vector<int>& chunk) {
  uint32_t m = 0;
  for (int b : chunk) {
    auto it = std::find(tile.begin(), tile.end(), b);
    m |= 1u << int(it - tile.begin());
  }
  return m;
}

}  // namespace

namespace {

std::vector<Group> make_groups(int n, int S) {
  // the low S bits, then windows of high bits that keep 32 (r = 5) or 16
  // (r = 4) consecutive amplitudes per contiguous run
  std::vector<Group> groups;
  Group low;
  for (int b = 0; b < S; ++b) low.sb.push_back(b), low.targets.push_back(b);
  groups.push_back(low);
  const int left = n - S;
  if (left > 0) {
    const int X5 = S - 5, X4 = S - 4;
    const int g5 = (left + X5 - 1) / X5, g4 = (left + X4 - 1) / X4;
    const int r = g5 <= g4 ? 5 : 4;
    const int X = S - r;
    for (int a = S; a < n; a += X) {
      const int b = std::min(n, a + X);
      Group g;
      for (int q = 0; q < r; ++q) g.sb.push_back(q);
      // a last window narrower than X is filled with the lowest bits above
      // the coalescing ones (r, r+1, ...), not the bits just below it: the
      // tile then spans fewer memory pages (its high bits are the targets
      // only) and bit r lengthens its contiguous runs
      for (int q = r; q < r + (X - (b - a)); ++q) g.sb.push_back(q);
      for (int q = a; q < b; ++q) g.sb.push_back(q), g.targets.push_back(q);
      groups.push_back(g);
    }
  }
  return groups;
}

enum OpKind { OP_MIX, OP_COST };
struct Op { OpKind kind; int layer, grp; };
struct Proto { int grp = -1; int a = -1, cost = -1, b = -1; };

// Packs an op sequence into passes of the form [mixer A][cost][mixer B], all
// mixers of a pass on one group, at most one cost phase per pass.
std::vector<Proto> pack_ops(const std::vector<Op>& ops) {
  std::vector<Proto> out;
  Proto cur;
  for (const Op& op : ops) {
    if (op.kind == OP_MIX) {
      if (cur.grp < 0 && cur.a < 0 && cur.b < 0) {
        cur.grp = op.grp;
        if (cur.cost >= 0) cur.b = op.layer; else cur.a = op.layer;
      } else if (cur.cost >= 0 && cur.b < 0 && (cur.grp < 0 || cur.grp == op.grp)) {
        cur.grp = op.grp;
        cur.b = op.layer;
      } else {
        out.push_back(cur);
        cur = Proto();
        cur.grp = op.grp;
        cur.a = op.layer;
      }
    } else {
      if (cur.cost < 0 && cur.b < 0) {
        cur.cost = op.layer;
      } else {
        out.push_back(cur);
        cur = Proto();
        cur.cost = op.layer;
      }
    }
  }
  if (cur.grp < 0) cur.grp = 0;
  out.push_back(cur);
  return out;
}

// extra[pi]: qubits whose mixer pass pi applies besides its group's (floating
// lane bits, see PLAN_FLOAT_LANES), or empty.
void build_passes(Plan& plan, const std::vector<Group>& groups, const std::vector<Proto>& protos, bool backward,
                  const std::vector<std::vector<int>>& extra) {
  const int n = plan.n, T = plan.shape.T();
  for (size_t pi = 0; pi < protos.size(); ++pi) {
    const Proto& pr = protos[pi];
    PassPlan pp;
    Group g = groups[pr.grp];
    if (!extra[pi].empty()) {
      g.targets.insert(g.targets.end(), extra[pi].begin(), extra[pi].end());
      std::sort(g.targets.begin(), g.targets.end());
    }
    pp.sb = g.sb;
    for (int b = 0; b < n; ++b)
      if (std::find(g.sb.begin(), g.sb.end(), b) == g.sb.end()) pp.outer.push_back(b);
    const bool first = pi == 0, last = pi + 1 == protos.size();
    pp.init = !backward && first;
    pp.linit = backward && first;
    pp.reduce = !backward && last;
    pp.store = !(backward && last);
    pp.layer_a = pr.a;
    pp.layer_c = pr.cost;
    pp.layer_b = pr.b;
    const bool has_cost = pr.cost >= 0;
    const bool has_b = pr.b >= 0;
    const bool has_mix = pr.a >= 0 || has_b;
    if (has_mix) pp.targets = g.targets;
    auto chunks = chunk_group(Group{g.sb, has_mix ? g.targets : std::vector<int>{}}, T);
    const int K = (int)chunks.size();
    struct SubOps { int chunk; bool a, cost, b; };
    std::vector<SubOps> seq;
    if (pr.a >= 0 && has_cost && has_b) {
      for (int i = 0; i < K - 1; ++i) seq.push_back({i, true, false, false});
      seq.push_back({K - 1, true, true, true});
      for (int i = K - 2; i >= 0; --i) seq.push_back({i, false, false, true});
    } else if (pr.a >= 0 && has_cost) {
      for (int i = 0; i < K - 1; ++i) seq.push_back({i, true, false, false});
      seq.push_back({K - 1, true, true, false});
    } else if (pr.a >= 0) {
      for (int i = 0; i < K; ++i) seq.push_back({i, true, false, false});
    } else if (has_cost) {
      seq.push_back({0, false, true, has_b});
      for (int i = 1; i < K; ++i) seq.push_back({i, false, false, has_b});
    } else {
      for (int i = 0; i < K; ++i) seq.push_back({i, false, false, false});
    }
    for (size_t s = 0; s < seq.size(); ++s) {
      const SubOps& so = seq[s];
      SubPassPlan sp;
      sp.T = T;
      const auto& tile = chunks[so.chunk].first;
      const auto& chunk = chunks[so.chunk].second;
      for (int j = 0; j < T; ++j) sp.pos[j] = int8_t(tile[j]);
      const uint32_t m = tile_mask(tile, chunk);
      const uint32_t am = so.a ? m : 0, bm = so.b ? m : 0;
      const bool lastsub = s + 1 == seq.size();
      const bool red = pp.reduce && lastsub;
      sp.init = pp.init && s == 0;
      sp.linit = pp.linit && s == 0;
      sp.store = pp.store || !lastsub;
      sp.rounds = plan_rounds(plan.shape, am, so.cost, bm, red, sp.init ? SRC_INIT : SRC_GLOBAL, sp.linit);
      sp.nA = popc(am);
      sp.nB = popc(bm);
      sp.needs_c = so.cost || red || sp.linit;
      pp.subs.push_back(sp);
    }
    plan.passes.push_back(pp);
  }
}

Plan make_plan(int n, int p, const TileShape& sh, int s_max, int min_units_log2, bool backward, int order) {
  const int T = sh.T();
  if (n < T) throw std::runtime_error("planner: n below the tile size");
  if (n > kMaxQubits) throw std::runtime_error("planner: n too large");
  if (backward && p < 1) throw std::runtime_error("planner: the adjoint needs p >= 1");
  Plan plan;
  plan.n = n;
  plan.p = p;
  plan.shape = sh;
  plan.backward = backward;
  int S = std::min(s_max, std::max(T, n - min_units_log2));
  S = std::min(S, n);
  plan.S = S;
  std::vector<Group> groups = make_groups(n, S);
  const int G = (int)groups.size();
  const int base_order = order & 3;
  // Base order ord[]: the last layer ends on ord[0]. ORDER_LOW_LAST keeps
  // groups by bit position (ending on the low, index-contiguous group: the
  // final pass sees whole contiguous blocks, for odd p the write-only first
  // pass gets the top group). ORDER_LOW_MIDDLE puts the two smallest high
  // groups at the ends and the low group next to ord[0].
  std::vector<int> ord(G);
  for (int i = 0; i < G; ++i) ord[i] = i;
  if (base_order == ORDER_LOW_MIDDLE && G >= 3) {
    std::vector<int> high;
    for (int i = 1; i < G; ++i) high.push_back(i);
    std::stable_sort(high.begin(), high.end(),
                     [&](int a, int b) { return groups[a].targets.size() < groups[b].targets.size(); });
    ord.clear();
    ord.push_back(high[0]);
    ord.push_back(0);
    for (size_t i = 2; i < high.size(); ++i) ord.push_back(high[i]);
    ord.push_back(high[1]);
  }
  // layer k runs ord reversed when (p - 1 - k) is even, so consecutive layers
  // meet on one group and the last layer ends on ord[0]
  auto fwd_grp = [&](int k, int i) { return ((p - 1 - k) % 2 == 0) ? ord[G - 1 - i] : ord[i]; };
  std::vector<Op> ops;
  if (!backward) {
    // [init] then per layer k: cost k, mixer k over the groups
    for (int k = 0; k < p; ++k) {
      ops.push_back({OP_COST, k, -1});
      for (int i = 0; i < G; ++i) ops.push_back({OP_MIX, k, fwd_grp(k, i)});
    }
  } else {
    // [lambda] then per layer k = p-1..0: inverse mixer k over the groups in the
    // reverse of the forward order of layer k, then inverse cost k
    for (int j = 0; j < p; ++j) {
      const int k = p - 1 - j;
      for (int i = 0; i < G; ++i) ops.push_back({OP_MIX, k, fwd_grp(k, G - 1 - i)});
      ops.push_back({OP_COST, k, -1});
    }
  }
  const std::vector<Proto> protos = pack_ops(ops);
  std::vector<std::vector<int>> extra(protos.size());
  if (!backward && (order & PLAN_FLOAT_LANES) && G >= 3) {
    // bits that every high group's tiles carry: 0..r-1
    int r = 32;
    for (int gi = 1; gi < G; ++gi) {
      int k = 0;
      while (k < (int)groups[gi].sb.size() && groups[gi].sb[k] == k) ++k;
      r = std::min(r, k);
    }
    // host of layer k: its plain pass on the high group with the fewest targets
    std::vector<int> host(p, -1);
    for (size_t pi = 0; pi < protos.size(); ++pi) {
      const Proto& pr = protos[pi];
      if (pr.a < 0 || pr.cost >= 0 || pr.b >= 0 || pr.grp == 0) continue;
      int& h = host[pr.a];
      if (h < 0 || groups[pr.grp].targets.size() < groups[protos[h].grp].targets.size()) h = (int)pi;
    }
    const bool ok = r > 0 && std::all_of(host.begin(), host.end(), [](int h) { return h >= 0; });
    if (ok) {
      std::vector<int> lanes;
      for (int b = 0; b < r; ++b) lanes.push_back(b);
      auto& t0 = groups[0].targets;
      t0.erase(std::remove_if(t0.begin(), t0.end(), [&](int b) { return b < r; }), t0.end());
      for (int k = 0; k < p; ++k) extra[host[k]] = lanes;
      plan.float_lanes = r;
    }
  }
  for (auto& g : groups) plan.groups.push_back(g.targets);
  build_passes(plan, groups, protos, backward, extra);
  return plan;
}

}  // namespace

Plan plan_forward(int n, int p, const TileShape& sh, int s_max, int min_units_log2, int order) {
  return make_plan(n, p, sh, s_max, min_units_log2, false, order);
}

Plan plan_backward(int n, int p, const TileShape& sh, int s_max, int min_units_log2, int order) {
  return make_plan(n, p, sh, s_max, min_units_log2, true, order);
}

std::string validate(const Plan& plan) {
  const int n = plan.n, P = plan.p;
  const bool bwd = plan.backward;
  // Dependencies. Forward: mixer of layer k after cost k; cost k after every
  // qubit's mixer of layer k-1. Adjoint (layers walked backwards): inverse
  // mixer of layer k after the inverse cost of layer k+1; inverse cost of
  // layer k after every qubit's inverse mixer of layer k. Each op once.
  std::vector<std::vector<int>> mix_count(P, std::vector<int>(n, 0));
  std::vector<int> cost_count(P, 0);
  auto mix = [&](int L, int q) -> std::string {
    if (L < 0 || L >= P) return "mixer without layer";
    if (!bwd && cost_count[L] != 1) return "mixer before its layer's cost";
    if (bwd && L + 1 < P && cost_count[L + 1] != 1) return "inverse mixer before the later layer's inverse cost";
    if (mix_count[L][q]++ != 0) return "mixer applied twice";
    return "";
  };
  auto cost = [&](int L) -> std::string {
    if (L < 0 || L >= P) return "cost without layer";
    const int need = bwd ? L : L - 1;
    if (need >= 0)
      for (int q = 0; q < n; ++q)
        if (mix_count[need][q] != 1) return "cost phase before the mixer it depends on completed";
    if (cost_count[L]++ != 0) return "cost applied twice";
    return "";
  };
  int init_count = 0, reduce_count = 0, linit_count = 0;
  for (size_t pi = 0; pi < plan.passes.size(); ++pi) {
    const PassPlan& pp = plan.passes[pi];
    const bool first = pi == 0, last = pi + 1 == plan.passes.size();
    init_count += pp.init;
    reduce_count += pp.reduce;
    linit_count += pp.linit;
    if ((pp.init || pp.linit) && !first) return "initialisation not in the first pass";
    if (pp.reduce && !last) return "reduce not in the last pass";
    if (!pp.store && !last) return "only the last pass may skip its store";
    for (size_t si = 0; si < pp.subs.size(); ++si) {
      const SubPassPlan& sp = pp.subs[si];
      if (!sp.store && !(last && si + 1 == pp.subs.size())) return "a sub-pass other than the very last skips its store";
      uint32_t am = 0, bm = 0;
      bool c = false, red = false;
      for (const RoundPlan& rp : sp.rounds) {
        for (int i = 0; i < plan.shape.R; ++i) {
          if (rp.mixA >> i & 1u) am |= 1u << rp.reg[i];
          if (rp.mixB >> i & 1u) bm |= 1u << rp.reg[i];
        }
        c |= rp.cost != 0;
        red |= rp.reduce != 0;
      }
      if (sp.linit && !sp.rounds.empty() && !sp.rounds[0].lam) return "lambda creation not in the first round";
      std::string e = validate_rounds(plan.shape, sp.rounds, am, c, bm, red);
      if (!e.empty()) return "round check: " + e;
      for (int j = 0; j < sp.T; ++j)
        if (am >> j & 1u) { e = mix(pp.layer_a, sp.pos[j]); if (!e.empty()) return e; }
      if (c) { e = cost(pp.layer_c); if (!e.empty()) return e; }
      for (int j = 0; j < sp.T; ++j)
        if (bm >> j & 1u) { e = mix(pp.layer_b, sp.pos[j]); if (!e.empty()) return e; }
    }
  }
  if (bwd ? (linit_count != 1 || init_count || reduce_count) : (init_count != 1 || reduce_count != 1 || linit_count))
    return "initialisation / reduction count";
  for (int k = 0; k < P; ++k) {
    if (cost_count[k] != 1) return "cost count of a layer";
    for (int q = 0; q < n; ++q)
      if (mix_count[k][q] != 1) return "mixer count of a qubit";
  }
  return "";
}

namespace {

// The gates a pass applies: (layer, qubit) of every mixer and (layer, -1) of
// the cost phase, sorted.
std::vector<std::pair<int, int>> pass_gates(const Plan& pl, const PassPlan& pp) {
  std::vector<std::pair<int, int>> g;
  for (const SubPassPlan& sp : pp.subs) {
    uint32_t am = 0, bm = 0;
    bool c = false;
    for (const RoundPlan& rp : sp.rounds) {
      for (int i = 0; i < pl.shape.R; ++i) {
        if (rp.mixA >> i & 1u) am |= 1u << rp.reg[i];
        if (rp.mixB >> i & 1u) bm |= 1u << rp.reg[i];
      }
      c |= rp.cost != 0;
    }
    for (int j = 0; j < sp.T; ++j) {
      if (am >> j & 1u) g.emplace_back(pp.layer_a, sp.pos[j]);
      if (bm >> j & 1u) g.emplace_back(pp.layer_b, sp.pos[j]);
    }
    if (c) g.emplace_back(pp.layer_c, -1);
  }
  std::sort(g.begin(), g.end());
  return g;
}

}  // namespace

bool plans_mirror(const Plan& fwd, const Plan& bwd) {
  const size_t np = fwd.passes.size();
  if (fwd.backward || !bwd.backward || fwd.n != bwd.n || fwd.p != bwd.p || bwd.passes.size() != np) return false;
  for (size_t j = 0; j < np; ++j) {
    const PassPlan& b = bwd.passes[j];
    if (b.subs.size() != 1) return false;
    if (pass_gates(bwd, b) != pass_gates(fwd, fwd.passes[np - 1 - j])) return false;
  }
  return true;
}

std::string Plan::describe() const {
  std::ostringstream os;
  os << "n=" << n << " p=" << p << " S=" << S << " T=" << shape.T() << " R=" << shape.R
     << " WB=" << shape.WB << " groups=" << groups.size() << " passes=" << passes.size();
  if (float_lanes) os << " float_lanes=" << float_lanes;
  os << "\n";
  for (size_t g = 0; g < groups.size(); ++g) {
    os << "group " << g << ":";
    for (int q : groups[g]) os << " " << q;
    os << "\n";
  }
  for (size_t pi = 0; pi < passes.size(); ++pi) {
    const PassPlan& pp = passes[pi];
    os << "pass " << pi << " a=" << pp.layer_a << " c=" << pp.layer_c << " b=" << pp.layer_b
       << (pp.init ? " init" : "") << (pp.linit ? " lambda" : "") << (pp.reduce ? " reduce" : "")
       << (pp.store ? "" : " nostore") << " sb=[";
    for (int b : pp.sb) os << b << ",";
    os << "] subs=" << pp.subs.size() << "\n";
    for (size_t s = 0; s < pp.subs.size(); ++s) {
      const SubPassPlan& sp = pp.subs[s];
      os << "  sub " << s << " tile=[";
      for (int j = 0; j < sp.T; ++j) os << int(sp.pos[j]) << (j + 1 < sp.T ? "," : "");
      os << "] nA=" << sp.nA << " nB=" << sp.nB << "\n";
      for (const RoundPlan& rp : sp.rounds) {
        os << "    round src=" << int(rp.src) << " dst=" << int(rp.dst) << " reg=";
        for (int i = 0; i < shape.R; ++i) os << int(rp.reg[i]) << (i + 1 < shape.R ? "," : "");
        os << " lane=";
        for (int i = 0; i < 5; ++i) os << int(rp.lane[i]) << (i < 4 ? "," : "");
        os << " warp=";
        for (int i = 0; i < shape.WB; ++i) os << int(rp.warp[i]) << (i + 1 < shape.WB ? "," : "");
        os << " A=" << int(rp.mixA) << " C=" << int(rp.cost) << " B=" << int(rp.mixB)
           << " R=" << int(rp.reduce) << (rp.lam ? " L=1" : "") << "\n";
      }
    }
  }
  return os.str();
}

}  // namespace qaoa
