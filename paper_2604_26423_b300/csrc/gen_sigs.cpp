// gen_sigs.cpp -- build-time generator of pass_sigs.inc: the round-signature
// sequences (plan.h, round_sig) of the single-sub-pass passes that the
// complex64 planner emits for the default configurations, so the library can
// compile one specialised pass kernel per sequence (pass_kernel.cuh,
// fwd_spec_kernel; adj_kernel.cuh, adj_spec_kernel). Passes whose sequence is
// not listed run the generic kernels.
//
// Configurations (forward plans with and without the paired global layout):
// tile shape 4x3 (T = 12), n = 13..34, p = 0..12, the forward
// group orders of qaoa_run (low group last) and of the gradient (low group in
// the middle), both with floating coalescing bits; adjoint plans in the
// gradient's order, p = 1..12. Tile shape 5x4 (T = 14): forward plans of
// qaoa_run's order for n = 27..34, p = 0..12 (the sizes where it takes one
// mixer group fewer than 4x3), without and with the paired layout, the latter
// preferring it on the storing last round (the default) or on the first.
//
// Usage: gen_sigs <output file>
#include <cstdio>
#include <set>
#include <vector>

#include "plan.h"

using namespace qaoa;

namespace {

// Single-sub-pass passes; a reduction round also without its reduction (the
// gradient's forward run skips <C>).
void collect(const Plan& pl, std::set<std::vector<uint32_t>>& out) {
  for (const PassPlan& pp : pl.passes) {
    if (pp.subs.size() != 1) continue;
    std::vector<uint32_t> sig;
    for (const RoundPlan& rp : pp.subs[0].rounds) sig.push_back(round_sig(rp));
    if (sig.size() > 6) continue;
    out.insert(sig);
    if (sig.back() & (1u << 6)) {
      sig.back() &= ~(1u << 6);
      out.insert(sig);
    }
  }
}

void emit(FILE* f, const char* macro, const std::set<std::vector<uint32_t>>& sigs) {
  for (const auto& s : sigs) {
    fprintf(f, "%s(%zu", macro, s.size());
    for (uint32_t r : s) fprintf(f, ", 0x%08xu", r);
    fprintf(f, ")\n");
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: gen_sigs <output file>\n");
    return 2;
  }
  TileShape sh;
  sh.R = 4;
  sh.WB = 3;
  sh.amp_bytes = 8;
  TileShape ash = sh;
  ash.nvec = 2;
  // forward plans may use the paired global layout; both menus are generated
  // (QAOA_PAIRED=0 selects the unpaired one at run time)
  TileShape shp = sh;
  shp.paired = true;
  const int T = sh.T();
  std::set<std::vector<uint32_t>> fwd, adj;
  for (int n = T + 1; n <= 34; ++n) {
    for (int p = 0; p <= 12; ++p) {
      for (int order : {ORDER_LOW_LAST | PLAN_FLOAT_LANES, ORDER_LOW_MIDDLE | PLAN_FLOAT_LANES}) {
        collect(plan_forward(n, p, sh, T, 9, order), fwd);
        collect(plan_forward(n, p, shp, T, 9, order), fwd);
      }
      if (p >= 1) collect(plan_backward(n, p, ash, T, 9, ORDER_LOW_MIDDLE), adj);
    }
  }
  TileShape sh54 = sh;
  sh54.R = 5;
  sh54.WB = 4;
  TileShape sh54p = sh54;
  sh54p.paired = true;
  TileShape sh54s = sh54p;
  sh54s.paired_store_first = true;  // the library's default 5x4 shape
  std::set<std::vector<uint32_t>> fwd54;
  for (int n = 27; n <= 34; ++n)
    for (int p = 0; p <= 12; ++p) {
      collect(plan_forward(n, p, sh54, sh54.T(), 9, ORDER_LOW_LAST | PLAN_FLOAT_LANES), fwd54);
      collect(plan_forward(n, p, sh54p, sh54p.T(), 9, ORDER_LOW_LAST | PLAN_FLOAT_LANES), fwd54);
      collect(plan_forward(n, p, sh54s, sh54s.T(), 9, ORDER_LOW_LAST | PLAN_FLOAT_LANES), fwd54);
    }
  FILE* f = fopen(argv[1], "w");
  if (!f) {
    perror(argv[1]);
    return 1;
  }
  fprintf(f, "// Generated by gen_sigs.cpp (build step): round-signature sequences of the\n");
  fprintf(f, "// specialised complex64 pass kernels. Do not edit.\n");
  fprintf(f, "// QAOA_FWD_SIG / QAOA_ADJ_SIG (4x3 tiles), QAOA_FWD_SIG54 (5x4 tiles)\n");
  fprintf(f, "// (number of rounds, round signatures...)\n");
  emit(f, "QAOA_FWD_SIG", fwd);
  emit(f, "QAOA_ADJ_SIG", adj);
  emit(f, "QAOA_FWD_SIG54", fwd54);
  fclose(f);
  printf("%zu forward, %zu adjoint, %zu forward 5x4 sequences\n", fwd.size(), adj.size(), fwd54.size());
  return 0;
}
