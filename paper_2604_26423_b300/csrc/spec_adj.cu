// spec_adj.cu -- specialised adjoint pass kernels (see spec.h): one
// instantiation of adj_spec_kernel<4, 3, fast form, signatures...> per
// sequence in pass_sigs.inc.
#include "spec.h"

namespace qaoa {

namespace {

struct AdjSpec {
  int nr;
  uint32_t rs[6];
  AdjPassKernel kern;
};

#define QAOA_FWD_SIG(nr, ...)
#define QAOA_FWD_SIG54(nr, ...)
#define QAOA_ADJ_SIG(nr, ...) {nr, {__VA_ARGS__}, &adj_spec_kernel<4, 3, true, __VA_ARGS__>},
const AdjSpec kAdjSpecs[] = {
#include "pass_sigs.inc"
};
#undef QAOA_FWD_SIG
#undef QAOA_FWD_SIG54
#undef QAOA_ADJ_SIG

}  // namespace

AdjPassKernel find_adj_spec(const SubDev& sd) {
  for (const AdjSpec& f : kAdjSpecs) {
    if (f.nr != sd.nrounds) continue;
    bool eq = true;
    for (int r = 0; r < f.nr && eq; ++r) eq = f.rs[r] == round_sig_dev(sd.rd[r]);
    if (eq) return f.kern;
  }
  return nullptr;
}

}  // namespace qaoa
