// spec_fwd.cu -- specialised forward pass kernels (see spec.h): one
// instantiation of fwd_spec_kernel<R, WB, fast form, signatures...> per
// sequence in pass_sigs.inc (4x3 and 5x4 tiles).
#include "spec.h"

#include "plan.h"

namespace qaoa {

namespace {

struct FwdSpec {
  int nr;
  uint32_t rs[6];
  FwdPassKernel kern;
};

#define QAOA_FWD_SIG(nr, ...) {nr, {__VA_ARGS__}, &fwd_spec_kernel<4, 3, true, __VA_ARGS__>},
#define QAOA_ADJ_SIG(nr, ...)
#define QAOA_FWD_SIG54(nr, ...)
const FwdSpec kFwdSpecs[] = {
#include "pass_sigs.inc"
};
#undef QAOA_FWD_SIG
#undef QAOA_FWD_SIG54

#define QAOA_FWD_SIG(nr, ...)
#define QAOA_FWD_SIG54(nr, ...) {nr, {__VA_ARGS__}, &fwd_spec_kernel<5, 4, true, __VA_ARGS__>},
const FwdSpec kFwdSpecs54[] = {
#include "pass_sigs.inc"
};
#undef QAOA_FWD_SIG
#undef QAOA_FWD_SIG54
#undef QAOA_ADJ_SIG

}  // namespace

uint32_t round_sig_dev(const RoundDev& rd) {
  return kSigValid | uint32_t(rd.layout & 3) | uint32_t(rd.layout >> 2 & 1) << 18 | uint32_t(rd.src & 3) << 2 |
         uint32_t(rd.dst == DST_GLOBAL_D) << 4 | uint32_t(rd.cost != 0) << 5 | uint32_t(rd.reduce != 0) << 6 |
         uint32_t(rd.lam != 0) << 7 | uint32_t(rd.mixA & 31) << 8 | uint32_t(rd.mixB & 31) << 13;
}

FwdPassKernel find_fwd_spec(const SubDev& sd, int R, int WB) {
  const FwdSpec* begin = nullptr;
  const FwdSpec* end = nullptr;
  if (R == 4 && WB == 3) {
    begin = kFwdSpecs;
    end = kFwdSpecs + sizeof(kFwdSpecs) / sizeof(kFwdSpecs[0]);
  } else if (R == 5 && WB == 4) {
    begin = kFwdSpecs54;
    end = kFwdSpecs54 + sizeof(kFwdSpecs54) / sizeof(kFwdSpecs54[0]);
  }
  for (const FwdSpec* it = begin; it != end; ++it) {
    const FwdSpec& f = *it;
    if (f.nr != sd.nrounds) continue;
    bool eq = true;
    for (int r = 0; r < f.nr && eq; ++r) eq = f.rs[r] == round_sig_dev(sd.rd[r]);
    if (eq) return f.kern;
  }
  return nullptr;
}

}  // namespace qaoa
