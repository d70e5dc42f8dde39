// spec.h -- registry of the specialised complex64 pass kernels (tile shapes
// 4x3 and 5x4, fast mixer form) compiled for the round-signature sequences
// listed in pass_sigs.inc (generated at build time by gen_sigs.cpp from the
// planner).
#pragma once
#include <cstdint>

#include "adj_kernel.cuh"
#include "device.cuh"
#include "pass_kernel.cuh"

namespace qaoa {

using FwdPassKernel = void (*)(PassDev, PassArgs, PassTma);
using AdjPassKernel = void (*)(PassDev, AdjArgs, PassTma);

// Round signature (plan.h, round_sig) of a round descriptor.
uint32_t round_sig_dev(const RoundDev& rd);

// The specialised forward pass kernel of tile shape RxWB (4x3 or 5x4) for the
// rounds of a single-sub-pass descriptor (its round signatures), or nullptr if
// none was compiled.
FwdPassKernel find_fwd_spec(const SubDev& sd, int R, int WB);

// The same for the adjoint pass kernel (4x3 tiles of psi and lambda).
AdjPassKernel find_adj_spec(const SubDev& sd);

}  // namespace qaoa
