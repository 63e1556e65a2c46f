// Hard-sphere collision kernel (paper Sec. 3.2, Eqs. 3-6).
#include "../../include/dvm.h"
#include "common.cuh"
#include "hs.hpp"

namespace dvm {

int hs_prepare(HsTables &, int64_t, const DevAlloc &, const DevFree &) { return DVM_ENOTIMPL; }

int launch_hs_collide(HsTables &, const StepParams &, void *, double, double) { return DVM_ENOTIMPL; }

}  // namespace dvm
