// Multi-step backward-Euler kernels of one operator in one precision form
// (FP32 Krylov inside FP64 refinement), instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(cme, mixed, PIT_OP_CME, MIXED, true)
}  // namespace pit
