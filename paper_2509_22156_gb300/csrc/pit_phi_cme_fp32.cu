// Multi-step backward-Euler kernels of one operator in one precision form
// (FP32 Krylov on the scaled FP32 state), instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(cme, fp32, PIT_OP_CME, SINGLE, false)
}  // namespace pit
