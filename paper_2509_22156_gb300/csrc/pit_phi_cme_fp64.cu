// Multi-step backward-Euler kernels of one operator in one precision form
// (FP64 Krylov), instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(cme, fp64, PIT_OP_CME, PLAIN, true)
}  // namespace pit
