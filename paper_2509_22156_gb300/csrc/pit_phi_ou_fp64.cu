// Multi-step backward-Euler kernels of one operator in one precision form
// (FP64 Krylov), instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(ou, fp64, PIT_OP_OU, PLAIN, true)
}  // namespace pit
