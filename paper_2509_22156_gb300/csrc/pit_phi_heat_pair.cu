// Multi-step backward-Euler kernels of the heat operator in the pair form
// (FP32 Krylov inside a refinement on FP32 pairs), instantiated for d = 1..6
// (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(heat, pair, PIT_OP_HEAT, PAIR, true)
}  // namespace pit
