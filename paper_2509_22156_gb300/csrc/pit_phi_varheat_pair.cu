// Multi-step backward-Euler kernels of the variable-coefficient heat operator
// in the pair form (FP32 Krylov inside a refinement on FP32 pairs),
// instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(varheat, pair, PIT_OP_VARHEAT, PAIR, true)
}  // namespace pit
