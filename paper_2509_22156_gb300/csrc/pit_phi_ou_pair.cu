// Multi-step backward-Euler kernels of the Fokker-Planck (drift) operator in
// the pair form (FP32 BiCGStab inside a refinement on FP32 pairs),
// instantiated for d = 1..6 (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP_PREC(ou, pair, PIT_OP_OU, PAIR, true)
}  // namespace pit
