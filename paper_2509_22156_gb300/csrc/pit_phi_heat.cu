// Multi-step backward-Euler kernels of one operator, instantiated for d = 1..6
// and both precision forms (device code in pit_phi.cuh).
#include "pit_phi.cuh"

namespace pit {
PIT_STEPS_OP(heat, PIT_OP_HEAT)
}  // namespace pit
