// Learned coarse propagator kernels (inference and training) for d = 1.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(1)
}  // namespace pit
