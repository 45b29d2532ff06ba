// Learned coarse propagator kernels (inference and training) for d = 3.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(3)
}  // namespace pit
