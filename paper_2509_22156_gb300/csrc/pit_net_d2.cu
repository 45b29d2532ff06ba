// Learned coarse propagator kernels (inference and training) for d = 2.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(2)
}  // namespace pit
