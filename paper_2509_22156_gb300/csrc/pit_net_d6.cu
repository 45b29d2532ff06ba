// Learned coarse propagator kernels (inference and training) for d = 6.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(6)
}  // namespace pit
