// Learned coarse propagator kernels (inference and training) for d = 4.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(4)
}  // namespace pit
