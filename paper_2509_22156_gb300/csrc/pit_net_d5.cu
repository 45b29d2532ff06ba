// Learned coarse propagator kernels (inference and training) for d = 5.
#include "pit_net.cuh"

namespace pit {
PIT_NET_DIM(5)
}  // namespace pit
