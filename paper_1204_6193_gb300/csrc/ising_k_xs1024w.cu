// ising_k_xs1024w.cu -- Ising kernels instantiated for RNG_XS1024W.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_XS1024W)
}  // namespace rngx
