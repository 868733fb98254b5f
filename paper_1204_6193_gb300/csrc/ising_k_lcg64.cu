// ising_k_lcg64.cu -- Ising kernels instantiated for RNG_LCG64.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_LCG64)
}  // namespace rngx
