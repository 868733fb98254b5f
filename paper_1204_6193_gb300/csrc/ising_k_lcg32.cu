// ising_k_lcg32.cu -- Ising kernels instantiated for RNG_LCG32.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_LCG32)
}  // namespace rngx
