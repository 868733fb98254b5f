// ising_k_philox4x32_10.cu -- Ising kernels instantiated for RNG_PHILOX4X32_10.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_PHILOX4X32_10)
}  // namespace rngx
