// ising_k_philox4x32_7.cu -- Ising kernels instantiated for RNG_PHILOX4X32_7.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_PHILOX4X32_7)
}  // namespace rngx
