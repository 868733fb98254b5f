// ising_k_xorwow.cu -- Ising kernels instantiated for RNG_XORWOW.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_XORWOW)
}  // namespace rngx
