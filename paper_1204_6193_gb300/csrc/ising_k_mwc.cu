// ising_k_mwc.cu -- Ising kernels instantiated for RNG_MWC.
#include "ising_kernels.cuh"

namespace rngx {
RNGX_ISING_INSTANTIATE(RNG_MWC)
}  // namespace rngx
