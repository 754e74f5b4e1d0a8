// Instantiation of the fused sweep for the D1Q13 velocity set.
#include "pkr_sweep.cuh"

namespace pkr {
PKR_INSTANTIATE_SWEEP(D1Q13)
}  // namespace pkr
