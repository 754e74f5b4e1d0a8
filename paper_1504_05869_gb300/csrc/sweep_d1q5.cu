// Instantiation of the fused sweep for the D1Q5 velocity set.
#include "pkr_sweep.cuh"

namespace pkr {
PKR_INSTANTIATE_SWEEP(D1Q5)
}  // namespace pkr
