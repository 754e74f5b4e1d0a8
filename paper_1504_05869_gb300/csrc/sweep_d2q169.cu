// Instantiation of the fused sweep for the D2Q169 velocity set.
#include "pkr_sweep.cuh"

namespace pkr {
PKR_INSTANTIATE_SWEEP(D2Q169)
}  // namespace pkr
