// Instantiation of the fused sweep for the D2Q81 velocity set.
#include "pkr_sweep.cuh"

namespace pkr {
PKR_INSTANTIATE_SWEEP(D2Q81)
}  // namespace pkr
