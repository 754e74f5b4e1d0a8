// Instantiation of the fused sweep for the D3Q111 velocity set.
#include "pkr_sweep.cuh"

namespace pkr {
PKR_INSTANTIATE_SWEEP(D3Q111)
}  // namespace pkr
