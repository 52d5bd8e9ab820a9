// hc_track_tb512.cu -- the block engine of the path tracker with 512-thread blocks, in
// double and double-double (its own translation unit, so the instances compile in
// parallel).
#include "track_kernel.cuh"

namespace hc {
HC_TRACK_INSTANTIATE_D_DD(512)
}  // namespace hc
