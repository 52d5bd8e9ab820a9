// hc_track_tb256.cu -- the block engine of the path tracker with 256-thread blocks (its
// own translation unit, so the instances compile in parallel).
#include "track_kernel.cuh"

namespace hc {
HC_TRACK_INSTANTIATE(256)
}  // namespace hc
