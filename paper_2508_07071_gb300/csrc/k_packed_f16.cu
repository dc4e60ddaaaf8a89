// Compiled float chains over packed 3-channel u8 images (crop, bilinear resize, placement),
// writing f16 outputs.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_packed_f16(const LaunchCtx& c) { return float_dispatch_type<fkl::ResizeU8C3, fkl::f16_t>(c); }

}  // namespace fkl_impl
