// Compiled float chains over NV12 frames (BT.601 decode, crop, bilinear resize, letterbox),
// writing f32 outputs.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_nv12_f32(const LaunchCtx& c) { return float_dispatch_type<fkl::ResizeNV12, float>(c); }

}  // namespace fkl_impl
