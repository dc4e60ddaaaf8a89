// Compiled float chains over NV12 frames (BT.601 decode, crop, bilinear resize, letterbox),
// writing e4m3 outputs.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_nv12_e4m3(const LaunchCtx& c) { return float_dispatch_type<fkl::ResizeNV12, fkl::e4m3_t>(c); }

}  // namespace fkl_impl
