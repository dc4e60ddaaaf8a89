// Compiled float chains over NV12 frames (BT.601 decode, crop, bilinear resize,
// letterbox), writing f32 outputs. Launches whose images are all exact 2x
// downscales use the division-free ResizeNV12x2 read op.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_nv12_f32(const LaunchCtx& c) {
  return c.all_exact2x ? float_dispatch_type<fkl::ResizeNV12x2, float>(c)
                       : float_dispatch_type<fkl::ResizeNV12, float>(c);
}

}  // namespace fkl_impl
