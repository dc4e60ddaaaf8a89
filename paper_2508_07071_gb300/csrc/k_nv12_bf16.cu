// Compiled float chains over NV12 frames (BT.601 decode, crop, bilinear resize,
// letterbox), writing bf16 outputs. Launches whose images are all exact 2x
// downscales use the division-free ResizeNV12x2 read op.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_nv12_bf16(const LaunchCtx& c) {
  return c.all_exact2x ? float_dispatch_type<fkl::ResizeNV12x2, fkl::bf16_t>(c)
                       : float_dispatch_type<fkl::ResizeNV12, fkl::bf16_t>(c);
}

}  // namespace fkl_impl
