// Compiled float chains over NV12 frames (BT.601 decode, crop, bilinear resize, letterbox),
// writing bf16 outputs.
#include "float_family.cuh"

namespace fkl_impl {

cudaError_t launch_nv12_bf16(const LaunchCtx& c) { return float_dispatch_type<fkl::ResizeNV12, fkl::bf16_t>(c); }

}  // namespace fkl_impl
