// Compiled integer chains over packed u8 images:
//   Crop -> [SwapRB] -> AddSatU8 -> WriteU8C3{Split,Packed}
// Every step is integer arithmetic, so results are exact.
#include <cstring>

#include "registry.h"

namespace fkl_impl {

namespace {

template <bool kSplit, bool kSwap, int RY, int CAP>
cudaError_t run_int(const LaunchCtx& c) {
  constexpr int V = 16;
  using RB = fkl::BatchRead<fkl::CropU8C3, CAP>;
  using W = fkl::WriteU8C3<kSplit>;
  fkl::IOp<fkl::AddSatU8> add;
  for (int k = 0; k < 3; ++k) add.params.k[k] = c.spec->addsat[k];
  auto cops = [&] {
    if constexpr (kSwap) {
      return fkl::make_tuple(fkl::IOp<fkl::SwapRB<fkl::U3>>{}, add);
    } else {
      return fkl::make_tuple(add);
    }
  }();
  fkl::Args2D<RB, W, decltype(cops)> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.wp = c.out;
  a.cops = cops;
  a.H = c.H;
  a.W_ = c.W;
  return fkl::launch_transform2d<V, RY>(a, c.n, c.shape.tx, c.shape.ty, c.stream);
}

template <bool kSplit, bool kSwap>
cudaError_t int_by_shape(const LaunchCtx& c) {
  if (c.shape.vec != 16) return cudaErrorInvalidConfiguration;
  const bool single = c.n <= 1;
  if (c.shape.ry == 1)
    return single ? run_int<kSplit, kSwap, 1, 1>(c) : run_int<kSplit, kSwap, 1, kBatchCap>(c);
  if (c.shape.ry == 2)
    return single ? run_int<kSplit, kSwap, 2, 1>(c) : run_int<kSplit, kSwap, 2, kBatchCap>(c);
  return cudaErrorInvalidConfiguration;
}

}  // namespace

cudaError_t launch_int(const LaunchCtx& c) {
  const Spec& s = *c.spec;
  if (s.split) return s.swap ? int_by_shape<true, true>(c) : int_by_shape<true, false>(c);
  return s.swap ? int_by_shape<false, true>(c) : int_by_shape<false, false>(c);
}

}  // namespace fkl_impl
