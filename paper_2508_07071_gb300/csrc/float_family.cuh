// Instantiation and dispatch of the float image chains
//   ROp -> [SwapRB] -> Mul -> Sub -> Div -> Write{Split,Packed}<OutT>
// for one resampling ROp. Included by exactly one translation unit per ROp
// (k_packed.cu, k_nv12.cu) so the families compile in parallel.
#pragma once

#include <cstring>

#include "registry.h"

namespace fkl_impl {

// Vector widths compiled per output type (pixels per thread along x).
template <class OutT, bool kSplit>
struct VecSet;
template <>
struct VecSet<float, true> {
  static constexpr int v[] = {4, 8};
};
template <>
struct VecSet<float, false> {
  static constexpr int v[] = {4};
};
template <>
struct VecSet<fkl::f16_t, true> {
  static constexpr int v[] = {8, 16};
};
template <>
struct VecSet<fkl::bf16_t, true> {
  static constexpr int v[] = {8, 16};
};
template <>
struct VecSet<fkl::e4m3_t, true> {
  static constexpr int v[] = {8, 16};
};

template <class ROp, class OutT, bool kSplit, bool kSwap, int V, int RY, int CAP>
cudaError_t run_float_chain(const LaunchCtx& c) {
  using RB = fkl::BatchRead<ROp, CAP>;
  using W = std::conditional_t<kSplit, fkl::WriteSplit<OutT>, fkl::WritePacked<OutT>>;
  const Spec& s = *c.spec;
  fkl::IOp<fkl::Mul3> mul;
  fkl::IOp<fkl::Sub3> sub;
  fkl::IOp<fkl::Div3> div;
  for (int k = 0; k < 3; ++k) {
    mul.params.c[k] = s.mul[k];
    sub.params.c[k] = s.sub[k];
    div.params.c[k] = s.div[k];
  }
  div.params.on = s.has_div ? 1 : 0;
  auto cops = [&] {
    if constexpr (kSwap) {
      return fkl::make_tuple(fkl::IOp<fkl::SwapRB<fkl::F3>>{}, mul, sub, div);
    } else {
      return fkl::make_tuple(mul, sub, div);
    }
  }();
  using Cops = decltype(cops);
  fkl::Args2D<RB, W, Cops> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.wp = c.out;
  a.cops = cops;
  a.H = c.H;
  a.W_ = c.W;
  return fkl::launch_transform2d<V, RY>(a, c.n, c.shape.tx, c.shape.ty, c.stream);
}

template <class ROp, class OutT, bool kSplit, bool kSwap, int V>
cudaError_t float_by_ry(const LaunchCtx& c) {
  const bool single = c.n <= 1;
  if (c.shape.ry == 1)
    return single ? run_float_chain<ROp, OutT, kSplit, kSwap, V, 1, 1>(c)
                  : run_float_chain<ROp, OutT, kSplit, kSwap, V, 1, kBatchCap>(c);
  if constexpr (V <= 8) {  // two rows of 16 pixels would not fit in registers
    if (c.shape.ry == 2)
      return single ? run_float_chain<ROp, OutT, kSplit, kSwap, V, 2, 1>(c)
                    : run_float_chain<ROp, OutT, kSplit, kSwap, V, 2, kBatchCap>(c);
  }
  return cudaErrorInvalidConfiguration;
}

template <class ROp, class OutT, bool kSplit, bool kSwap, size_t... I>
cudaError_t float_by_vec(const LaunchCtx& c, std::index_sequence<I...>) {
  cudaError_t err = cudaErrorInvalidConfiguration;
  const bool hit = ((c.shape.vec == VecSet<OutT, kSplit>::v[I]
                         ? (err = float_by_ry<ROp, OutT, kSplit, kSwap, VecSet<OutT, kSplit>::v[I]>(c), true)
                         : false) ||
                    ...);
  (void)hit;
  return err;
}

template <class ROp, class OutT, bool kSplit, bool kSwap>
cudaError_t float_by_type(const LaunchCtx& c) {
  constexpr size_t n = sizeof(VecSet<OutT, kSplit>::v) / sizeof(int);
  return float_by_vec<ROp, OutT, kSplit, kSwap>(c, std::make_index_sequence<n>{});
}

// Entry for one (ROp, output type): picks the packed/split writer and the
// swap variant. Each translation unit instantiates one output type.
template <class ROp, class OutT>
cudaError_t float_dispatch_type(const LaunchCtx& c) {
  const Spec& s = *c.spec;
  if (!s.split) {
    if constexpr (std::is_same_v<OutT, float>) {
      return s.swap ? float_by_type<ROp, float, false, true>(c) : float_by_type<ROp, float, false, false>(c);
    }
    return cudaErrorInvalidConfiguration;
  }
  return s.swap ? float_by_type<ROp, OutT, true, true>(c) : float_by_type<ROp, OutT, true, false>(c);
}

}  // namespace fkl_impl
