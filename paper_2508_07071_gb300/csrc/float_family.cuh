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

// Compute ops after the optional swap, fixed at compile time so that an
// absent op costs nothing: 0 = Mul; 1 = Mul, Sub; 2 = Mul, Sub, Div.
// (An absent Mul or Sub inside a tail is bound as its exact identity.)
inline int tail_of(const Spec& s) { return s.has_div ? 2 : (s.has_sub ? 1 : 0); }

template <int kTail>
auto make_tail(const Spec& s) {
  fkl::IOp<fkl::Mul3> mul;
  fkl::IOp<fkl::Sub3> sub;
  fkl::IOp<fkl::Div3> div;
  for (int k = 0; k < 3; ++k) {
    mul.params.c[k] = s.mul[k];
    sub.params.c[k] = s.sub[k];
    div.params.c[k] = s.div[k];
  }
  div.params.on = 1;
  if constexpr (kTail == 0) {
    return fkl::make_tuple(mul);
  } else if constexpr (kTail == 1) {
    return fkl::make_tuple(mul, sub);
  } else {
    return fkl::make_tuple(mul, sub, div);
  }
}

// Batches of up to kSmallCap images use a small parameter block (a launch
// carries its whole parameter block, 16 KB for kBatchCap entries), for ROps
// that serve single images.
constexpr int kSmallCap = 8;
template <class ROp>
struct SmallBatches : std::false_type {};
template <>
struct SmallBatches<fkl::ResizeU8C3> : std::true_type {};

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, int V, int RY, int CAP>
cudaError_t run_float_chain_cap(const LaunchCtx& c) {
  using RB = fkl::BatchRead<ROp, CAP>;
  using W = std::conditional_t<kSplit, fkl::WriteSplit<OutT>, fkl::WritePacked<OutT>>;
  const Spec& s = *c.spec;
  auto tail = make_tail<kTail>(s);
  auto cops = [&] {
    if constexpr (kSwap) {
      return fkl::prepend(fkl::IOp<fkl::SwapRB<fkl::F3>>{}, tail);
    } else {
      return tail;
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

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, int V, int RY>
cudaError_t run_float_chain(const LaunchCtx& c) {
  if constexpr (SmallBatches<ROp>::value) {
    if (c.n <= kSmallCap) return run_float_chain_cap<ROp, OutT, kSplit, kSwap, kTail, V, RY, kSmallCap>(c);
  }
  return run_float_chain_cap<ROp, OutT, kSplit, kSwap, kTail, V, RY, kBatchCap>(c);
}

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, int V>
cudaError_t float_by_ry(const LaunchCtx& c) {
  if (c.shape.ry == 1) return run_float_chain<ROp, OutT, kSplit, kSwap, kTail, V, 1>(c);
  if constexpr (V <= 8) {  // two rows of 16 pixels would not fit in registers
    if (c.shape.ry == 2) return run_float_chain<ROp, OutT, kSplit, kSwap, kTail, V, 2>(c);
  }
  return cudaErrorInvalidConfiguration;
}

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, size_t... I>
cudaError_t float_by_vec(const LaunchCtx& c, std::index_sequence<I...>) {
  cudaError_t err = cudaErrorInvalidConfiguration;
  const bool hit = ((c.shape.vec == VecSet<OutT, kSplit>::v[I]
                         ? (err = float_by_ry<ROp, OutT, kSplit, kSwap, kTail, VecSet<OutT, kSplit>::v[I]>(c), true)
                         : false) ||
                    ...);
  (void)hit;
  return err;
}

template <class ROp, class OutT, bool kSplit, bool kSwap>
cudaError_t float_by_type(const LaunchCtx& c) {
  constexpr size_t n = sizeof(VecSet<OutT, kSplit>::v) / sizeof(int);
  switch (tail_of(*c.spec)) {
    case 0:
      return float_by_vec<ROp, OutT, kSplit, kSwap, 0>(c, std::make_index_sequence<n>{});
    case 1:
      return float_by_vec<ROp, OutT, kSplit, kSwap, 1>(c, std::make_index_sequence<n>{});
    default:
      return float_by_vec<ROp, OutT, kSplit, kSwap, 2>(c, std::make_index_sequence<n>{});
  }
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
