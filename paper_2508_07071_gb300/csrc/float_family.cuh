// Instantiation and dispatch of the float image chains
//   ROp -> [SwapRB] -> Mul -> Sub -> Div -> Write{Split,Packed}<OutT>
// for one resampling ROp. Included by exactly one translation unit per ROp
// (k_packed.cu, k_nv12.cu) so the families compile in parallel.
#pragma once

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "fkl/staged.cuh"
#include "fkl/tiles.cuh"
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

// The packed-u8 reader also takes 1 and 2 pixels per thread: its workloads
// (one image, crops) are small, and more threads in flight hide their
// latency. (The NV12 exact-2x path reads 16-byte vectors: 8 pixels or more.)
template <class ROp, class OutT, bool kSplit>
struct VecSetFor : VecSet<OutT, kSplit> {};
template <>
struct VecSetFor<fkl::ResizeU8C3, float, true> {
  static constexpr int v[] = {1, 2, 4, 8};
};
template <>
struct VecSetFor<fkl::ResizeU8C3, fkl::f16_t, true> {
  static constexpr int v[] = {2, 8, 16};
};
template <>
struct VecSetFor<fkl::ResizeU8C3, fkl::bf16_t, true> {
  static constexpr int v[] = {2, 8, 16};
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
constexpr int kMidCap = 64;  // 4 KB of parameters: crop batches of tens of images
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
    if (c.n <= kMidCap) return run_float_chain_cap<ROp, OutT, kSplit, kSwap, kTail, V, RY, kMidCap>(c);
  }
  return run_float_chain_cap<ROp, OutT, kSplit, kSwap, kTail, V, RY, kBatchCap>(c);
}

// Row-staged launch (shape.ry <= 0, shape.ty = output rows per job) of the
// exact-2x NV12 read: a persistent grid of min(jobs, SMs x resident CTAs)
// CTAs of shape.tx threads with a ring of -shape.ry stages (shape.ry == 0:
// as many as fill about kStageBudget bytes, 2..kMaxStages).
constexpr int kStageBudget = 64 * 1024;
constexpr int kStagedSmemMax = 200 * 1024;

inline int staged_stages(const fkl_launch_shape& sh, int stage_bytes) {
  if (sh.ry < 0) return -sh.ry;
  return std::max(2, std::min(fkl::kMaxStages, kStageBudget / std::max(stage_bytes, 1)));
}

template <class OutT, bool kSwap, int kTail, int V>
cudaError_t run_staged(const LaunchCtx& c) {
  using RB = fkl::BatchRead<fkl::ResizeNV12x2, kBatchCap>;
  using W = fkl::WriteSplit<OutT>;
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
  fkl::StagedArgs<RB, W, Cops> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.wp = c.out;
  a.cops = cops;
  a.H = c.H;
  a.W_ = c.W;
  a.R = c.shape.ty;
  a.row_bytes = 2 * c.W;
  const int stage_bytes = 3 * a.R * a.row_bytes;
  a.stages = staged_stages(c.shape, stage_bytes);
  a.jobs_per_image = (c.H + a.R - 1) / a.R;
  a.jobs = c.n * a.jobs_per_image;
  a.error = c.device_error;
  a.wait_ns = c.wait_ns ? c.wait_ns : 1000000000ull;
  const int smem = a.stages * stage_bytes;
  if (a.jobs == 0) return cudaSuccess;

  auto kernel = fkl::staged_nv12x2_kernel<V, RB, W, Cops>;
  // per (device, threads, shared bytes): resident CTAs per SM, after the
  // kernel's shared-memory limit has been raised once on that device
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> resident;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, c.shape.tx, smem);
    auto it = resident.find(key);
    if (it == resident.end()) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, c.shape.tx, smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      resident.emplace(key, per_sm);
    } else {
      per_sm = it->second;
    }
  }
  const int grid = std::min(a.jobs, sm_count() * per_sm);
  kernel<<<grid, c.shape.tx, smem, c.stream>>>(a);
  return cudaGetLastError();
}

// Whether the row-staged kernel can run this launch (its preconditions).
inline bool staged_eligible(const LaunchCtx& c, int V) {
  if (!c.all_exact2x || !c.device_error || c.W % V || (2 * c.W) % 16) return false;
  if (c.shape.ty < 1 || c.shape.tx < 32 || c.shape.tx > 256 || c.shape.tx % 32) return false;
  const int stage_bytes = 3 * c.shape.ty * 2 * c.W;
  const int stages = staged_stages(c.shape, stage_bytes);
  if (stages < 2 || stages > fkl::kMaxStages || int64_t(stages) * stage_bytes > kStagedSmemMax) return false;
  for (int i = 0; i < c.n; ++i) {
    const auto& p = c.imgs[i];
    if (!(p.flags & fkl::kFast2x) || p.ox != 0 || p.dw != c.W) return false;
  }
  return true;
}

// Tile-staged launch of the packed reader (shape.ry == -1): tiles of
// (shape.tx * V) x shape.ty outputs, each staging its tap rows' column span in
// shared memory. Eligible when every image's span fits kTileSmemMax bytes.
constexpr int kTileSmemMax = 48 * 1024;

// Shared bytes per staged row for this launch (0: a span does not fit).
inline int tile_row_stride(const LaunchCtx& c, int V) {
  if (c.shape.ty < 1 || c.shape.ty > fkl::kTileMaxRows || c.shape.tx < 1 || c.shape.tx * c.shape.ty > 256) return 0;
  const int64_t tile_w = int64_t(c.shape.tx) * V;
  int64_t nb_max = 0;
  for (int i = 0; i < c.n; ++i) {
    const auto& p = c.imgs[i];
    // tap columns of tile_w consecutive outputs span at most
    // (tile_w - 1) rw / dw + 3 source pixels
    const int64_t span = ((tile_w - 1) * p.rw + p.dw - 1) / p.dw + 3;
    nb_max = std::max(nb_max, 3 * span);
  }
  const int64_t stride = ((nb_max + 30) / 16 + 1) * 16;
  return 2 * c.shape.ty * stride <= kTileSmemMax ? static_cast<int>(stride) : 0;
}

template <class OutT, bool kSplit, bool kSwap, int kTail, int V, int CAP>
cudaError_t run_tiles_cap(const LaunchCtx& c, int stride) {
  using RB = fkl::BatchRead<fkl::ResizeU8C3, CAP>;
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
  fkl::TileArgs<RB, W, Cops> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.wp = c.out;
  a.cops = cops;
  a.H = c.H;
  a.W_ = c.W;
  a.row_stride = stride;
  const int tile_w = c.shape.tx * V;
  const dim3 grid((c.W + tile_w - 1) / tile_w, (c.H + c.shape.ty - 1) / c.shape.ty, c.n);
  fkl::tile_resize_kernel<V, RB, W, Cops><<<grid, dim3(c.shape.tx, c.shape.ty, 1), 2 * c.shape.ty * stride,
                                              c.stream>>>(a);
  return cudaGetLastError();
}

template <class OutT, bool kSplit, bool kSwap, int kTail, int V>
cudaError_t run_tiles(const LaunchCtx& c, int stride) {
  if (c.n <= kSmallCap) return run_tiles_cap<OutT, kSplit, kSwap, kTail, V, kSmallCap>(c, stride);
  if (c.n <= kMidCap) return run_tiles_cap<OutT, kSplit, kSwap, kTail, V, kMidCap>(c, stride);
  return run_tiles_cap<OutT, kSplit, kSwap, kTail, V, kBatchCap>(c, stride);
}

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, int V>
cudaError_t float_by_ry(const LaunchCtx& c) {
  if constexpr (std::is_same_v<ROp, fkl::ResizeU8C3> && V <= 4) {
    if (c.shape.ry == -1) {
      const int stride = tile_row_stride(c, V);
      if (stride > 0) return run_tiles<OutT, kSplit, kSwap, kTail, V>(c, stride);
    }
  }
  if (c.shape.ry <= 0) {
    if constexpr (std::is_same_v<ROp, fkl::ResizeNV12x2> && kSplit && V % 8 == 0) {
      if (staged_eligible(c, V)) return run_staged<OutT, kSwap, kTail, V>(c);
    }
    // not eligible: the register kernel with a fixed block
    LaunchCtx d = c;
    d.shape = fkl_launch_shape{V, 32, 8, 1};
    return run_float_chain<ROp, OutT, kSplit, kSwap, kTail, V, 1>(d);
  }
  if (c.shape.ry == 1) return run_float_chain<ROp, OutT, kSplit, kSwap, kTail, V, 1>(c);
  if constexpr (V <= 8) {  // two rows of 16 pixels would not fit in registers
    if (c.shape.ry == 2) return run_float_chain<ROp, OutT, kSplit, kSwap, kTail, V, 2>(c);
  }
  return cudaErrorInvalidConfiguration;
}

template <class ROp, class OutT, bool kSplit, bool kSwap, int kTail, size_t... I>
cudaError_t float_by_vec(const LaunchCtx& c, std::index_sequence<I...>) {
  cudaError_t err = cudaErrorInvalidConfiguration;
  const bool hit = ((c.shape.vec == VecSetFor<ROp, OutT, kSplit>::v[I]
                         ? (err = float_by_ry<ROp, OutT, kSplit, kSwap, kTail, VecSetFor<ROp, OutT, kSplit>::v[I]>(c),
                            true)
                         : false) ||
                    ...);
  (void)hit;
  return err;
}

template <class ROp, class OutT, bool kSplit, bool kSwap>
cudaError_t float_by_type(const LaunchCtx& c) {
  constexpr size_t n = sizeof(VecSetFor<ROp, OutT, kSplit>::v) / sizeof(int);
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
