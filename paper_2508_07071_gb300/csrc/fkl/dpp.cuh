// Data Parallel Patterns (paper §IV-C): thread organisation only. A DPP
// holds no data-touching code; it decides which thread handles which output
// and calls the Ops' exec functions in chain order.
#pragma once

#include "ops.cuh"

namespace fkl {

// ---------------------------------------------------------------------------
// TransformDPP over 2-D outputs with thread coarsening (paper §IV-C Fig. 11):
// each thread owns V consecutive output pixels of RY consecutive rows and
// writes each plane's V values with one vector store. blockIdx.z is the batch
// index (horizontal fusion, paper §II Fig. 6, §IV-B).
// ---------------------------------------------------------------------------
template <class RB, class W, class Cops>
struct Args2D {
  typename RB::ParamsType rp;
  typename W::ParamsType wp;
  Cops cops;
  int32_t H, W_;  // output rows and columns per image
};

// One body, two kernels. Most variants keep the compiler's register choice;
// the exact-2x NV12 read writing 16-bit or FP8 planes is compiled for a
// minimum number of resident 256-thread blocks per SM (OccupancyBound), which
// caps its registers: 8 pixels per thread, bf16/f16, 6 blocks (40 registers
// instead of 48, 16 spilled bytes; +2% on 256 frames); 16 pixels per thread,
// FP8, 4 blocks (64 instead of 78, 32 spilled bytes; +5%). These loads are
// latency-bound, so more resident warps pay for the spills; under the same
// caps the general resize and the two-row variants spilled 44-550 bytes.
template <class RB, class W, int V, int RY>
struct OccupancyBase : std::integral_constant<int, 0> {};  // 0: the compiler's choice
template <int CAP>
struct OccupancyBase<BatchRead<ResizeNV12x2, CAP>, WriteSplit<e4m3_t, 3>, 16, 1> : std::integral_constant<int, 4> {};
template <int CAP>
struct OccupancyBase<BatchRead<ResizeNV12x2, CAP>, WriteSplit<bf16_t, 3>, 8, 1> : std::integral_constant<int, 6> {};
template <int CAP>
struct OccupancyBase<BatchRead<ResizeNV12x2, CAP>, WriteSplit<f16_t, 3>, 8, 1> : std::integral_constant<int, 6> {};
// Only chains that run on packed pixel pairs (a chain that divides does not,
// and spilled 44-80 bytes under the cap).
template <class RB, class W, class Cops, int V, int RY>
struct OccupancyBound
    : std::integral_constant<int, ChainHasPair<Cops>::value ? OccupancyBase<RB, W, V, RY>::value : 0> {};

// A WOp may offer prepare(params): the parameters its threads write with,
// computed once when a thread starts.
template <class W, class = void>
struct HasPrepare : std::false_type {};
template <class W>
struct HasPrepare<W, std::void_t<decltype(&W::prepare)>> : std::true_type {};

// A read may offer fill(pt, n, params, v): whether its n outputs from pt are
// all one fill value v (the letterbox area of a placed image).
template <class RB, class = void>
struct HasFill : std::false_type {};
template <class RB>
struct HasFill<RB, std::void_t<decltype(&RB::fill)>> : std::true_type {};

template <int V, int RY, class RB, class W, class Cops>
FKL_D void transform2d_body(const Args2D<RB, W, Cops>& a) {
  using RT = typename RB::OutputType;
  using WT = typename ChainResult<RT, Cops>::type;
  static_assert(std::is_same_v<WT, typename W::InputType>, "chain output must match the WOp input");

  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const int ybase = (blockIdx.y * blockDim.y + threadIdx.y) * RY;
  const int z = blockIdx.z;
  if (x0 >= a.W_ || z >= a.rp.count) return;
  const int n = min(V, a.W_ - x0);
  const typename W::ParamsType wp = [&] {
    if constexpr (HasPrepare<W>::value) {
      return W::prepare(a.wp);
    } else {
      return a.wp;
    }
  }();

  // A span wholly in the fill runs the chain once and writes that value V
  // times (the same bits as the per-pixel path: every lane of a packed op
  // rounds as the scalar op); the write's conversions collapse to one.
  if constexpr (RY == 1 && HasFill<RB>::value) {
    RT fv;
    if (ybase < a.H && RB::fill(Point{x0, ybase, z}, n, a.rp, fv)) {
      const WT o = apply_chain(fv, a.cops);
      WT out[V];
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = o;
      W::template exec_span<V>(Point{x0, ybase, z}, n, out, wp);
      return;
    }
  }

  // Read every row first so that all loads of the thread are in flight
  // before the first store.
  RT in[RY][V];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = ybase + r;
    if (y < a.H) {
      const Point pt{x0, y, z};
      if (n == V) {
        RB::template exec_span<V>(pt, a.rp, in[r]);
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
          if (k < n) in[r][k] = RB::exec(Point{x0 + k, y, z}, a.rp);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = ybase + r;
    if (y < a.H) {
      WT out[V];
      if constexpr (ChainHasPair<Cops>::value && std::is_same_v<RT, F3> && std::is_same_v<WT, F3> && V % 2 == 0) {
#pragma unroll
        for (int k = 0; k < V; k += 2)
          unpack_pair(apply_chain_pair(pack_pair(in[r][k], in[r][k + 1]), a.cops), out[k], out[k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = apply_chain(in[r][k], a.cops);
      }
      W::template exec_span<V>(Point{x0, y, z}, n, out, wp);
    }
  }
}

template <int V, int RY, class RB, class W, class Cops>
__global__ void __launch_bounds__(256) transform2d_kernel(const __grid_constant__ Args2D<RB, W, Cops> a) {
  transform2d_body<V, RY>(a);
}
template <int V, int RY, int kMinBlocks, class RB, class W, class Cops>
__global__ void __launch_bounds__(256, kMinBlocks) transform2d_occ_kernel(const __grid_constant__ Args2D<RB, W, Cops> a) {
  transform2d_body<V, RY>(a);
}

template <int V, int RY, class RB, class W, class Cops>
cudaError_t launch_transform2d(Args2D<RB, W, Cops>& a, int batch, int tx, int ty, cudaStream_t s) {
  const int cols = (a.W_ + V - 1) / V;
  const int rows = (a.H + RY - 1) / RY;
  const dim3 block(tx, ty, 1);
  const dim3 grid((cols + tx - 1) / tx, (rows + ty - 1) / ty, batch);
  constexpr int kMinBlocks = OccupancyBound<RB, W, Cops, V, RY>::value;
  if constexpr (kMinBlocks > 0) {
    transform2d_occ_kernel<V, RY, kMinBlocks, RB, W, Cops><<<grid, block, 0, s>>>(a);
  } else {
    transform2d_kernel<V, RY, RB, W, Cops><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace fkl
