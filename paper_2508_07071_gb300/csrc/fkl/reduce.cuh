#pragma once

#include "ops.cuh"

namespace fkl {

// ---------------------------------------------------------------------------
// ReduceDPP (paper §IV-C, the reduction pattern): the ROp and COps of a chain
// are evaluated once per output pixel, as in TransformDPP, and the values
// feed several reductions at once instead of a write: per-channel minimum,
// maximum and sum, and the maximum absolute value. Per thread, then per warp
// (shuffles), then per block (shared memory), then one atomic per block and
// statistic. Min/max travel as order-preserving unsigned keys; sums as
// 64-bit fixed point (2^-20), so every accumulation is exact integer
// arithmetic and the result does not depend on the order blocks finish.
// ---------------------------------------------------------------------------
struct ReduceAcc {
  unsigned int min_key[3];
  unsigned int max_key[3];
  unsigned long long sum_fx[3];  // two's complement fixed point, 2^-20 units
  unsigned int absmax_key;
  unsigned int _pad;
};
constexpr float kSumScale = 1048576.f;  // 2^20

FKL_D unsigned int order_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
FKL_D float key_value(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

template <class RB, class Cops>
struct ReduceArgs {
  typename RB::ParamsType rp;
  Cops cops;
  int32_t H, W_;
  ReduceAcc* acc;
};

template <int V, class RB, class Cops>
__global__ void __launch_bounds__(256) reduce2d_kernel(const __grid_constant__ ReduceArgs<RB, Cops> a) {
  using RT = typename RB::OutputType;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  float mn[3], mx[3], sm[3], am = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mn[c] = __int_as_float(0x7f800000);
    mx[c] = -__int_as_float(0x7f800000);
    sm[c] = 0.f;
  }
  if (x0 < a.W_ && y < a.H && z < a.rp.count) {
    const int n = min(V, a.W_ - x0);
    RT in[V];
    const Point pt{x0, y, z};
    if (n == V) {
      RB::template exec_span<V>(pt, a.rp, in);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (k < n) in[k] = RB::exec(Point{x0 + k, y, z}, a.rp);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      if (k < n) {
        const auto v = apply_chain(in[k], a.cops);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mn[c] = fminf(mn[c], v.v[c]);
          mx[c] = fmaxf(mx[c], v.v[c]);
          sm[c] = __fadd_rn(sm[c], v.v[c]);
          am = fmaxf(am, fabsf(v.v[c]));
        }
      }
    }
  }
  unsigned int kmin[3], kmax[3], kabs = order_key(am);
  long long fx[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    kmin[c] = order_key(mn[c]);
    kmax[c] = order_key(mx[c]);
    fx[c] = __float2ll_rn(__fmul_rn(sm[c], kSumScale));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      kmin[c] = min(kmin[c], __shfl_xor_sync(0xffffffffu, kmin[c], off));
      kmax[c] = max(kmax[c], __shfl_xor_sync(0xffffffffu, kmax[c], off));
      fx[c] += __shfl_xor_sync(0xffffffffu, fx[c], off);
    }
    kabs = max(kabs, __shfl_xor_sync(0xffffffffu, kabs, off));
  }
  __shared__ unsigned int s_min[8][3], s_max[8][3], s_abs[8];
  __shared__ long long s_sum[8][3];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s_min[warp][c] = kmin[c];
      s_max[warp][c] = kmax[c];
      s_sum[warp][c] = fx[c];
    }
    s_abs[warp] = kabs;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < nwarps; ++w) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        kmin[c] = min(kmin[c], s_min[w][c]);
        kmax[c] = max(kmax[c], s_max[w][c]);
        fx[c] += s_sum[w][c];
      }
      kabs = max(kabs, s_abs[w]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(&a.acc->min_key[c], kmin[c]);
      atomicMax(&a.acc->max_key[c], kmax[c]);
      atomicAdd(&a.acc->sum_fx[c], static_cast<unsigned long long>(fx[c]));
    }
    atomicMax(&a.acc->absmax_key, kabs);
  }
}

}  // namespace fkl
