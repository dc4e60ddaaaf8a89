#pragma once

#include "ops.cuh"

namespace fkl {

// ---------------------------------------------------------------------------
// ReduceDPP (paper §IV-C, the reduction pattern): the ROp and COps of a chain
// are evaluated once per output pixel, as in TransformDPP, and the values
// feed several reductions at once instead of a write: per-channel minimum,
// maximum and sum (the maximum absolute value follows from the extremes).
// A persistent grid of blocks walks jobs of blockDim.y rows x blockDim.x * V
// columns of one image; every thread keeps its minima and maxima as floats
// and its sums as 64-bit fixed point (2^-20; each job's V values are summed
// in float32 first), then per warp (shuffles), per block (shared memory) and
// one atomic per block and statistic. Min/max travel as order-preserving
// unsigned keys and the sums are integers, so the result does not depend on
// the order in which blocks finish.
// ---------------------------------------------------------------------------
struct ReduceAcc {
  unsigned int min_key[3];
  unsigned int max_key[3];
  unsigned long long sum_fx[3];  // two's complement fixed point, 2^-20 units
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
  int32_t col_tiles;  // jobs per row band: ceil(ceil(W_ / V) / blockDim.x)
  int32_t row_tiles;  // row bands per image: ceil(H / blockDim.y)
  ReduceAcc* acc;
};

// Folds n <= V chain values into the thread's extremes and sums.
template <int V, class Cops>
FKL_D void reduce_values(const Cops& cops, const F3 (&in)[V], int n, float (&mn)[3], float (&mx)[3],
                         long long (&fx)[3]) {
  float ps[3] = {0.f, 0.f, 0.f};
  if constexpr (ChainHasPair<Cops>::value && V % 2 == 0) {
    if (n == V) {
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        F3 v0, v1;
        unpack_pair(apply_chain_pair(pack_pair(in[k], in[k + 1]), cops), v0, v1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mn[c] = fminf(mn[c], fminf(v0.v[c], v1.v[c]));
          mx[c] = fmaxf(mx[c], fmaxf(v0.v[c], v1.v[c]));
          ps[c] = __fadd_rn(__fadd_rn(ps[c], v0.v[c]), v1.v[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) fx[c] += __float2ll_rn(__fmul_rn(ps[c], kSumScale));
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (k < n) {
      const auto v = apply_chain(in[k], cops);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        mn[c] = fminf(mn[c], v.v[c]);
        mx[c] = fmaxf(mx[c], v.v[c]);
        ps[c] = __fadd_rn(ps[c], v.v[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) fx[c] += __float2ll_rn(__fmul_rn(ps[c], kSumScale));
}

template <int V, class RB, class Cops>
FKL_D void reduce_span(const ReduceArgs<RB, Cops>& a, int x0, int y, int z, float (&mn)[3], float (&mx)[3],
                       long long (&fx)[3]) {
  using RT = typename RB::OutputType;
  static_assert(std::is_same_v<RT, F3>, "reductions run on three-channel float values");
  const int n = min(V, a.W_ - x0);
  if constexpr (Placed<typename RB::Op>::value) {
    const ResampleParams& q = a.rp.p[z];
    if (fill_span(q, x0, y, n)) {  // n copies of one value: the chain runs once
      const auto v = apply_chain(F3{{q.pad, q.pad, q.pad}}, a.cops);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        mn[c] = fminf(mn[c], v.v[c]);
        mx[c] = fmaxf(mx[c], v.v[c]);
        fx[c] += __float2ll_rn(__fmul_rn(__fmul_rn(v.v[c], static_cast<float>(n)), kSumScale));
      }
      return;
    }
  }
  RT in[V];
  const Point pt{x0, y, z};
  if (n == V) {
    RB::template exec_span<V>(pt, a.rp, in);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (k < n) in[k] = RB::exec(Point{x0 + k, y, z}, a.rp);
  }
  reduce_values<V>(a.cops, in, n, mn, mx, fx);
}

template <int V, class RB, class Cops>
FKL_D void reduce2d_body(const ReduceArgs<RB, Cops>& a) {
  float mn[3], mx[3];
  long long fx[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mn[c] = __int_as_float(0x7f800000);
    mx[c] = -__int_as_float(0x7f800000);
    fx[c] = 0;
  }
  // jobs in (image, row band, column tile) order; the job index is the same
  // for the whole block
  const int per_image = a.col_tiles * a.row_tiles;
  const int jobs = per_image * a.rp.count;
  for (int job = blockIdx.x; job < jobs; job += gridDim.x) {
    const int z = job / per_image;
    const int r = job - z * per_image;
    const int band = r / a.col_tiles;
    const int x0 = ((r - band * a.col_tiles) * blockDim.x + threadIdx.x) * V;
    const int y = band * blockDim.y + threadIdx.y;
    if (x0 < a.W_ && y < a.H) reduce_span<V>(a, x0, y, z, mn, mx, fx);
  }
  unsigned int kmin[3], kmax[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    kmin[c] = order_key(mn[c]);
    kmax[c] = order_key(mx[c]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      kmin[c] = min(kmin[c], __shfl_xor_sync(0xffffffffu, kmin[c], off));
      kmax[c] = max(kmax[c], __shfl_xor_sync(0xffffffffu, kmax[c], off));
      fx[c] += __shfl_xor_sync(0xffffffffu, fx[c], off);
    }
  }
  __shared__ unsigned int s_min[8][3], s_max[8][3];
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
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(&a.acc->min_key[c], kmin[c]);
      atomicMax(&a.acc->max_key[c], kmax[c]);
      atomicAdd(&a.acc->sum_fx[c], static_cast<unsigned long long>(fx[c]));
    }
  }
}

// kMinBlocks > 0 caps the registers so that many 256-thread blocks are
// resident per SM (more loads in flight); 0 keeps the compiler's choice.
template <int V, int kMinBlocks, class RB, class Cops>
__global__ void __launch_bounds__(256, kMinBlocks > 0 ? kMinBlocks : 1)
    reduce2d_kernel(const __grid_constant__ ReduceArgs<RB, Cops> a) {
  reduce2d_body<V>(a);
}

}  // namespace fkl
