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

// One body, two kernels. The exact-2x NV12 read writing FP8 with 16 pixels
// per thread (78 registers when unbounded, 6 blocks of 128 threads per SM) is
// compiled for at least 4 blocks of 256 threads per SM (64 registers, 16-44
// spilled bytes): the extra occupancy lifted that chain by 5%. Every other
// variant keeps the compiler's register choice; under the same cap the
// 16-bit outputs, the general resize and the two-row variants spilled
// 44-550 bytes, and the 8-pixel ones already use <= 64 registers.
template <class RB, class W, int V, int RY>
struct OccupancyBound : std::false_type {};
template <int CAP>
struct OccupancyBound<BatchRead<ResizeNV12x2, CAP>, WriteSplit<e4m3_t, 3>, 16, 1> : std::true_type {};

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
      W::template exec_span<V>(Point{x0, y, z}, n, out, a.wp);
    }
  }
}

template <int V, int RY, class RB, class W, class Cops>
__global__ void __launch_bounds__(256) transform2d_kernel(const __grid_constant__ Args2D<RB, W, Cops> a) {
  transform2d_body<V, RY>(a);
}
template <int V, int RY, class RB, class W, class Cops>
__global__ void __launch_bounds__(256, 4) transform2d_occ_kernel(const __grid_constant__ Args2D<RB, W, Cops> a) {
  transform2d_body<V, RY>(a);
}

struct Shape2D {
  int vec, tx, ty, ry;
};

template <int V, int RY, class RB, class W, class Cops>
cudaError_t launch_transform2d(Args2D<RB, W, Cops>& a, int batch, int tx, int ty, cudaStream_t s) {
  const int cols = (a.W_ + V - 1) / V;
  const int rows = (a.H + RY - 1) / RY;
  const dim3 block(tx, ty, 1);
  const dim3 grid((cols + tx - 1) / tx, (rows + ty - 1) / ty, batch);
  if constexpr (OccupancyBound<RB, W, V, RY>::value) {
    transform2d_occ_kernel<V, RY, RB, W, Cops><<<grid, block, 0, s>>>(a);
  } else {
    transform2d_kernel<V, RY, RB, W, Cops><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

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

// ---------------------------------------------------------------------------
// Linear TransformDPP for 1-D float tensors (the vertical Mul/Add chain of
// paper §VI-B/§VI-G). The chain is a table of constants plus a bitmask of op
// kinds held in the kernel parameters; each thread keeps U float4 vectors in
// registers and applies every op to all of them before the next op, so the
// dependent chain of one element is interleaved with 4U - 1 independent ones.
// ---------------------------------------------------------------------------
template <int CAP>
struct VChainParams {
  const void* in;  // float32, or u8 converted exactly
  float* out;
  int64_t n;          // elements
  int32_t len;        // ops in this launch (<= CAP)
  int32_t alternating;  // 1: kinds are Mul, Add, Mul, Add, ... from op 0
  uint32_t add_mask[(CAP + 31) / 32];  // bit i set: op i is an Add
  float c[CAP];
};

// E consecutive input elements as floats (vector loads when `vec`).
template <class InT, int E>
FKL_D void vchain_load(const void* in, int64_t base, int64_t n, bool vec, float (&x)[E]) {
  if constexpr (std::is_same_v<InT, float>) {
    const float* f = static_cast<const float*>(in);
    if (vec) {
#pragma unroll
      for (int u = 0; u < E / 4; ++u) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(f + base) + u);
        x[4 * u] = v.x;
        x[4 * u + 1] = v.y;
        x[4 * u + 2] = v.z;
        x[4 * u + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = base + e < n ? f[base + e] : 0.f;
    }
  } else {
    static_assert(std::is_same_v<InT, uint8_t> && E % 8 == 0, "u8 chains load 8-byte multiples");
    const uint8_t* b = static_cast<const uint8_t*>(in);
    if (vec) {
      uint32_t w[E / 4];
      if constexpr (E == 8) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(b + base));
        w[0] = v.x;
        w[1] = v.y;
      } else {
#pragma unroll
        for (int u = 0; u < E / 16; ++u) {
          const uint4 v = __ldcs(reinterpret_cast<const uint4*>(b + base) + u);
          w[4 * u] = v.x;
          w[4 * u + 1] = v.y;
          w[4 * u + 2] = v.z;
          w[4 * u + 3] = v.w;
        }
      }
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = static_cast<float>((w[e / 4] >> (8 * (e % 4))) & 0xFFu);
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = base + e < n ? static_cast<float>(b[base + e]) : 0.f;
    }
  }
}

template <int U, int CAP, bool kAlt, class InT = float>
__global__ void __launch_bounds__(512) vchain_kernel(const __grid_constant__ VChainParams<CAP> p) {
  constexpr int E = 4 * U;  // elements per thread
  constexpr int kInBytes = static_cast<int>(sizeof(InT));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * E;
  for (int64_t base = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * E; base < p.n;
       base += stride) {
    float x[E];
    const bool full = base + E <= p.n && (reinterpret_cast<uintptr_t>(p.in) % (kInBytes * E < 16 ? kInBytes * E : 16)) == 0 &&
                      (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
    vchain_load<InT, E>(p.in, base, p.n, full, x);
    if constexpr (kAlt) {
      // Mul, Add pairs: no per-op branch.
      int i = 0;
#pragma unroll 1
      for (; i + 1 < p.len; i += 2) {
        const float cm = p.c[i], ca = p.c[i + 1];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = __fadd_rn(__fmul_rn(x[e], cm), ca);
      }
      if (i < p.len) {
        const float cm = p.c[i];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], cm);
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < p.len; ++i) {
        const float c = p.c[i];
        if ((p.add_mask[i >> 5] >> (i & 31)) & 1u) {
#pragma unroll
          for (int e = 0; e < E; ++e) x[e] = __fadd_rn(x[e], c);
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], c);
        }
      }
    }
    if (full) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        __stcs(reinterpret_cast<float4*>(p.out + base) + u,
               make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]));
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (base + e < p.n) p.out[base + e] = x[e];
    }
  }
}

}  // namespace fkl
