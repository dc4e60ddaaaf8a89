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

template <int V, int RY, class RB, class W, class Cops>
__global__ void __launch_bounds__(256) transform2d_kernel(const __grid_constant__ Args2D<RB, W, Cops> a) {
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
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = apply_chain(in[r][k], a.cops);
      W::template exec_span<V>(Point{x0, y, z}, n, out, a.wp);
    }
  }
}

struct Shape2D {
  int vec, tx, ty, ry;
};

template <int V, int RY, class RB, class W, class Cops>
cudaError_t launch_transform2d(const Args2D<RB, W, Cops>& a, int batch, int tx, int ty,
                               cudaStream_t s) {
  const int cols = (a.W_ + V - 1) / V;
  const int rows = (a.H + RY - 1) / RY;
  const dim3 block(tx, ty, 1);
  const dim3 grid((cols + tx - 1) / tx, (rows + ty - 1) / ty, batch);
  transform2d_kernel<V, RY, RB, W, Cops><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
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
  const float* in;
  float* out;
  int64_t n;          // elements
  int32_t len;        // ops in this launch (<= CAP)
  int32_t alternating;  // 1: kinds are Mul, Add, Mul, Add, ... from op 0
  uint32_t add_mask[(CAP + 31) / 32];  // bit i set: op i is an Add
  float c[CAP];
};

template <int U, int CAP, bool kAlt>
__global__ void __launch_bounds__(512) vchain_kernel(const __grid_constant__ VChainParams<CAP> p) {
  constexpr int E = 4 * U;  // elements per thread
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * E;
  for (int64_t base = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * E; base < p.n;
       base += stride) {
    float x[E];
    const bool full = base + E <= p.n && (reinterpret_cast<uintptr_t>(p.in) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
    if (full) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(p.in + base) + u);
        x[4 * u] = v.x;
        x[4 * u + 1] = v.y;
        x[4 * u + 2] = v.z;
        x[4 * u + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = base + e < p.n ? p.in[base + e] : 0.f;
    }
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
