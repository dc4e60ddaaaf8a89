// Typed chains (paper §VI-I, the data-type experiment): Read -> Cast ->
// Multiply -> Subtract -> Divide -> Write over a batch of linear tensors.
// The input element is cast to the compute type CT (float64 for a float64
// output, float32 otherwise), then each present op runs once in CT with IEEE
// round-to-nearest-even; absent ops are skipped (a uniform branch). The
// write rounds to the output type (FP8: sat_RNE(v / s), with v / s formed as
// the float32 product with fl32(1/s): next to an E4M3 tie the code may be the
// neighbour of the rounded exact quotient, within one E4M3 ulp, and is
// otherwise the same). One thread handles E
// consecutive elements of one tensor; blockIdx.y is the tensor (horizontal
// fusion).
#pragma once

#include "core.cuh"

namespace fkl {

constexpr int kCastCap = 256;  // tensors per launch

struct CastArgs {
  const void* in[kCastCap];  // tensor z's elements
  void* out;                 // n * len elements of CT, tensor z at z * len
  int64_t len;               // elements per tensor
  int32_t n;                 // tensors in this launch
  int32_t has_mul, has_sub, has_div;
  float scale_inv;           // FP8 output: fl32(1 / s)
  double mul, sub, div;      // constants; each float converts exactly to CT
};

template <class OutT>
struct CastCompute {
  using type = float;
};
template <>
struct CastCompute<double> {
  using type = double;
};

template <class InT, class CT>
FKL_D CT cast_to(InT v) {
  if constexpr (std::is_same_v<InT, double> && std::is_same_v<CT, float>) {
    return __double2float_rn(v);
  } else {
    return static_cast<CT>(v);  // exact: u8, u16 and f32 in f32 or f64, f64 in f64
  }
}

FKL_D float mul_rn(float a, float b) { return __fmul_rn(a, b); }
FKL_D float sub_rn(float a, float b) { return __fsub_rn(a, b); }
FKL_D float div_rn(float a, float b) { return __fdiv_rn(a, b); }
FKL_D double mul_rn(double a, double b) { return __dmul_rn(a, b); }
FKL_D double sub_rn(double a, double b) { return __dsub_rn(a, b); }
FKL_D double div_rn(double a, double b) { return __ddiv_rn(a, b); }

// E elements as 16-byte (or 8-byte) vectors when they are aligned and whole.
template <class T, int E>
FKL_D void load_run(const T* p, bool vec, int n, T (&x)[E]) {
  constexpr int B = E * static_cast<int>(sizeof(T));
  if (vec) {
    if constexpr (B % 16 == 0) {
#pragma unroll
      for (int k = 0; k < B / 16; ++k) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(p) + k);
        reinterpret_cast<uint4*>(x)[k] = w;
      }
      return;
    } else if constexpr (B == 8) {
      const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
      reinterpret_cast<uint2*>(x)[0] = w;
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k)
    if (k < n) x[k] = __ldg(p + k);
}

template <class T, int E>
FKL_D void store_run_linear(T* p, bool vec, int n, const T (&x)[E]) {
  constexpr int B = E * static_cast<int>(sizeof(T));
  if (vec) {
    if constexpr (B % 16 == 0) {
#pragma unroll
      for (int k = 0; k < B / 16; ++k) __stcs(reinterpret_cast<uint4*>(p) + k, reinterpret_cast<const uint4*>(x)[k]);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k)
    if (k < n) p[k] = x[k];
}

template <class InT, class OutT, int E>
__global__ void __launch_bounds__(256) cast_chain_kernel(const __grid_constant__ CastArgs a) {
  using CT = typename CastCompute<OutT>::type;
  const int z = blockIdx.y;
  const int64_t i0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * E;
  if (z >= a.n || i0 >= a.len) return;
  const int n = a.len - i0 < E ? static_cast<int>(a.len - i0) : E;
  const InT* src = static_cast<const InT*>(a.in[z]) + i0;
  constexpr uintptr_t kInVec = E * sizeof(InT) >= 16 ? 16 : E * sizeof(InT);
  const bool vin = n == E && reinterpret_cast<uintptr_t>(src) % kInVec == 0;
  InT v[E];
  load_run<InT, E>(src, vin, n, v);
  const CT m = static_cast<CT>(a.mul), s = static_cast<CT>(a.sub), d = static_cast<CT>(a.div);
  CT x[E];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    CT t = cast_to<InT, CT>(v[k]);
    if (a.has_mul) t = mul_rn(t, m);
    if (a.has_sub) t = sub_rn(t, s);
    if (a.has_div) t = div_rn(t, d);
    x[k] = t;
  }
  if constexpr (std::is_same_v<OutT, double>) {
    double* dst = static_cast<double*>(a.out) + static_cast<int64_t>(z) * a.len + i0;
    store_run_linear<double, E>(dst, n == E && reinterpret_cast<uintptr_t>(dst) % 16 == 0, n, x);
  } else {
    constexpr int B = Format<OutT>::bytes;
    uint8_t* q = static_cast<uint8_t*>(a.out) + (static_cast<int64_t>(z) * a.len + i0) * B;
    if constexpr (std::is_same_v<OutT, e4m3_t>) {
#pragma unroll
      for (int k = 0; k < E; ++k) x[k] = __fmul_rn(x[k], a.scale_inv);
    }
    constexpr uintptr_t kOutVec = E * B >= 16 ? 16 : E * B;
    if (n == E && reinterpret_cast<uintptr_t>(q) % kOutVec == 0) {
      store_run<OutT, E>(q, x);
    } else {
#pragma unroll
      for (int k = 0; k < E; ++k)
        if (k < n) store_one<OutT>(q + k * B, x[k]);
    }
  }
}

}  // namespace fkl
