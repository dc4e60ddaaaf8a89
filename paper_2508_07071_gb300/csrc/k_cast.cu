// Typed chains over batches of linear tensors (paper §VI-I): the fused form
// (one launch per 256 tensors) and the unfused form (one kernel per op and
// tensor, each a full read and write of the tensor; 16-bit and FP8 outputs
// add a final kernel that writes the output type from a float32 workspace).
#include <algorithm>
#include <cstring>

#include "fkl/cast.cuh"
#include "registry.h"

namespace fkl_impl {

namespace {

template <class InT, class OutT, int E>
cudaError_t run(const fkl::CastArgs& a, int block, cudaStream_t st) {
  const int64_t per_block = static_cast<int64_t>(block) * E;
  const int64_t gx = (a.len + per_block - 1) / per_block;
  if (gx == 0 || a.n == 0) return cudaSuccess;
  if (gx > 0x7fffffff) return cudaErrorInvalidConfiguration;
  fkl::cast_chain_kernel<InT, OutT, E><<<dim3(static_cast<unsigned>(gx), a.n, 1), block, 0, st>>>(a);
  return cudaGetLastError();
}

template <class InT, class OutT>
cudaError_t by_vec(const fkl::CastArgs& a, const fkl_launch_shape& sh, cudaStream_t st) {
  switch (sh.vec) {
    case 8:
      return run<InT, OutT, 8>(a, sh.tx, st);
    case 16:
      return run<InT, OutT, 16>(a, sh.tx, st);
    default:
      return cudaErrorInvalidConfiguration;
  }
}

template <class OutT>
cudaError_t by_in(int in_dtype, const fkl::CastArgs& a, const fkl_launch_shape& sh, cudaStream_t st) {
  switch (in_dtype) {
    case FKL_U8:
      return by_vec<uint8_t, OutT>(a, sh, st);
    case FKL_U16:
      return by_vec<uint16_t, OutT>(a, sh, st);
    case FKL_F32:
      return by_vec<float, OutT>(a, sh, st);
    case FKL_F64:
      return by_vec<double, OutT>(a, sh, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch(int in_dtype, int out_dtype, const fkl::CastArgs& a, const fkl_launch_shape& sh,
                     cudaStream_t st) {
  switch (out_dtype) {
    case FKL_F32:
      return by_in<float>(in_dtype, a, sh, st);
    case FKL_F64:
      return by_in<double>(in_dtype, a, sh, st);
    case FKL_F16:
      return by_in<fkl::f16_t>(in_dtype, a, sh, st);
    case FKL_BF16:
      return by_in<fkl::bf16_t>(in_dtype, a, sh, st);
    case FKL_E4M3:
      return by_in<fkl::e4m3_t>(in_dtype, a, sh, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int64_t cast_bytes(int dtype) {
  switch (dtype) {
    case FKL_F64:
      return 8;
    case FKL_F32:
      return 4;
    case FKL_F16:
    case FKL_BF16:
      return 2;
    default:
      return 1;
  }
}

fkl::CastArgs base_args(const Spec& s, void* out, int64_t len) {
  fkl::CastArgs a;
  std::memset(&a, 0, sizeof(a));
  a.out = out;
  a.len = len;
  a.mul = s.mul[0];
  a.sub = s.sub[0];
  a.div = s.div[0];
  a.scale_inv = s.out_dtype == FKL_E4M3 ? static_cast<float>(1.0 / s.fp8_scale) : 1.f;
  return a;
}

}  // namespace

cudaError_t launch_cast(const Spec& s, const fkl_launch_shape& sh, int n, const void* const* ins, void* out,
                        int64_t len, cudaStream_t st) {
  const int64_t esz = cast_bytes(s.out_dtype);
  for (int start = 0; start < n; start += fkl::kCastCap) {
    fkl::CastArgs a = base_args(s, static_cast<uint8_t*>(out) + start * len * esz, len);
    a.n = std::min(fkl::kCastCap, n - start);
    for (int i = 0; i < a.n; ++i) a.in[i] = ins[start + i];
    a.has_mul = s.has_mul;
    a.has_sub = s.has_sub;
    a.has_div = s.has_div;
    const cudaError_t e = dispatch(s.in_dtype, s.out_dtype, a, sh, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_unfused_cast(const Spec& s, int n, const void* const* ins, void* out, int64_t len, void* ws,
                                cudaStream_t st) {
  const fkl_launch_shape sh{8, 256, 1, 1};
  const int64_t esz = cast_bytes(s.out_dtype);
  // float32 / float64 outputs hold the intermediate in place; 16-bit and FP8
  // outputs keep a float32 intermediate in `ws` (one tensor, reused)
  const bool in_place = s.out_dtype == FKL_F32 || s.out_dtype == FKL_F64;
  const int ct = s.out_dtype == FKL_F64 ? FKL_F64 : FKL_F32;
  if (!in_place && !ws) return cudaErrorInvalidValue;
  for (int i = 0; i < n; ++i) {
    void* o = static_cast<uint8_t*>(out) + i * len * esz;
    void* mid = in_place ? o : ws;
    // Read -> Cast -> Write, then one in-place kernel per op
    fkl::CastArgs a = base_args(s, mid, len);
    a.n = 1;
    a.in[0] = ins[i];
    cudaError_t e = dispatch(s.in_dtype, ct, a, sh, st);
    const int32_t present[3] = {s.has_mul, s.has_sub, s.has_div};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      if (!present[k]) continue;
      fkl::CastArgs b = base_args(s, mid, len);
      b.n = 1;
      b.in[0] = mid;
      b.has_mul = k == 0;
      b.has_sub = k == 1;
      b.has_div = k == 2;
      e = dispatch(ct, ct, b, sh, st);
    }
    if (e == cudaSuccess && !in_place) {  // the write: float32 -> output type
      fkl::CastArgs w = base_args(s, o, len);
      w.n = 1;
      w.in[0] = mid;
      e = dispatch(FKL_F32, s.out_dtype, w, sh, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fkl_impl
