// Typed chains over batches of linear tensors (paper §VI-I): the fused form
// (one launch per 256 tensors) and the unfused form (one kernel per op and
// tensor, each a full read and write of the tensor).
#include <algorithm>
#include <cstring>

#include "fkl/cast.cuh"
#include "registry.h"

namespace fkl_impl {

namespace {

template <class InT, class CT, int E>
cudaError_t run(const fkl::CastArgs& a, int block, cudaStream_t st) {
  const int64_t per_block = static_cast<int64_t>(block) * E;
  const int64_t gx = (a.len + per_block - 1) / per_block;
  if (gx == 0 || a.n == 0) return cudaSuccess;
  if (gx > 0x7fffffff) return cudaErrorInvalidConfiguration;
  fkl::cast_chain_kernel<InT, CT, E><<<dim3(static_cast<unsigned>(gx), a.n, 1), block, 0, st>>>(a);
  return cudaGetLastError();
}

template <class InT, class CT>
cudaError_t by_vec(const fkl::CastArgs& a, const fkl_launch_shape& sh, cudaStream_t st) {
  switch (sh.vec) {
    case 8:
      return run<InT, CT, 8>(a, sh.tx, st);
    case 16:
      return run<InT, CT, 16>(a, sh.tx, st);
    default:
      return cudaErrorInvalidConfiguration;
  }
}

template <class CT>
cudaError_t by_in(int in_dtype, const fkl::CastArgs& a, const fkl_launch_shape& sh, cudaStream_t st) {
  switch (in_dtype) {
    case FKL_U8:
      return by_vec<uint8_t, CT>(a, sh, st);
    case FKL_U16:
      return by_vec<uint16_t, CT>(a, sh, st);
    case FKL_F32:
      return by_vec<float, CT>(a, sh, st);
    case FKL_F64:
      return by_vec<double, CT>(a, sh, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch(int in_dtype, int out_dtype, const fkl::CastArgs& a, const fkl_launch_shape& sh,
                     cudaStream_t st) {
  if (out_dtype == FKL_F32) return by_in<float>(in_dtype, a, sh, st);
  if (out_dtype == FKL_F64) return by_in<double>(in_dtype, a, sh, st);
  return cudaErrorInvalidValue;
}

fkl::CastArgs base_args(const Spec& s, void* out, int64_t len) {
  fkl::CastArgs a;
  std::memset(&a, 0, sizeof(a));
  a.out = out;
  a.len = len;
  a.mul = s.mul[0];
  a.sub = s.sub[0];
  a.div = s.div[0];
  return a;
}

}  // namespace

cudaError_t launch_cast(const Spec& s, const fkl_launch_shape& sh, int n, const void* const* ins, void* out,
                        int64_t len, cudaStream_t st) {
  const int64_t esz = s.out_dtype == FKL_F64 ? 8 : 4;
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

cudaError_t launch_unfused_cast(const Spec& s, int n, const void* const* ins, void* out, int64_t len,
                                cudaStream_t st) {
  const fkl_launch_shape sh{8, 256, 1, 1};
  const int64_t esz = s.out_dtype == FKL_F64 ? 8 : 4;
  for (int i = 0; i < n; ++i) {
    void* o = static_cast<uint8_t*>(out) + i * len * esz;
    // Read -> Cast -> Write, then one in-place kernel per op
    fkl::CastArgs a = base_args(s, o, len);
    a.n = 1;
    a.in[0] = ins[i];
    cudaError_t e = dispatch(s.in_dtype, s.out_dtype, a, sh, st);
    const int32_t present[3] = {s.has_mul, s.has_sub, s.has_div};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      if (!present[k]) continue;
      fkl::CastArgs b = base_args(s, o, len);
      b.n = 1;
      b.in[0] = o;
      b.has_mul = k == 0;
      b.has_sub = k == 1;
      b.has_div = k == 2;
      e = dispatch(s.out_dtype, s.out_dtype, b, sh, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fkl_impl
