// The vertical Mul/Add chain over a linear float32 tensor (paper §VI-B,
// §VI-D, §VI-G): all ops of a chunk of up to kVChainCap ops run in one
// kernel, every intermediate in registers.
#include <algorithm>
#include <cstring>

#include "registry.h"

namespace fkl_impl {

namespace {

constexpr int kU = 4;  // float4 vectors per thread
constexpr int kBlock = 256;

template <int CAP>
cudaError_t run_chunk(const Spec& s, size_t start, int len, const float* in, float* out,
                      int64_t n, cudaStream_t st) {
  fkl::VChainParams<CAP> p;
  std::memset(&p, 0, sizeof(p));
  p.in = in;
  p.out = out;
  p.n = n;
  p.len = len;
  bool alt = true;
  for (int i = 0; i < len; ++i) {
    const int kind = s.vkinds[start + i];
    p.c[i] = s.vconsts[start + i];
    if (kind == 1) p.add_mask[i >> 5] |= 1u << (i & 31);
    if (kind != (i & 1)) alt = false;
  }
  p.alternating = alt ? 1 : 0;
  const int64_t per_block = static_cast<int64_t>(kBlock) * 4 * kU;
  const int64_t need = (n + per_block - 1) / per_block;
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(sm_count()) * 8)));
  if (alt)
    fkl::vchain_kernel<kU, CAP, true><<<blocks, kBlock, 0, st>>>(p);
  else
    fkl::vchain_kernel<kU, CAP, false><<<blocks, kBlock, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_vchain(const Spec& s, const float* in, float* out, int64_t n, cudaStream_t st) {
  const size_t L = s.vkinds.size();
  if (L == 0) return run_chunk<8>(s, 0, 0, in, out, n, st);
  for (size_t start = 0; start < L; start += kVChainCap) {
    const int len = static_cast<int>(std::min<size_t>(kVChainCap, L - start));
    const float* src = start == 0 ? in : out;
    const cudaError_t e = len <= 128 ? run_chunk<128>(s, start, len, src, out, n, st)
                                     : run_chunk<kVChainCap>(s, start, len, src, out, n, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Unfused form: one kernel per op over the whole tensor.
cudaError_t launch_unfused_vchain(const Spec& s, const float* in, float* out, int64_t n,
                                  cudaStream_t st) {
  const size_t L = s.vkinds.size();
  if (L == 0) return run_chunk<8>(s, 0, 0, in, out, n, st);
  for (size_t i = 0; i < L; ++i) {
    const cudaError_t e = run_chunk<8>(s, i, 1, i == 0 ? in : out, out, n, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fkl_impl
