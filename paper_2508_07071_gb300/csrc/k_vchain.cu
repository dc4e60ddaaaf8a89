// The vertical Mul/Add chain over a linear float32 tensor (paper §VI-B,
// §VI-D, §VI-G): all ops of a chunk of up to kVChainCap ops run in one
// kernel, every intermediate in registers.
#include <algorithm>
#include <cstring>

#include "fkl/vchain.cuh"
#include "registry.h"

namespace fkl_impl {

namespace {

constexpr int kDefaultE = 16;  // elements per thread
constexpr int kDefaultBlock = 256;

template <int E, int CAP>
cudaError_t run_chunk(const Spec& s, size_t start, int len, const void* in, bool in_u8, float* out, int64_t n,
                      int block, bool persistent, cudaStream_t st) {
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
  const int64_t per_block = static_cast<int64_t>(block) * E;
  const int64_t need = std::max<int64_t>(1, (n + per_block - 1) / per_block);
  const int64_t cap = persistent ? int64_t(sm_count()) * std::max(1, 2048 / block) : need;
  const int blocks = static_cast<int>(std::min<int64_t>(need, std::min<int64_t>(cap, 0x7fffffff)));
  if (in_u8) {
    if (alt)
      fkl::vchain_kernel<E, CAP, true, uint8_t><<<blocks, block, 0, st>>>(p);
    else
      fkl::vchain_kernel<E, CAP, false, uint8_t><<<blocks, block, 0, st>>>(p);
  } else {
    if (alt)
      fkl::vchain_kernel<E, CAP, true><<<blocks, block, 0, st>>>(p);
    else
      fkl::vchain_kernel<E, CAP, false><<<blocks, block, 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <int CAP>
cudaError_t run_shape(const Spec& s, const fkl_launch_shape& sh, size_t start, int len, const void* in, bool in_u8,
                      float* out, int64_t n, cudaStream_t st) {
  const bool persistent = sh.ry != 0;
  switch (sh.vec) {
    case 2:
      return run_chunk<2, CAP>(s, start, len, in, in_u8, out, n, sh.tx, persistent, st);
    case 4:
      return run_chunk<4, CAP>(s, start, len, in, in_u8, out, n, sh.tx, persistent, st);
    case 8:
      return run_chunk<8, CAP>(s, start, len, in, in_u8, out, n, sh.tx, persistent, st);
    case 16:
      return run_chunk<16, CAP>(s, start, len, in, in_u8, out, n, sh.tx, persistent, st);
    case 32:
      return run_chunk<32, CAP>(s, start, len, in, in_u8, out, n, sh.tx, persistent, st);
    default:
      return cudaErrorInvalidConfiguration;
  }
}

}  // namespace

cudaError_t launch_vchain(const Spec& s, const fkl_launch_shape& sh, const void* in, float* out, int64_t n,
                          cudaStream_t st) {
  const size_t L = s.vkinds.size();
  if (L == 0) return run_shape<8>(s, sh, 0, 0, in, s.vinput_u8, out, n, st);
  for (size_t start = 0; start < L; start += kVChainCap) {
    const int len = static_cast<int>(std::min<size_t>(kVChainCap, L - start));
    const void* src = start == 0 ? in : out;
    const bool u8 = start == 0 && s.vinput_u8;
    const cudaError_t e = len <= 128 ? run_shape<128>(s, sh, start, len, src, u8, out, n, st)
                                     : run_shape<kVChainCap>(s, sh, start, len, src, u8, out, n, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Unfused form: one kernel per op over the whole tensor.
cudaError_t launch_unfused_vchain(const Spec& s, const void* in, float* out, int64_t n, cudaStream_t st) {
  const size_t L = s.vkinds.size();
  if (L == 0) return run_chunk<kDefaultE, 8>(s, 0, 0, in, s.vinput_u8, out, n, kDefaultBlock, true, st);
  for (size_t i = 0; i < L; ++i) {
    const cudaError_t e = run_chunk<kDefaultE, 8>(s, i, 1, i == 0 ? in : out, i == 0 && s.vinput_u8, out, n,
                                                  kDefaultBlock, true, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fkl_impl
