// ReduceDPP instantiations: per-channel min, max, sum and the maximum
// absolute value of a float image chain's values, from one read.
#include <cstring>

#include "float_family.cuh"
#include "fkl/reduce.cuh"

namespace fkl_impl {

namespace {

constexpr int kV = 8;
constexpr int kTX = 32;
constexpr int kTY = 8;

template <class ROp, bool kSwap, int kTail>
cudaError_t run_reduce(const LaunchCtx& c, fkl::ReduceAcc* acc) {
  using RB = fkl::BatchRead<ROp, kBatchCap>;
  auto tail = make_tail<kTail>(*c.spec);
  auto cops = [&] {
    if constexpr (kSwap) {
      return fkl::prepend(fkl::IOp<fkl::SwapRB<fkl::F3>>{}, tail);
    } else {
      return tail;
    }
  }();
  using Cops = decltype(cops);
  fkl::ReduceArgs<RB, Cops> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.cops = cops;
  a.H = c.H;
  a.W_ = c.W;
  a.acc = acc;
  const int cols = (c.W + kV - 1) / kV;
  const dim3 grid((cols + kTX - 1) / kTX, (c.H + kTY - 1) / kTY, c.n);
  fkl::reduce2d_kernel<kV, RB, Cops><<<grid, dim3(kTX, kTY, 1), 0, c.stream>>>(a);
  return cudaGetLastError();
}

template <class ROp, bool kSwap>
cudaError_t by_tail(const LaunchCtx& c, fkl::ReduceAcc* acc) {
  switch (tail_of(*c.spec)) {
    case 0:
      return run_reduce<ROp, kSwap, 0>(c, acc);
    case 1:
      return run_reduce<ROp, kSwap, 1>(c, acc);
    default:
      return run_reduce<ROp, kSwap, 2>(c, acc);
  }
}

template <class ROp>
cudaError_t by_swap(const LaunchCtx& c, fkl::ReduceAcc* acc) {
  return c.spec->swap ? by_tail<ROp, true>(c, acc) : by_tail<ROp, false>(c, acc);
}

__global__ void finalize_kernel(const fkl::ReduceAcc* acc, double count, float* stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int c = 0; c < 3; ++c) {
    stats[c] = fkl::key_value(acc->min_key[c]);
    stats[3 + c] = fkl::key_value(acc->max_key[c]);
    const double sum = static_cast<double>(static_cast<long long>(acc->sum_fx[c])) / fkl::kSumScale;
    stats[6 + c] = static_cast<float>(count > 0 ? sum / count : 0.0);
  }
  const float amax = fkl::key_value(acc->absmax_key);
  stats[9] = amax;
  const float s = amax > 0.f ? __fdiv_rn(amax, 448.f) : 1.f;  // E4M3 per-tensor scale
  stats[10] = s;
  stats[11] = __fdiv_rn(1.f, s);
}

}  // namespace

cudaError_t launch_reduce(const LaunchCtx& c, fkl::ReduceAcc* acc) {
  const Spec& s = *c.spec;
  if (s.family == FAM_PACKED) return by_swap<fkl::ResizeU8C3>(c, acc);
  if (s.family == FAM_NV12)
    return c.all_exact2x ? by_swap<fkl::ResizeNV12x2>(c, acc) : by_swap<fkl::ResizeNV12>(c, acc);
  return cudaErrorInvalidValue;
}

cudaError_t finalize_reduce(const fkl::ReduceAcc* acc, double count, float* stats, cudaStream_t st) {
  finalize_kernel<<<1, 32, 0, st>>>(acc, count, stats);
  return cudaGetLastError();
}

}  // namespace fkl_impl
