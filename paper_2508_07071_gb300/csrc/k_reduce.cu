// ReduceDPP instantiations: per-channel min, max, sum and the maximum
// absolute value of a float image chain's values, from one read.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "float_family.cuh"
#include "fkl/reduce.cuh"

namespace fkl_impl {

namespace {

// 16 pixels per thread, 8 x 32 threads (8 x 16 pixels: a 640-pixel row is
// five column tiles), the compiler's register choice: among the measured
// shapes on the 256-frame NV12 letterbox batch, 140 us (capping registers
// for three blocks per SM: 137 us, but 128-248 spilled bytes in other
// chains; 8 pixels per thread: 164 us; software-pipelined variants, with the
// next job's words in registers or in a shared-memory ring filled by
// cp.async: 168 us or more, the decode's arithmetic sets the time).
constexpr int kV = 16;
constexpr int kTX = 8;
constexpr int kTY = 32;
constexpr int kMinBlocks = 0;

// Resident blocks per SM of one reduce kernel on the current device (cached).
cudaError_t resident_blocks(const void* kernel, int& per_sm) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, kernel);
  auto it = cache.find(key);
  if (it != cache.end()) {
    per_sm = it->second;
    return cudaSuccess;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTX * kTY, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cache.emplace(key, per_sm);
  return cudaSuccess;
}

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
  const int64_t cols = (int64_t(c.W) + kV - 1) / kV;
  a.col_tiles = static_cast<int32_t>((cols + kTX - 1) / kTX);
  a.row_tiles = (c.H + kTY - 1) / kTY;
  const int64_t jobs = int64_t(a.col_tiles) * a.row_tiles * c.n;
  if (jobs == 0) return cudaSuccess;
  if (jobs > (int64_t(1) << 30)) return cudaErrorInvalidConfiguration;  // job indices stay in int
  auto kernel = fkl::reduce2d_kernel<kV, kMinBlocks, RB, Cops>;
  int per_sm = 0;
  const cudaError_t e = resident_blocks(reinterpret_cast<const void*>(kernel), per_sm);
  if (e != cudaSuccess) return e;
  // a persistent grid: every block resident at once, each walking its share
  // of the jobs, so the accumulator takes one atomic per block and statistic
  const int grid = static_cast<int>(std::min<int64_t>(jobs, int64_t(sm_count()) * per_sm));
  kernel<<<grid, dim3(kTX, kTY, 1), 0, c.stream>>>(a);
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
  // the largest magnitude is that of a channel's minimum or maximum
  float amax = 0.f;
  if (count > 0)
    for (int c = 0; c < 3; ++c) amax = fmaxf(amax, fmaxf(fabsf(stats[c]), fabsf(stats[3 + c])));
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
