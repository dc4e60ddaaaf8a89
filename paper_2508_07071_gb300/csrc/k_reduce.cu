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

// 8 window pixels per thread, 16 x 16 threads (a 640-pixel window row is five
// column tiles of 128 pixels, a job 16 rows), registers capped for four
// resident 256-thread blocks per SM (32 warps): the fold of each pixel pair
// needs no array of pixels, so the cap costs no spills.
constexpr int kV = 8;
constexpr int kTX = 16;
constexpr int kTY = 16;
constexpr int kMinBlocks = 4;

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

template <class ROp>
cudaError_t run_reduce(const LaunchCtx& c, fkl::ReduceAcc* acc, ReduceLaunch& info) {
  using RB = fkl::BatchRead<ROp, kBatchCap>;
  fkl::ReduceArgs<RB> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.acc = acc;
  int64_t max_w = 0, max_h = 0;
  for (int i = 0; i < c.n; ++i) {
    max_w = std::max<int64_t>(max_w, c.imgs[i].dw);
    max_h = std::max<int64_t>(max_h, c.imgs[i].dh);
  }
  const int64_t cols = (max_w + kV - 1) / kV;
  a.col_tiles = static_cast<int32_t>((cols + kTX - 1) / kTX);
  a.row_tiles = static_cast<int32_t>((max_h + kTY - 1) / kTY);
  const int64_t jobs = int64_t(a.col_tiles) * a.row_tiles * c.n;
  if (jobs == 0) return cudaSuccess;
  if (jobs > (int64_t(1) << 30)) return cudaErrorInvalidConfiguration;  // job indices stay in int
  auto kernel = fkl::reduce2d_kernel<kV, kMinBlocks, RB>;
  int per_sm = 0;
  const cudaError_t e = resident_blocks(reinterpret_cast<const void*>(kernel), per_sm);
  if (e != cudaSuccess) return e;
  // a persistent grid: every block resident at once, each walking its share
  // of the jobs, so the accumulator takes one atomic per block and statistic
  const int grid = static_cast<int>(std::min<int64_t>(jobs, int64_t(sm_count()) * per_sm));
  kernel<<<grid, dim3(kTX, kTY, 1), 0, c.stream>>>(a);
  info.jobs += jobs;
  info.grid = std::max(info.grid, grid);
  return cudaGetLastError();
}

struct FinalizeArgs {
  const fkl::ReduceAcc* acc;
  float* stats;
  double count;       // output pixels per channel
  double fill_count;  // of them, fill pixels (the pad value)
  fkl::ReduceChain chain;
  int32_t jobs, grid;
};

__global__ void finalize_kernel(const FinalizeArgs f) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float* stats = f.stats;
  const fkl::ReduceChain& ch = f.chain;
  float amax = 0.f;
  for (int c = 0; c < 3; ++c) {
    const int rc = ch.swap ? 2 - c : c;  // the read channel output channel c comes from
    float lo = fkl::key_value(f.acc->min_key[rc]);
    float hi = fkl::key_value(f.acc->max_key[rc]);
    if (f.fill_count > 0) {
      lo = fminf(lo, ch.pad);
      hi = fmaxf(hi, ch.pad);
    }
    const float a = fkl::apply_reduce_chain(ch, c, lo), b = fkl::apply_reduce_chain(ch, c, hi);
    stats[c] = f.count > 0 ? fminf(a, b) : __int_as_float(0x7fc00000);
    stats[3 + c] = f.count > 0 ? fmaxf(a, b) : __int_as_float(0x7fc00000);
    // the mean: the chain's affine map of the read values' mean, in float64
    const double sum = static_cast<double>(static_cast<long long>(f.acc->sum_fx[rc])) / fkl::kSumScale +
                       f.fill_count * static_cast<double>(ch.pad);
    double m = f.count > 0 ? sum / f.count : 0.0;
    m = (m * ch.mul[c] - ch.sub[c]) / (ch.has_div ? static_cast<double>(ch.div[c]) : 1.0);
    stats[6 + c] = f.count > 0 ? static_cast<float>(m) : 0.f;
    // the largest magnitude is that of a channel's minimum or maximum
    if (f.count > 0) amax = fmaxf(amax, fmaxf(fabsf(stats[c]), fabsf(stats[3 + c])));
  }
  stats[9] = amax;
  const float s = amax > 0.f ? __fdiv_rn(amax, 448.f) : 1.f;  // E4M3 per-tensor scale
  stats[10] = s;
  stats[11] = __fdiv_rn(1.f, s);
  reinterpret_cast<int32_t*>(stats)[12] = f.jobs;
  reinterpret_cast<int32_t*>(stats)[13] = f.grid;
}

}  // namespace

cudaError_t launch_reduce(const LaunchCtx& c, fkl::ReduceAcc* acc, ReduceLaunch& info) {
  const Spec& s = *c.spec;
  if (s.family == FAM_PACKED) return run_reduce<fkl::ResizeU8C3>(c, acc, info);
  if (s.family == FAM_NV12)
    return c.all_exact2x ? run_reduce<fkl::ResizeNV12x2>(c, acc, info) : run_reduce<fkl::ResizeNV12>(c, acc, info);
  return cudaErrorInvalidValue;
}

cudaError_t finalize_reduce(const Spec& s, const fkl::ReduceAcc* acc, double count, double fill_count,
                            const ReduceLaunch& info, float* stats, cudaStream_t st) {
  FinalizeArgs f;
  std::memset(&f, 0, sizeof(f));
  f.acc = acc;
  f.stats = stats;
  f.count = count;
  f.fill_count = fill_count;
  f.chain.swap = s.swap ? 1 : 0;
  f.chain.has_div = s.has_div ? 1 : 0;
  std::memcpy(f.chain.mul, s.mul, sizeof(f.chain.mul));
  std::memcpy(f.chain.sub, s.sub, sizeof(f.chain.sub));
  std::memcpy(f.chain.div, s.div, sizeof(f.chain.div));
  f.chain.pad = s.pad;
  f.jobs = static_cast<int32_t>(std::min<int64_t>(info.jobs, INT32_MAX));
  f.grid = info.grid;
  finalize_kernel<<<1, 32, 0, st>>>(f);
  return cudaGetLastError();
}

}  // namespace fkl_impl
