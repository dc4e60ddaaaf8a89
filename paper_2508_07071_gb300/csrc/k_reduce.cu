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
auto reduce_kernel() {
  return fkl::reduce2d_kernel<kV, kMinBlocks, fkl::BatchRead<ROp, kBatchCap>>;
}

template <class ROp>
cudaError_t plan_t(const LaunchCtx& c, ReducePlan& pl) {
  pl = ReducePlan{};
  int64_t max_w = 0, max_h = 0;
  for (int i = 0; i < c.n; ++i) {
    max_w = std::max<int64_t>(max_w, c.imgs[i].dw);
    max_h = std::max<int64_t>(max_h, c.imgs[i].dh);
  }
  const int64_t cols = (max_w + kV - 1) / kV;
  pl.col_tiles = static_cast<int32_t>((cols + kTX - 1) / kTX);
  pl.row_tiles = static_cast<int32_t>((max_h + kTY - 1) / kTY);
  pl.jobs = int64_t(pl.col_tiles) * pl.row_tiles * c.n;
  if (pl.jobs == 0) return cudaSuccess;
  if (pl.jobs > (int64_t(1) << 30)) return cudaErrorInvalidConfiguration;  // job indices stay in int
  int per_sm = 0;
  const cudaError_t e = resident_blocks(reinterpret_cast<const void*>(reduce_kernel<ROp>()), per_sm);
  if (e != cudaSuccess) return e;
  // a persistent grid: every block resident at once, each walking its share
  // of the jobs, so the accumulator takes one atomic per block and statistic
  pl.grid = static_cast<int>(std::min<int64_t>(pl.jobs, int64_t(sm_count()) * per_sm));
  return cudaSuccess;
}

template <class ROp>
cudaError_t run_t(const LaunchCtx& c, const ReducePlan& pl, fkl::ReduceAcc* acc, const fkl::ReduceFinal& fin) {
  if (pl.grid == 0) return cudaSuccess;
  using RB = fkl::BatchRead<ROp, kBatchCap>;
  fkl::ReduceArgs<RB> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = c.n;
  std::memcpy(a.rp.p, c.imgs, sizeof(fkl::ResampleParams) * c.n);
  a.col_tiles = pl.col_tiles;
  a.row_tiles = pl.row_tiles;
  a.acc = acc;
  a.fin = fin;
  reduce_kernel<ROp>()<<<pl.grid, dim3(kTX, kTY, 1), 0, c.stream>>>(a);
  return cudaGetLastError();
}

// A call with no reduction launch (no window pixels) still writes its statistics.
__global__ void finish_kernel(const fkl::ReduceAcc* acc, const fkl::ReduceFinal fin) {
  if (threadIdx.x == 0 && blockIdx.x == 0) fkl::reduce_finish(acc, fin);
}

}  // namespace

cudaError_t plan_reduce(const LaunchCtx& c, ReducePlan& pl) {
  const Spec& s = *c.spec;
  if (s.family == FAM_PACKED) return plan_t<fkl::ResizeU8C3>(c, pl);
  if (s.family == FAM_NV12)
    return c.all_exact2x ? plan_t<fkl::ResizeNV12x2>(c, pl) : plan_t<fkl::ResizeNV12>(c, pl);
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce(const LaunchCtx& c, const ReducePlan& pl, fkl::ReduceAcc* acc,
                          const fkl::ReduceFinal& fin) {
  const Spec& s = *c.spec;
  if (s.family == FAM_PACKED) return run_t<fkl::ResizeU8C3>(c, pl, acc, fin);
  if (s.family == FAM_NV12)
    return c.all_exact2x ? run_t<fkl::ResizeNV12x2>(c, pl, acc, fin) : run_t<fkl::ResizeNV12>(c, pl, acc, fin);
  return cudaErrorInvalidValue;
}

fkl::ReduceFinal reduce_final(const Spec& s, float* stats, double count, double fill_count, int64_t jobs, int grid,
                              int64_t blocks) {
  fkl::ReduceFinal f;
  std::memset(&f, 0, sizeof(f));
  f.stats = stats;
  f.count = count;
  f.fill_count = fill_count;
  f.chain.swap = s.swap ? 1 : 0;
  f.chain.has_div = s.has_div ? 1 : 0;
  std::memcpy(f.chain.mul, s.mul, sizeof(f.chain.mul));
  std::memcpy(f.chain.sub, s.sub, sizeof(f.chain.sub));
  std::memcpy(f.chain.div, s.div, sizeof(f.chain.div));
  f.chain.pad = s.pad;
  f.jobs = static_cast<int32_t>(std::min<int64_t>(jobs, INT32_MAX));
  f.grid = grid;
  f.blocks = static_cast<uint32_t>(blocks);
  return f;
}

cudaError_t finish_reduce(const fkl::ReduceAcc* acc, const fkl::ReduceFinal& fin, cudaStream_t st) {
  finish_kernel<<<1, 32, 0, st>>>(acc, fin);
  return cudaGetLastError();
}

}  // namespace fkl_impl
