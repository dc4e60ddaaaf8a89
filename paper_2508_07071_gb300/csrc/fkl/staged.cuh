// Row-staged TransformDPP for the exact-2x NV12 read (a DPP of paper §IV-C
// built on Blackwell's bulk-copy engine): persistent CTAs walk jobs of R
// output rows; one thread copies each job's source rows (two luma rows and
// one chroma row per output row) from global to shared memory with 1-D
// `cp.async.bulk` copies that complete on an mbarrier (expect-tx), S jobs
// ahead; the CTA computes from shared memory while the next jobs' rows are in
// flight. The arithmetic is ResizeNV12::compute2x, the same as the
// register-load path, so both give the same bits.
//
// Every wait is bounded by the global timer: a wait that runs out (after
// `wait_ns`, 1 s unless the host set another limit) records a timeout in a
// device flag (read by the host through the C ABI), lets the CTA's copies in
// flight land (a separate, fixed 1 s bound) and leaves the kernel.
#pragma once

#include "ops.cuh"

namespace fkl {

FKL_D uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

FKL_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
FKL_D void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
FKL_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
FKL_D bool mbar_test_wait(uint64_t* bar, uint32_t parity) {  // non-blocking poll
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared; 16-byte aligned addresses, size a multiple of 16.
FKL_D void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
FKL_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
FKL_D unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Limit of the wait that lets a CTA's copies in flight land before it leaves
// after a timeout; fixed, whatever the consumer-wait limit is.
constexpr unsigned long long kStagedDrainNs = 1000ull * 1000 * 1000;  // 1 s
constexpr int kMaxStages = 8;

template <class RB, class W, class Cops>
struct StagedArgs {
  typename RB::ParamsType rp;
  typename W::ParamsType wp;
  Cops cops;
  int32_t H, W_;
  int32_t R;               // output rows per job
  int32_t stages;          // shared-memory ring depth, 2..kMaxStages
  int32_t row_bytes;       // bytes of one staged source row (2 W_)
  int32_t jobs_per_image;  // ceil(H / R)
  int32_t jobs;            // images x jobs_per_image
  int* error;              // device flag, set to 1 when a wait gives up
  unsigned long long wait_ns;  // limit of one consumer wait on a stage
};

// Bounded wait on `bar` for `parity`; false when it gave up after limit_ns.
// try_wait may itself suspend the thread for a while, so the phase is first
// polled without blocking; a limit below the global timer's 1 us resolution
// allows that one poll only.
FKL_D bool staged_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit_ns < 1000) return false;
  const unsigned long long t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (now_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Source rows of output row y of an image, false for a band row.
template <class P>
FKL_D bool staged_rows(const P& p, int y, const uint8_t*& y0, const uint8_t*& y1, const uint8_t*& uv) {
  const int ly = y - p.oy;
  if (ly < 0 || ly >= p.dh) return false;
  const int64_t sy = p.ry + 2 * ly;
  y0 = p.src + sy * p.pitch + p.rx;
  y1 = y0 + p.pitch;
  uv = p.uv + (sy >> 1) * p.pitch + p.rx;
  return true;
}

// Preconditions (checked on the host): every image is an exact 2x downscale
// with 16-byte aligned rows (kFast2x), fills the output width (ox == 0,
// dw == W_), W_ % V == 0 and 2 W_ % 16 == 0; dynamic shared memory holds
// stages x 3 R x row_bytes bytes.
template <int V, class RB, class W, class Cops>
__global__ void __launch_bounds__(256) staged_nv12x2_kernel(const __grid_constant__ StagedArgs<RB, W, Cops> a) {
  extern __shared__ __align__(128) uint8_t stage[];
  __shared__ __align__(8) uint64_t bars[kMaxStages];
  const int rb = a.row_bytes, R = a.R, S = a.stages;
  const int stage_bytes = 3 * R * rb;
  const int groups = a.W_ / V;

  // Thread 0: the copies of one job into stage s, all completing on bars[s].
  auto issue = [&](int job, int s) {
    const int z = job / a.jobs_per_image;
    const int row0 = (job - z * a.jobs_per_image) * R;
    const auto& p = a.rp.p[z];
    const uint8_t *y0, *y1, *uv;
    uint32_t bytes = 0;
    for (int r = 0; r < R; ++r)
      if (row0 + r < a.H && staged_rows(p, row0 + r, y0, y1, uv)) bytes += 3 * rb;
    mbar_arrive_expect_tx(&bars[s], bytes);
    uint8_t* base = stage + s * stage_bytes;
    for (int r = 0; r < R; ++r) {
      if (row0 + r < a.H && staged_rows(p, row0 + r, y0, y1, uv)) {
        bulk_load(base + (3 * r) * rb, y0, rb, &bars[s]);
        bulk_load(base + (3 * r + 1) * rb, y1, rb, &bars[s]);
        bulk_load(base + (3 * r + 2) * rb, uv, rb, &bars[s]);
      }
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < S; ++i) {  // prologue: this CTA's first S jobs
      const int job = blockIdx.x + i * gridDim.x;
      if (job < a.jobs) issue(job, i);
    }
  }
  __syncthreads();

  int i = 0;
  bool ok = true;
  for (int job = blockIdx.x; job < a.jobs; job += gridDim.x, ++i) {
    const int s = i % S;
    // every thread waits (the acquire of the copied bytes); the CTA leaves
    // together if any of them gave up
    if (!__syncthreads_and(staged_wait(&bars[s], (i / S) & 1, a.wait_ns))) {
      ok = false;
      break;
    }
    const int z = job / a.jobs_per_image;
    const int row0 = (job - z * a.jobs_per_image) * R;
    const auto& p = a.rp.p[z];
    const uint8_t* base = stage + s * stage_bytes;
    for (int it = threadIdx.x; it < R * groups; it += blockDim.x) {
      const int r = it / groups;
      const int y = row0 + r;
      if (y >= a.H) break;  // later items have larger r
      const int x0 = (it - r * groups) * V;
      F3 in[V];
      const int ly = y - p.oy;
      if (ly < 0 || ly >= p.dh) {
#pragma unroll
        for (int k = 0; k < V; ++k) in[k] = F3{{p.pad, p.pad, p.pad}};
      } else {
        constexpr int Wd = V / 8;
        uint4 wa[Wd], wb[Wd], wc[Wd];
        const uint4* r0 = reinterpret_cast<const uint4*>(base + (3 * r) * rb + 2 * x0);
        const uint4* r1 = reinterpret_cast<const uint4*>(base + (3 * r + 1) * rb + 2 * x0);
        const uint4* rc = reinterpret_cast<const uint4*>(base + (3 * r + 2) * rb + 2 * x0);
#pragma unroll
        for (int k = 0; k < Wd; ++k) {
          wa[k] = r0[k];
          wb[k] = r1[k];
          wc[k] = rc[k];
        }
        ResizeNV12::compute2x<V>(wa, wb, wc, in);
      }
      F3 out[V];
      if constexpr (ChainHasPair<Cops>::value) {
#pragma unroll
        for (int k = 0; k < V; k += 2)
          unpack_pair(apply_chain_pair(pack_pair(in[k], in[k + 1]), a.cops), out[k], out[k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = apply_chain(in[k], a.cops);
      }
      W::template exec_span<V>(Point{x0, y, z}, V, out, a.wp);
    }
    __syncthreads();  // every thread is done reading stage s
    if (threadIdx.x == 0) {
      const int next = job + S * gridDim.x;
      if (next < a.jobs) {
        fence_proxy_async();  // order the generic reads of stage s before the async writes
        issue(next, s);
      }
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(a.error, 1);
    // let the copies still in flight land before the CTA's shared memory is released
    for (int k = 0; k < S; ++k) {
      const int ii = i + k;
      if (blockIdx.x + ii * gridDim.x < a.jobs) staged_wait(&bars[ii % S], (ii / S) & 1, kStagedDrainNs);
    }
  }
}

}  // namespace fkl
