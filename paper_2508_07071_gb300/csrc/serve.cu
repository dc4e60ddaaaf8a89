// Serving runtime (include/fkl.h, fkl_server_*): continuous batching of
// preprocessing requests with admission by free device memory.
//
// Persistent mode: a persistent kernel whose CTAs claim tasks from a ring in
// mapped host memory (tail written by the host with release order, head
// claimed on the device with compare-and-swap). A task is a band of 16
// output rows of one image: the CTA first gathers the source rows that band's
// bilinear taps reference straight from the request's pinned host image into
// device memory (16-byte loads over the host link; for a downscale by more
// than 2 only the two tap rows of each output row, at most 2 x 224 rows of a
// 224-row output, instead of the whole image), then runs the chain's Ops on
// the band. Each request slot has a device counter of finished tasks that only
// grows; the CTA that brings it to the request's target publishes the
// request's sequence number to the host. Every device wait is bounded by an
// idle timeout on the global timer and by a stop flag.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda/atomic>

#include "registry.h"

namespace fkl_impl {
namespace serve {

constexpr int kQueue = 8192;    // task ring entries
constexpr int kMaxSlots = 1024;  // request slots
constexpr int kV = 8;            // output pixels per thread and item
constexpr int kThreads = 256;
constexpr int kBand = 16;        // output rows per task
constexpr int kMaxStaged = 2 * kBand + 2;  // staged source rows of one band (bound)
constexpr int32_t kRowPairs = 1 << 4;      // flags: staged rows 2 ly, 2 ly + 1 are output row ly's taps

// One band of one image of one request. rp describes the staged copy of the
// image's crop window in device memory: rp.src its first staged row, rp.pitch
// the staged row pitch, rp.uv (as int32) the staged rows' byte offsets (a
// row's first byte sits `offset` bytes into it, the host row's address mod
// 16), rp.flags & kRowPairs the staging mode; the rest is the placement of
// image_params (rx = ry = 0: the window starts the staged rows).
struct Task {
  fkl::ResampleParams rp;
  const uint8_t* host;  // device address of the host image's window origin
  int64_t host_pitch;   // bytes between host rows
  uint8_t* out;         // this image's first output plane
  int64_t plane;        // bytes between output planes
  uint64_t seq;         // request sequence number (its completion value)
  uint64_t target;      // slot counter value once every task of the request is done
  int32_t slot;         // request slot
  int32_t band;         // first output row = band * kBand
  int32_t _pad[2];
};
static_assert(sizeof(Task) == 128, "task ring entry");

struct HostCtl {  // mapped pinned memory
  unsigned long long tail;  // tasks published (host writes, release)
  int stop;                 // host asks the kernel to finish
  int active;               // CTAs running (device decrements on exit)
  int _pad[12];
  unsigned long long done[kMaxSlots];  // completion: request seq per slot
  Task tasks[kQueue];
};

struct DevCtl {  // device memory
  unsigned long long head;               // tasks claimed
  unsigned long long finished[kMaxSlots];  // tasks finished per slot, all requests (never reset)
};

struct KArgs {
  HostCtl* hc;  // device view of the mapped block
  DevCtl* dc;
  int H, W;
  int64_t pitch;
  float scale_inv;
  int aligned;
  fkl::C3Params mul, sub;
  fkl::Div3Params div;
  unsigned long long idle_ns;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: claim the next task; its ring position in *slot_out. 1 =
// claimed, 0 = stop or idle. (The CTA then copies the task, see copy_task.)
__device__ int claim(const KArgs& a, unsigned long long* slot_out) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> head(a.dc->head);
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(a.hc->tail);
  cuda::atomic_ref<int, cuda::thread_scope_system> stop(a.hc->stop);
  const unsigned long long t0 = globaltimer_ns();
  unsigned ns = 1024;
  for (;;) {
    if (stop.load(cuda::memory_order_relaxed)) return 0;
    unsigned long long h = head.load(cuda::memory_order_relaxed);
    const unsigned long long t = tail.load(cuda::memory_order_acquire);
    if (h < t) {
      if (head.compare_exchange_strong(h, h + 1, cuda::memory_order_acq_rel)) {
        *slot_out = h;
        return 1;
      }
      continue;
    }
    if (globaltimer_ns() - t0 > a.idle_ns) return 0;
    __nanosleep(ns);
    ns = min(ns * 2, 65536u);
  }
}

// The CTA's first 16 threads copy a claimed task (16 words of 8 bytes) from
// the ring in mapped host memory into shared memory in parallel, one word
// each: one round trip over the host link instead of sixteen. The ring entry
// was written before the host's release store of `tail`, which the claim
// read with acquire order, and is not rewritten before the task completes.
__device__ void copy_task(const KArgs& a, unsigned long long h, Task& dst) {
  if (threadIdx.x < sizeof(Task) / 8) {
    const volatile unsigned long long* src =
        reinterpret_cast<const volatile unsigned long long*>(&a.hc->tasks[h % kQueue]);
    reinterpret_cast<unsigned long long*>(&dst)[threadIdx.x] = src[threadIdx.x];
  }
}

// The source row that staged row t of a band holds (staging index t):
// kRowPairs: t = 2 ly + k holds tap row k of output row ly; otherwise staged
// rows are the window's rows, t = source row.
__device__ int staged_source_row(const fkl::ResampleParams& q, int t) {
  if (q.flags & kRowPairs) {
    const fkl::AxisTap ty = fkl::AxisWalker(t >> 1, q.rh, q.dh).tap();
    return (t & 1) ? ty.i1 : ty.i0;
  }
  return t;
}

// Gathers the staged rows of output rows [ly0, ly1) of the window (all
// threads of the CTA): each row's 3 rw bytes are copied from the host image
// with 16-byte loads of the aligned chunks wholly inside the row and single
// bytes at its two ends (nothing outside the row is read); staged row t keeps
// the host row's alignment: byte b of the row sits at t * pitch + off + b,
// off = (host row address) mod 16, recorded in the offset table.
__device__ void gather_band(const Task& task, int ly0, int ly1, int* s_rows, int* s_src, int* s_off) {
  const fkl::ResampleParams& q = task.rp;
  const bool pairs = q.flags & kRowPairs;
  int first, last;  // staged rows of the band: [first, last]
  if (pairs) {
    first = 2 * ly0;
    last = 2 * ly1 - 1;
  } else {
    first = fkl::AxisWalker(ly0, q.rh, q.dh).tap().i0;
    last = fkl::AxisWalker(ly1 - 1, q.rh, q.dh).tap().i1;
  }
  const int rows = last - first + 1;  // <= kMaxStaged for a downscale band; full windows may need more
  const int nb = 3 * q.rw;
  int32_t* offsets = const_cast<int32_t*>(reinterpret_cast<const int32_t*>(q.uv));
  uint8_t* stage = const_cast<uint8_t*>(q.src);
  for (int base = 0; base < rows; base += kMaxStaged) {
    const int k = min(kMaxStaged, rows - base);
    __syncthreads();  // the previous round's table is no longer read
    if (threadIdx.x < k) {
      const int t = first + base + threadIdx.x;
      const int src = staged_source_row(q, t);
      const uint8_t* g = task.host + static_cast<int64_t>(src) * task.host_pitch;
      s_rows[threadIdx.x] = t;
      s_src[threadIdx.x] = src;
      s_off[threadIdx.x] = static_cast<int>(reinterpret_cast<uintptr_t>(g) & 15);
      offsets[t] = s_off[threadIdx.x];
    }
    __syncthreads();
    const int chunks = (nb + 30) / 16 + 1;  // per row, whatever its offset
    // the chunks wholly inside a row: four 16-byte loads in flight per thread
    // before their stores (the host link's latency is paid once per four)
    constexpr int kU = 4;
    for (int i = threadIdx.x; i < k * chunks; i += kU * blockDim.x) {
      uint4 v[kU];
      uint8_t* d[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        d[u] = nullptr;
        const int j = i + u * blockDim.x;
        if (j >= k * chunks) continue;
        const int r = j / chunks, c = j - r * chunks;
        const int lo = 16 * c - s_off[r];  // row byte of the chunk's first byte
        if (lo < 0 || lo + 16 > nb) continue;
        d[u] = stage + static_cast<int64_t>(s_rows[r]) * q.pitch + 16 * c;
        v[u] = __ldcs(reinterpret_cast<const uint4*>(task.host + static_cast<int64_t>(s_src[r]) * task.host_pitch + lo));
      }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (d[u]) __stcg(reinterpret_cast<uint4*>(d[u]), v[u]);
    }
    // the partial chunks at the two ends of each row, byte by byte
    for (int i = threadIdx.x; i < k * 32; i += blockDim.x) {
      const int r = i / 32, e = i - r * 32;
      const int off = s_off[r];
      const int c = e < 16 ? 0 : (off + nb - 1) / 16;  // first or last chunk of the row
      if (e >= 16 && c == 0) continue;                 // a one-chunk row: done with e < 16
      const int lo = 16 * c - off;
      if (lo >= 0 && lo + 16 <= nb) continue;          // a whole chunk: copied above
      const int b = lo + (e & 15);
      if (b < 0 || b >= nb) continue;
      stage[static_cast<int64_t>(s_rows[r]) * q.pitch + off + b] =
          __ldcs(task.host + static_cast<int64_t>(s_src[r]) * task.host_pitch + b);
    }
  }
  __threadfence_block();
  __syncthreads();
}

// The bilinear value of window pixel (lx, ly) from the staged rows (the
// integer blend of ResizeU8C3T::blend_bytes: the fused reader's bits).
__device__ fkl::F3 staged_pixel(const fkl::ResampleParams& q, const fkl::AxisTap& tx, const fkl::AxisTap& ty, int ly) {
  const bool pairs = q.flags & kRowPairs;
  const int t0 = pairs ? 2 * ly : ty.i0, t1 = pairs ? 2 * ly + 1 : ty.i1;
  const int32_t* offsets = reinterpret_cast<const int32_t*>(q.uv);
  const uint8_t* r0 = q.src + static_cast<int64_t>(t0) * q.pitch + __ldcg(offsets + t0);
  const uint8_t* r1 = q.src + static_cast<int64_t>(t1) * q.pitch + __ldcg(offsets + t1);
  uint32_t b[4][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b[0][c] = __ldcg(r0 + 3 * tx.i0 + c);
    b[1][c] = __ldcg(r0 + 3 * tx.i1 + c);
    b[2][c] = __ldcg(r1 + 3 * tx.i0 + c);
    b[3][c] = __ldcg(r1 + 3 * tx.i1 + c);
  }
  return fkl::ResizeU8C3::blend_bytes(b, tx, 2 * q.dw, ty, 2 * q.dh, q.inv_area);
}

template <bool kSwap, class OutT>
__global__ void __launch_bounds__(kThreads, 4) serve_kernel(const __grid_constant__ KArgs a) {
  using Wr = fkl::WriteSplit<OutT>;
  __shared__ Task task;
  __shared__ int cmd;
  __shared__ unsigned long long claimed;
  __shared__ int s_rows[kMaxStaged], s_src[kMaxStaged], s_off[kMaxStaged];
  const int cols = (a.W + kV - 1) / kV;
  for (;;) {
    if (threadIdx.x == 0) {
      int c = claim(a, &claimed);
      while (c == 0) {
        // Leaving: the last CTA re-checks the ring after its decrement, so a
        // task published while it was deciding is never stranded (either it
        // sees the task here or the host sees no active CTA and relaunches).
        cuda::atomic_ref<int, cuda::thread_scope_system> active(a.hc->active);
        cuda::atomic_ref<int, cuda::thread_scope_system> stop(a.hc->stop);
        const int left = active.fetch_sub(1, cuda::memory_order_acq_rel) - 1;
        if (left != 0 || stop.load(cuda::memory_order_relaxed)) break;
        cuda::atomic_thread_fence(cuda::memory_order_seq_cst, cuda::thread_scope_system);
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> head(a.dc->head);
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(a.hc->tail);
        if (head.load(cuda::memory_order_relaxed) >= tail.load(cuda::memory_order_acquire)) break;
        active.fetch_add(1, cuda::memory_order_acq_rel);
        c = claim(a, &claimed);
      }
      cmd = c;
    }
    __syncthreads();
    if (cmd == 0) return;
    copy_task(a, claimed, task);
    __syncthreads();
    const fkl::ResampleParams& q = task.rp;
    const int y0 = task.band * kBand, y1 = min(y0 + kBand, a.H);
    // the band's rows inside the placed window
    const int ly0 = max(y0 - q.oy, 0), ly1 = min(y1 - q.oy, q.dh);
    if (ly0 < ly1) gather_band(task, ly0, ly1, s_rows, s_src, s_off);
    fkl::OutParams wp;
    wp.base = task.out;
    wp.img = 0;
    wp.plane = task.plane;
    wp.pitch = a.pitch;
    wp.scale_inv = a.scale_inv;
    wp.aligned = a.aligned;
    wp.scale_inv_dev = nullptr;
    const int items = cols * (y1 - y0);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int y = y0 + it / cols;
      const int x0 = (it % cols) * kV;
      const int n = min(kV, a.W - x0);
      const int ly = y - q.oy;
      const bool row_in = ly >= 0 && ly < q.dh;
      fkl::AxisTap ty{0, 0, 0};
      if (row_in) ty = fkl::AxisWalker(ly, q.rh, q.dh).tap();
      const int lx0 = x0 - q.ox;
      fkl::AxisWalker wx(max(lx0, 0), q.rw, q.dw);
      fkl::F3 o[kV];
#pragma unroll
      for (int k = 0; k < kV; ++k) {
        const int lx = lx0 + k;
        fkl::F3 v{{q.pad, q.pad, q.pad}};
        if (k < n && row_in && lx >= 0 && lx < q.dw) {
          v = staged_pixel(q, wx.tap(), ty, ly);
          wx.next();
        }
        if constexpr (kSwap) v = fkl::SwapRB<fkl::F3>::exec(v);
        v = fkl::Mul3::exec(v, a.mul);
        v = fkl::Sub3::exec(v, a.sub);
        o[k] = fkl::Div3::exec(v, a.div);
      }
      Wr::template exec_span<kV>(fkl::Point{x0, y, 0}, n, o, wp);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> fin(a.dc->finished[task.slot]);
      if (fin.fetch_add(1, cuda::memory_order_acq_rel) + 1 == task.target) {
        cuda::atomic_thread_fence(cuda::memory_order_seq_cst, cuda::thread_scope_system);
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> done(a.hc->done[task.slot]);
        done.store(task.seq, cuda::memory_order_release);
      }
    }
  }
}

using KernelFn = void (*)(KArgs);

template <class OutT>
KernelFn pick(bool swap) {
  return swap ? serve_kernel<true, OutT> : serve_kernel<false, OutT>;
}

KernelFn kernel_for(const Spec& s) {
  switch (s.out_dtype) {
    case FKL_F32:
      return pick<float>(s.swap);
    case FKL_F16:
      return pick<fkl::f16_t>(s.swap);
    case FKL_BF16:
      return pick<fkl::bf16_t>(s.swap);
    case FKL_E4M3:
      return pick<fkl::e4m3_t>(s.swap);
    default:
      return nullptr;
  }
}

double now_s() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + ts.tv_nsec * 1e-9;
}

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t len, size_t& off) {
    len = up(len, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        off = it->first;
        const size_t rest = it->second - len;
        const size_t start = it->first + len;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += len;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t len) {
    len = up(len, 256);
    used_ -= len;
    auto it = free_.emplace(off, len).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t id = 0, seq = 0;
  int n = 0, slot = -1, state = 0;
  std::vector<fkl_tensor> host;
  std::vector<const uint8_t*> window;  // persistent mode: device address of each host window's origin
  std::vector<fkl::ResampleParams> rp;
  uint64_t ntasks = 0, target = 0;     // persistent mode: band tasks, slot counter at completion
  size_t off = 0, len = 0, in_bytes = 0;
  uint64_t first_task = 0;
  double t_submit = 0, t_admit = 0, t_ready = 0, t_done = 0;
  cudaEvent_t ev_copy = nullptr, ev_done = nullptr;
};

}  // namespace serve
}  // namespace fkl_impl

using namespace fkl_impl;
using namespace fkl_impl::serve;

struct fkl_server_s {
  fkl_pipeline p = nullptr;
  fkl_server_config cfg{};
  int device = 0;
  int H = 0, W = 0, el = 0;
  int64_t out_pitch = 0;
  size_t out_img = 0;
  uint8_t* arena_base = nullptr;
  Arena* arena = nullptr;
  HostCtl* hc = nullptr;
  HostCtl* hc_dev = nullptr;
  DevCtl* dc = nullptr;
  std::vector<uint64_t> slot_tasks;  // persistent mode: tasks ever assigned to each slot
  int bands = 0;                     // tasks per image (output rows / kBand, rounded up)
  uint8_t* ws[2] = {nullptr, nullptr};  // unfused-mode workspace per copy stream
  size_t ws_bytes = 0;
  KernelFn kernel = nullptr;
  KArgs kargs{};
  int grid = 0;
  cudaStream_t s_copy[2] = {nullptr, nullptr};  // requests alternate between two copy engines
  std::vector<cudaStream_t> s_kernel;
  std::thread thread;
  std::mutex mu;
  std::condition_variable cv;
  bool quit = false;
  std::deque<uint64_t> pending;
  std::map<uint64_t, Request> reqs;
  std::vector<int> free_slots;
  uint64_t next_id = 1, next_seq = 1, tail = 0;
  fkl_server_stats stats{};
  std::string thread_error;
};

namespace {

fkl_status sfail(fkl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

// Relaunch CTAs if some have left (persistent mode). Called with the lock.
void ensure_kernel(fkl_server_s* s) {
  cuda::atomic_ref<int, cuda::thread_scope_system> active(s->hc->active);
  std::atomic_thread_fence(std::memory_order_seq_cst);
  const int a = active.load(cuda::memory_order_acquire);
  if (a >= s->grid) return;
  for (cudaStream_t st : s->s_kernel) {
    if (cudaStreamQuery(st) != cudaSuccess) continue;  // a kernel still runs there
    const int add = s->grid - a;
    active.fetch_add(add, cuda::memory_order_acq_rel);
    s->kernel<<<add, kThreads, 0, st>>>(s->kargs);
    if (cudaGetLastError() != cudaSuccess) {
      active.fetch_sub(add, cuda::memory_order_acq_rel);
      s->thread_error = "persistent kernel launch failed";
      return;
    }
    s->stats.kernel_launches++;
    return;
  }
}

// The source window and placement of image i of a request.
fkl::ResampleParams window_params(const fkl_server_s* s, const fkl_tensor& h) {
  fkl::ResampleParams p;
  std::memset(&p, 0, sizeof(p));
  const Spec& sp = s->p->spec;
  p.rw = sp.has_crop ? sp.crop[2] : static_cast<int32_t>(h.dims[1]);
  p.rh = sp.has_crop ? sp.crop[3] : static_cast<int32_t>(h.dims[0]);
  place(sp, s->W, s->H, p);
  return p;
}

// Persistent mode's device memory for one image: the staged rows (kRowPairs:
// two per window row of the output, when that is fewer than the window's
// rows) with room for their host alignment, then their offset table.
struct StagedLayout {
  int rows;
  int64_t pitch, rows_bytes, bytes;
  bool pairs;
};
StagedLayout staged_layout(const fkl::ResampleParams& p) {
  StagedLayout L;
  L.pairs = p.rh > 2 * p.dh;
  L.rows = L.pairs ? 2 * p.dh : p.rh;
  L.pitch = static_cast<int64_t>(up(static_cast<size_t>(3) * p.rw + 32, 16));
  L.rows_bytes = static_cast<int64_t>(up(static_cast<size_t>(L.rows * L.pitch), 256));
  L.bytes = L.rows_bytes + static_cast<int64_t>(up(static_cast<size_t>(L.rows) * 4, 256));
  return L;
}

// Persistent mode: the arena holds each image's staged rows and the outputs;
// nothing is copied here -- the kernel gathers each band's rows from the
// pinned host image itself.
bool admit_persistent(fkl_server_s* s, Request& r) {
  std::vector<StagedLayout> lay(r.n);
  std::vector<fkl::ResampleParams> wp(r.n);
  size_t in_bytes = 0;
  for (int i = 0; i < r.n; ++i) {
    wp[i] = window_params(s, r.host[i]);
    lay[i] = staged_layout(wp[i]);
    in_bytes += static_cast<size_t>(lay[i].bytes);
  }
  const size_t len = in_bytes + r.n * s->out_img;
  size_t off = 0;
  if (!s->arena->alloc(len, off)) return false;
  r.slot = s->free_slots.back();
  s->free_slots.pop_back();
  r.off = off;
  r.len = len;
  r.in_bytes = in_bytes;
  r.seq = s->next_seq++;
  uint8_t* base = s->arena_base + off;
  r.rp.resize(r.n);
  size_t at = 0;
  for (int i = 0; i < r.n; ++i) {
    fkl::ResampleParams& p = r.rp[i];
    p = wp[i];
    p.src = base + at;
    p.uv = base + at + lay[i].rows_bytes;  // the staged rows' offset table (int32)
    p.pitch = static_cast<int32_t>(lay[i].pitch);
    p.flags = lay[i].pairs ? kRowPairs : 0;
    at += static_cast<size_t>(lay[i].bytes);
  }
  r.ntasks = static_cast<uint64_t>(r.n) * s->bands;
  s->slot_tasks[r.slot] += r.ntasks;
  r.target = s->slot_tasks[r.slot];
  r.state = 1;
  r.t_admit = now_s();
  s->stats.admitted++;
  return true;
}

bool admit(fkl_server_s* s, Request& r) {
  if (s->free_slots.empty()) return false;
  if (s->cfg.mode == FKL_SERVE_PERSISTENT) return admit_persistent(s, r);
  // layout: images at their tight row size (one contiguous copy each when
  // the host rows are tight too), 256-byte aligned, then the outputs
  size_t in_bytes = 0;
  std::vector<size_t> offs(r.n);
  for (int i = 0; i < r.n; ++i) {
    offs[i] = in_bytes;
    in_bytes += up(static_cast<size_t>(r.host[i].dims[0]) * r.host[i].dims[1] * 3, 256);
  }
  const size_t len = in_bytes + r.n * s->out_img;
  size_t off = 0;
  if (!s->arena->alloc(len, off)) return false;
  r.slot = s->free_slots.back();
  s->free_slots.pop_back();
  r.off = off;
  r.len = len;
  r.in_bytes = in_bytes;
  r.seq = s->next_seq++;
  uint8_t* base = s->arena_base + off;
  const cudaStream_t cs = s->s_copy[r.seq & 1];
  r.rp.resize(r.n);
  cudaError_t ce = cudaSuccess;
  std::vector<fkl_tensor> dev_in(r.n);
  for (int i = 0; i < r.n && ce == cudaSuccess; ++i) {
    const fkl_tensor& h = r.host[i];
    const int64_t row = h.dims[1] * 3;
    const int64_t hp = h.pitch_bytes ? h.pitch_bytes : row;
    const int64_t dp = row;
    ce = hp == row ? cudaMemcpyAsync(base + offs[i], h.data, static_cast<size_t>(row * h.dims[0]),
                                     cudaMemcpyHostToDevice, cs)
                   : cudaMemcpy2DAsync(base + offs[i], dp, h.data, hp, row, h.dims[0], cudaMemcpyHostToDevice, cs);
    fkl::ResampleParams& p = r.rp[i];
    std::memset(&p, 0, sizeof(p));
    p.src = base + offs[i];
    p.pitch = static_cast<int32_t>(dp);
    const Spec& sp = s->p->spec;
    p.rx = sp.has_crop ? sp.crop[0] : 0;
    p.ry = sp.has_crop ? sp.crop[1] : 0;
    p.rw = sp.has_crop ? sp.crop[2] : static_cast<int32_t>(h.dims[1]);
    p.rh = sp.has_crop ? sp.crop[3] : static_cast<int32_t>(h.dims[0]);
    place(sp, s->W, s->H, p);
    dev_in[i] = h;
    dev_in[i].data = base + offs[i];
    dev_in[i].pitch_bytes = dp;
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(r.ev_copy, cs);
  if (ce == cudaSuccess) {
    fkl_tensor out{};
    out.data = base + in_bytes;
    out.dims[0] = r.n;
    out.dims[1] = 3;
    out.dims[2] = s->H;
    out.dims[3] = s->W;
    out.pitch_bytes = s->out_pitch;
    out.dtype = s->p->spec.out_dtype;
    out.layout = FKL_LAYOUT_NCHW;
    const fkl_status st =
        s->cfg.mode == FKL_SERVE_BATCH
            ? fkl_execute_batch(s->p, r.n, dev_in.data(), nullptr, &out, cs)
            : fkl_execute_batch_unfused(s->p, r.n, dev_in.data(), nullptr, &out, s->ws[r.seq & 1], s->ws_bytes, cs);
    if (st != FKL_OK) s->thread_error = fkl_last_error();
    s->stats.kernel_launches += s->cfg.mode == FKL_SERVE_BATCH ? 1 : 0;
    ce = cudaEventRecord(r.ev_done, cs);
  }
  if (ce != cudaSuccess) s->thread_error = cudaGetErrorString(ce);
  r.state = 1;
  r.t_admit = now_s();
  s->stats.admitted++;
  return true;
}

// Writes a request's band tasks into the ring (persistent mode); false when
// the ring has no room for them yet.
bool publish(fkl_server_s* s, Request& r) {
  uint64_t oldest = s->tail;
  for (auto& kv : s->reqs)
    if (kv.second.state == 2) oldest = std::min(oldest, kv.second.first_task);
  if (s->tail + r.ntasks - oldest > static_cast<uint64_t>(kQueue)) return false;  // ring full
  uint8_t* out = s->arena_base + r.off + r.in_bytes;
  r.first_task = s->tail;
  uint64_t k = s->tail;
  for (int i = 0; i < r.n; ++i) {
    const int64_t hp = r.host[i].pitch_bytes ? r.host[i].pitch_bytes : r.host[i].dims[1] * 3;
    for (int b = 0; b < s->bands; ++b, ++k) {
      Task& t = s->hc->tasks[k % kQueue];
      t.rp = r.rp[i];
      t.host = r.window[i];
      t.host_pitch = hp;
      t.out = out + i * s->out_img;
      t.plane = static_cast<int64_t>(s->H) * s->out_pitch;
      t.seq = r.seq;
      t.target = r.target;
      t.slot = r.slot;
      t.band = b;
    }
  }
  s->tail = k;
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(s->hc->tail);
  tail.store(s->tail, cuda::memory_order_release);
  ensure_kernel(s);
  return true;
}

// How long destroy waits for in-flight requests before it stops the kernels.
constexpr double kShutdownGraceS = 10.0;

void server_loop(fkl_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  double t_quit = 0.0;
  for (;;) {
    bool progress = false;
    int busy = 0;
    for (auto& kv : s->reqs) {
      Request& r = kv.second;
      if (r.state == 1 && (s->cfg.mode == FKL_SERVE_PERSISTENT || cudaEventQuery(r.ev_copy) == cudaSuccess)) {
        if (s->cfg.mode == FKL_SERVE_PERSISTENT) {
          if (!publish(s, r)) continue;
        }
        r.state = 2;
        r.t_ready = now_s();
        progress = true;
      }
      if (r.state == 2) {
        bool done;
        if (s->cfg.mode == FKL_SERVE_PERSISTENT) {
          cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> d(s->hc->done[r.slot]);
          done = d.load(cuda::memory_order_acquire) == r.seq;
        } else {
          done = cudaEventQuery(r.ev_done) == cudaSuccess;
        }
        if (done) {
          r.state = 3;
          r.t_done = now_s();
          s->stats.completed++;
          s->stats.images_completed += r.n;
          progress = true;
        }
      }
      if (r.state == 1 || r.state == 2) ++busy;
    }
    while (!s->pending.empty()) {
      Request& r = s->reqs[s->pending.front()];
      if (!admit(s, r)) break;  // FIFO: the head waits for a slot or memory
      s->pending.pop_front();
      progress = true;
    }
    if (s->cfg.mode == FKL_SERVE_PERSISTENT && s->tail > 0 && busy > 0) ensure_kernel(s);
    s->stats.queued = static_cast<int32_t>(s->pending.size());
    s->stats.inflight = busy;
    if (progress) s->cv.notify_all();
    if (s->quit) {
      if (t_quit == 0.0) t_quit = now_s();
      if ((busy == 0 && s->pending.empty()) || now_s() - t_quit > kShutdownGraceS) break;
    }
    if (!progress) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(busy ? 5 : 50));
      lk.lock();
    }
  }
}

void teardown(fkl_server_s* s) {
  if (s->hc) {
    cuda::atomic_ref<int, cuda::thread_scope_system> stop(s->hc->stop);
    stop.store(1, cuda::memory_order_release);
  }
  for (cudaStream_t st : s->s_kernel)
    if (st) cudaStreamSynchronize(st);
  for (cudaStream_t st : s->s_copy)
    if (st) cudaStreamSynchronize(st);
  for (auto& kv : s->reqs) {
    if (kv.second.ev_copy) cudaEventDestroy(kv.second.ev_copy);
    if (kv.second.ev_done) cudaEventDestroy(kv.second.ev_done);
  }
  for (cudaStream_t st : s->s_kernel)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : s->s_copy)
    if (st) cudaStreamDestroy(st);
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->dc) cudaFree(s->dc);
  for (uint8_t* w : s->ws)
    if (w) cudaFree(w);
  if (s->hc) cudaFreeHost(s->hc);
  delete s->arena;
  delete s;
}

}  // namespace

extern "C" {

fkl_status fkl_server_create(fkl_pipeline p, const fkl_server_config* cfg, fkl_server* out) {
  if (!out) return sfail(FKL_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!p || !cfg) return sfail(FKL_ERR_INVALID, "null argument");
  const Spec& sp = p->spec;
  if (sp.family != FAM_PACKED || sp.geom == GEOM_NONE || !sp.split)
    return sfail(FKL_ERR_UNSUPPORTED, "servers run READ_U8C3 [CROP] RESIZE|LETTERBOX ... WRITE_SPLIT chains");
  if (cfg->mode < FKL_SERVE_PERSISTENT || cfg->mode > FKL_SERVE_UNFUSED || cfg->max_inflight < 1 ||
      cfg->max_inflight > kMaxSlots || cfg->arena_bytes < (1u << 20) || cfg->ctas_per_sm < 1 ||
      cfg->ctas_per_sm > 8 || cfg->idle_us < 1)
    return sfail(FKL_ERR_INVALID, "bad server config (mode, 1..%d slots, arena >= 1 MiB, 1..8 CTAs/SM, idle_us > 0)",
                 kMaxSlots);
  auto* s = new (std::nothrow) fkl_server_s;
  if (!s) return sfail(FKL_ERR_OOM, "host allocation failed");
  s->p = p;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->H = sp.out_h;
  s->W = sp.out_w;
  s->el = sp.out_dtype == FKL_F32 ? 4 : (sp.out_dtype == FKL_E4M3 ? 1 : 2);
  s->out_pitch = static_cast<int64_t>(up(static_cast<size_t>(s->W) * s->el, 16));
  s->out_img = up(3 * static_cast<size_t>(s->H) * s->out_pitch, 256);
  s->kernel = kernel_for(sp);
  cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(&s->arena_base), cfg->arena_bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void**>(&s->dc), sizeof(DevCtl));
  if (ce == cudaSuccess) ce = cudaMemset(s->dc, 0, sizeof(DevCtl));
  if (ce == cudaSuccess) ce = cudaHostAlloc(reinterpret_cast<void**>(&s->hc), sizeof(HostCtl), cudaHostAllocMapped);
  if (ce == cudaSuccess) {
    std::memset(s->hc, 0, sizeof(HostCtl));
    ce = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->hc_dev), s->hc, 0);
  }
  if (ce == cudaSuccess && cfg->mode == FKL_SERVE_UNFUSED) {
    s->ws_bytes = 2 * up(static_cast<size_t>(s->H) * s->W * 12, 256);
    for (int i = 0; i < 2 && ce == cudaSuccess; ++i) ce = cudaMalloc(reinterpret_cast<void**>(&s->ws[i]), s->ws_bytes);
  }
  for (int i = 0; i < 2 && ce == cudaSuccess; ++i) ce = cudaStreamCreateWithFlags(&s->s_copy[i], cudaStreamNonBlocking);
  for (int i = 0; i < 4 && ce == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->s_kernel.push_back(st);
  }
  if (ce != cudaSuccess) {
    teardown(s);
    return sfail(FKL_ERR_CUDA, "server setup: %s", cudaGetErrorString(ce));
  }
  s->arena = new Arena(cfg->arena_bytes);
  for (int i = cfg->max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->slot_tasks.assign(cfg->max_inflight, 0);
  s->bands = (s->H + kBand - 1) / kBand;
  s->grid = sm_count() * cfg->ctas_per_sm;
  KArgs& k = s->kargs;
  k.hc = s->hc_dev;
  k.dc = s->dc;
  k.H = s->H;
  k.W = s->W;
  k.pitch = s->out_pitch;
  k.scale_inv = sp.out_dtype == FKL_E4M3 ? static_cast<float>(1.0 / sp.fp8_scale) : 1.f;
  k.aligned = 1;
  std::memcpy(k.mul.c, sp.mul, sizeof(k.mul.c));
  std::memcpy(k.sub.c, sp.sub, sizeof(k.sub.c));
  std::memcpy(k.div.c, sp.div, sizeof(k.div.c));
  k.div.on = sp.has_div ? 1 : 0;
  k.idle_ns = static_cast<unsigned long long>(cfg->idle_us) * 1000ull;
  s->thread = std::thread(server_loop, s);
  *out = s;
  return FKL_OK;
}

fkl_status fkl_server_submit(fkl_server s, int32_t n, const fkl_tensor* images, uint64_t* request_id) {
  if (!s || !request_id || n < 1 || !images) return sfail(FKL_ERR_INVALID, "bad submit arguments");
  if (n > kQueue / 2) return sfail(FKL_ERR_INVALID, "a request may hold at most %d images", kQueue / 2);
  Request r;
  r.n = n;
  r.host.assign(images, images + n);
  size_t need = 0;
  const Spec& sp = s->p->spec;
  const bool persistent = s->cfg.mode == FKL_SERVE_PERSISTENT;
  if (persistent && static_cast<int64_t>(n) * s->bands > kQueue)
    return sfail(FKL_ERR_INVALID, "a request may hold at most %d images (%d tasks of %d output rows each)",
                 kQueue / s->bands, s->bands, kBand);
  for (int i = 0; i < n; ++i) {
    const fkl_tensor& t = images[i];
    if (!t.data || t.layout != FKL_LAYOUT_HWC || t.dtype != FKL_U8 || t.dims[2] != 3 || t.dims[0] < 1 ||
        t.dims[1] < 1 || t.dims[0] > 16384 || t.dims[1] > 16384)
      return sfail(FKL_ERR_INVALID, "image %d: host HWC u8 with 3 channels, 1..16384 per side", i);
    if (t.pitch_bytes && t.pitch_bytes < t.dims[1] * 3) return sfail(FKL_ERR_INVALID, "image %d: pitch too small", i);
    if (sp.has_crop && (sp.crop[0] + int64_t(sp.crop[2]) > t.dims[1] || sp.crop[1] + int64_t(sp.crop[3]) > t.dims[0]))
      return sfail(FKL_ERR_INVALID, "image %d: the chain's crop does not fit", i);
    if (persistent) {
      // the kernel reads the image itself: it must be pinned (device-accessible) host memory
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, t.data) != cudaSuccess || at.type != cudaMemoryTypeHost ||
          !at.devicePointer) {
        cudaGetLastError();
        return sfail(FKL_ERR_INVALID, "image %d: persistent servers read pinned host memory (cudaHostAlloc or "
                     "cudaHostRegister)", i);
      }
      const int64_t hp = t.pitch_bytes ? t.pitch_bytes : t.dims[1] * 3;
      const int64_t x = sp.has_crop ? sp.crop[0] : 0, y = sp.has_crop ? sp.crop[1] : 0;
      r.window.push_back(static_cast<const uint8_t*>(at.devicePointer) + y * hp + 3 * x);
      need += static_cast<size_t>(staged_layout(window_params(s, t)).bytes);
    } else {
      need += up(static_cast<size_t>(t.dims[0]) * t.dims[1] * 3, 256);
    }
  }
  need += n * s->out_img;
  if (up(need, 256) > s->arena->size())
    return sfail(FKL_ERR_INVALID, "request needs %zu bytes, the server arena holds %zu", need, s->arena->size());
  if (cudaEventCreateWithFlags(&r.ev_copy, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r.ev_done, cudaEventDisableTiming) != cudaSuccess)
    return sfail(FKL_ERR_CUDA, "event creation failed");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->quit) {
    cudaEventDestroy(r.ev_copy);
    cudaEventDestroy(r.ev_done);
    return sfail(FKL_ERR_INVALID, "server is shutting down");
  }
  r.id = s->next_id++;
  r.t_submit = now_s();
  *request_id = r.id;
  s->pending.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  s->stats.submitted++;
  return FKL_OK;
}

static void fill_out(fkl_server s, const Request& r, fkl_tensor* out) {
  if (!out) return;
  std::memset(out, 0, sizeof(*out));
  out->data = s->arena_base + r.off + r.in_bytes;
  out->dims[0] = r.n;
  out->dims[1] = 3;
  out->dims[2] = s->H;
  out->dims[3] = s->W;
  out->pitch_bytes = s->out_pitch;
  out->dtype = s->p->spec.out_dtype;
  out->layout = FKL_LAYOUT_NCHW;
}

fkl_status fkl_server_poll(fkl_server s, uint64_t id, int32_t* done, fkl_tensor* out) {
  if (!s || !done) return sfail(FKL_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(FKL_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
  *done = it->second.state == 3;
  if (*done) fill_out(s, it->second, out);
  return FKL_OK;
}

fkl_status fkl_server_wait(fkl_server s, uint64_t id, int32_t timeout_ms, fkl_tensor* out) {
  if (!s) return sfail(FKL_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(FKL_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
  const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return it->second.state == 3; });
  if (!ok) return sfail(FKL_ERR_TIMEOUT, "request %llu not done after %d ms", (unsigned long long)id, timeout_ms);
  fill_out(s, it->second, out);
  return FKL_OK;
}

fkl_status fkl_server_request_info(fkl_server s, uint64_t id, fkl_request_info* info) {
  if (!s || !info) return sfail(FKL_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(FKL_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
  const Request& r = it->second;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_ready = r.t_ready;
  info->t_done = r.t_done;
  info->n_images = r.n;
  info->state = r.state;
  return FKL_OK;
}

fkl_status fkl_server_release(fkl_server s, uint64_t id) {
  if (!s) return sfail(FKL_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(FKL_ERR_INVALID, "unknown request %llu", (unsigned long long)id);
  if (it->second.state != 3) return sfail(FKL_ERR_INVALID, "request %llu is not done", (unsigned long long)id);
  Request& r = it->second;
  s->arena->release(r.off, r.len);
  s->free_slots.push_back(r.slot);
  cudaEventDestroy(r.ev_copy);
  cudaEventDestroy(r.ev_done);
  s->reqs.erase(it);
  return FKL_OK;
}

fkl_status fkl_server_get_stats(fkl_server s, fkl_server_stats* st) {
  if (!s || !st) return sfail(FKL_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->arena_peak_bytes = s->arena->peak();
  if (!s->thread_error.empty()) return sfail(FKL_ERR_CUDA, "server thread: %s", s->thread_error.c_str());
  return FKL_OK;
}

void fkl_server_destroy(fkl_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->quit = true;
  }
  if (s->thread.joinable()) s->thread.join();
  teardown(s);
}

}  // extern "C"
