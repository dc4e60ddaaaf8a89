// Serving runtime (include/fkl.h, fkl_server_*): continuous batching of
// preprocessing requests with admission by free device memory.
//
// Persistent mode: a persistent kernel whose CTAs claim image tasks from a
// ring in mapped host memory (tail written by the host with release order,
// head claimed on the device with compare-and-swap), run the chain's Ops on
// the image, and count the request down; the CTA that finishes a request's
// last image publishes its sequence number to the host. Every device wait is
// bounded by an idle timeout on the global timer and by a stop flag.
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

struct Task {  // one image of one request
  fkl::ResampleParams rp;
  uint8_t* out;     // this image's first output plane
  int64_t plane;    // bytes between output planes
  uint64_t seq;     // request sequence number (its completion value)
  int32_t slot;     // request slot
  int32_t _pad[9];
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
  unsigned long long head;  // tasks claimed
  int remaining[kMaxSlots];  // images left per slot
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

// Thread 0: claim the next task into `dst`; 1 = claimed, 0 = stop or idle.
__device__ int claim(const KArgs& a, Task& dst) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> head(a.dc->head);
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(a.hc->tail);
  cuda::atomic_ref<int, cuda::thread_scope_system> stop(a.hc->stop);
  const unsigned long long t0 = globaltimer_ns();
  unsigned ns = 128;
  for (;;) {
    if (stop.load(cuda::memory_order_relaxed)) return 0;
    unsigned long long h = head.load(cuda::memory_order_relaxed);
    const unsigned long long t = tail.load(cuda::memory_order_acquire);
    if (h < t) {
      if (head.compare_exchange_strong(h, h + 1, cuda::memory_order_acq_rel)) {
        const volatile unsigned long long* src =
            reinterpret_cast<const volatile unsigned long long*>(&a.hc->tasks[h % kQueue]);
        unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
#pragma unroll
        for (int i = 0; i < static_cast<int>(sizeof(Task) / 8); ++i) d[i] = src[i];
        return 1;
      }
      continue;
    }
    if (globaltimer_ns() - t0 > a.idle_ns) return 0;
    __nanosleep(ns);
    ns = min(ns * 2, 16384u);
  }
}

template <bool kSwap, class OutT>
__global__ void __launch_bounds__(kThreads) serve_kernel(const __grid_constant__ KArgs a) {
  using R = fkl::ResizeU8C3T<true>;  // L2-coherent loads: the arena is reused while we run
  using Wr = fkl::WriteSplit<OutT>;
  __shared__ Task task;
  __shared__ int cmd;
  const int cols = (a.W + kV - 1) / kV;
  const int items = cols * a.H;
  for (;;) {
    if (threadIdx.x == 0) {
      int c = claim(a, task);
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
        c = claim(a, task);
      }
      cmd = c;
    }
    __syncthreads();
    if (cmd == 0) return;
    fkl::OutParams wp;
    wp.base = task.out;
    wp.img = 0;
    wp.plane = task.plane;
    wp.pitch = a.pitch;
    wp.scale_inv = a.scale_inv;
    wp.aligned = a.aligned;
    wp.scale_inv_dev = nullptr;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int y = it / cols;
      const int x0 = (it - y * cols) * kV;
      const int n = min(kV, a.W - x0);
      fkl::F3 in[kV];
      if (n == kV) {
        R::template exec_span<kV>(fkl::Point{x0, y, 0}, task.rp, in);
      } else {
        for (int k = 0; k < n; ++k) in[k] = R::exec(fkl::Point{x0 + k, y, 0}, task.rp);
      }
      fkl::F3 o[kV];
#pragma unroll
      for (int k = 0; k < kV; ++k) {
        fkl::F3 v = in[k];
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
      cuda::atomic_ref<int, cuda::thread_scope_device> rem(a.dc->remaining[task.slot]);
      if (rem.fetch_sub(1, cuda::memory_order_acq_rel) == 1) {
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
  std::vector<fkl::ResampleParams> rp;
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
  int* rem_staging = nullptr;  // pinned, one int per slot
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

bool admit(fkl_server_s* s, Request& r) {
  if (s->free_slots.empty()) return false;
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
  if (ce == cudaSuccess && s->cfg.mode == FKL_SERVE_PERSISTENT) {
    s->rem_staging[r.slot] = r.n;
    ce = cudaMemcpyAsync(&s->dc->remaining[r.slot], &s->rem_staging[r.slot], sizeof(int), cudaMemcpyHostToDevice,
                         cs);
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(r.ev_copy, cs);
  if (ce == cudaSuccess && s->cfg.mode != FKL_SERVE_PERSISTENT) {
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

bool publish(fkl_server_s* s, Request& r) {
  uint64_t oldest = s->tail;
  for (auto& kv : s->reqs)
    if (kv.second.state == 2) oldest = std::min(oldest, kv.second.first_task);
  if (s->tail + r.n - oldest > static_cast<uint64_t>(kQueue)) return false;  // ring full
  uint8_t* out = s->arena_base + r.off + r.in_bytes;
  r.first_task = s->tail;
  for (int i = 0; i < r.n; ++i) {
    Task& t = s->hc->tasks[(s->tail + i) % kQueue];
    t.rp = r.rp[i];
    t.out = out + i * s->out_img;
    t.plane = static_cast<int64_t>(s->H) * s->out_pitch;
    t.seq = r.seq;
    t.slot = r.slot;
  }
  s->tail += r.n;
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
      if (r.state == 1 && cudaEventQuery(r.ev_copy) == cudaSuccess) {
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
  if (s->rem_staging) cudaFreeHost(s->rem_staging);
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
  if (ce == cudaSuccess) ce = cudaHostAlloc(reinterpret_cast<void**>(&s->rem_staging), kMaxSlots * sizeof(int), 0);
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
  for (int i = 0; i < n; ++i) {
    const fkl_tensor& t = images[i];
    if (!t.data || t.layout != FKL_LAYOUT_HWC || t.dtype != FKL_U8 || t.dims[2] != 3 || t.dims[0] < 1 ||
        t.dims[1] < 1 || t.dims[0] > 16384 || t.dims[1] > 16384)
      return sfail(FKL_ERR_INVALID, "image %d: host HWC u8 with 3 channels, 1..16384 per side", i);
    if (t.pitch_bytes && t.pitch_bytes < t.dims[1] * 3) return sfail(FKL_ERR_INVALID, "image %d: pitch too small", i);
    if (sp.has_crop && (sp.crop[0] + int64_t(sp.crop[2]) > t.dims[1] || sp.crop[1] + int64_t(sp.crop[3]) > t.dims[0]))
      return sfail(FKL_ERR_INVALID, "image %d: the chain's crop does not fit", i);
    need += up(static_cast<size_t>(t.dims[0]) * t.dims[1] * 3, 256);
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
