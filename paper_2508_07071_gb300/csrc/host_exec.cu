// Host-buffer executor (include/fkl.h): chunked, overlapped copy-in, fused
// launch and copy-out on three streams with a ring of device slots.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "registry.h"

struct fkl_host_executor_s {
  fkl_pipeline p = nullptr;
  int chunk = 0, depth = 0;
  size_t in_stride = 0, out_bytes = 0;  // per image, in_stride rounded to 256
  std::vector<uint8_t*> d_in, d_out;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_run, ev_free;
  std::vector<bool> used;
  cudaEvent_t ev_start = nullptr;
};

namespace {

// Failures are reported through the library's thread-local message
// (fkl_last_error).
fkl_status exec_fail(fkl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  fkl_impl::set_last_error(buf);
  return s;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct HostImage {
  int64_t rows, row_bytes, pitch;
};

fkl_status host_image(const fkl_tensor& t, int i, HostImage& h) {
  if (!t.data) return exec_fail(FKL_ERR_INVALID, "host input %d missing", i);
  if (t.layout == FKL_LAYOUT_NV12) {
    h.rows = t.dims[0] * 3 / 2;
    h.row_bytes = t.dims[1];
  } else if (t.layout == FKL_LAYOUT_HWC) {
    h.rows = t.dims[0];
    h.row_bytes = t.dims[1] * t.dims[2];
  } else {
    return exec_fail(FKL_ERR_INVALID, "host input %d: HWC or NV12 layout expected", i);
  }
  if (h.rows <= 0 || h.row_bytes <= 0) return exec_fail(FKL_ERR_INVALID, "host input %d: empty", i);
  h.pitch = t.pitch_bytes ? t.pitch_bytes : h.row_bytes;
  if (h.pitch < h.row_bytes) return exec_fail(FKL_ERR_INVALID, "host input %d: pitch below row bytes", i);
  return FKL_OK;
}

int64_t out_image_bytes(const fkl_tensor& o, int64_t& pitch) {
  const int64_t el = o.dtype == FKL_F32 ? 4 : (o.dtype == FKL_F16 || o.dtype == FKL_BF16) ? 2 : 1;
  if (o.layout == FKL_LAYOUT_NCHW) {
    pitch = o.pitch_bytes ? o.pitch_bytes : o.dims[3] * el;
    return o.dims[1] * o.dims[2] * pitch;
  }
  pitch = o.pitch_bytes ? o.pitch_bytes : o.dims[2] * o.dims[3] * el;
  return o.dims[1] * pitch;
}

void release(fkl_host_executor e) {
  if (!e) return;
  if (e->s_in) cudaStreamSynchronize(e->s_in);
  if (e->s_run) cudaStreamSynchronize(e->s_run);
  if (e->s_out) cudaStreamSynchronize(e->s_out);
  for (auto* p : e->d_in)
    if (p) cudaFree(p);
  for (auto* p : e->d_out)
    if (p) cudaFree(p);
  for (auto v : {&e->ev_in, &e->ev_run, &e->ev_free})
    for (auto ev : *v)
      if (ev) cudaEventDestroy(ev);
  if (e->ev_start) cudaEventDestroy(e->ev_start);
  for (auto s : {e->s_in, e->s_run, e->s_out})
    if (s) cudaStreamDestroy(s);
  delete e;
}

}  // namespace

extern "C" {

fkl_status fkl_host_executor_create(fkl_pipeline p, int32_t chunk, int32_t depth, size_t in_bytes,
                                    size_t out_bytes, fkl_host_executor* out) {
  if (!out) return exec_fail(FKL_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!p) return exec_fail(FKL_ERR_INVALID, "null pipeline");
  if (chunk < 1 || chunk > 256 || depth < 1 || depth > 8 || !in_bytes || !out_bytes)
    return exec_fail(FKL_ERR_INVALID, "need 1 <= chunk <= 256, 1 <= depth <= 8, nonzero sizes");
  auto* e = new (std::nothrow) fkl_host_executor_s;
  if (!e) return exec_fail(FKL_ERR_OOM, "host allocation failed");
  e->p = p;
  e->chunk = chunk;
  e->depth = depth;
  e->in_stride = round_up(in_bytes, 256);
  e->out_bytes = out_bytes;
  e->d_in.assign(depth, nullptr);
  e->d_out.assign(depth, nullptr);
  e->ev_in.assign(depth, nullptr);
  e->ev_run.assign(depth, nullptr);
  e->ev_free.assign(depth, nullptr);
  e->used.assign(depth, false);
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < depth && ce == cudaSuccess; ++i) {
    ce = cudaMalloc(reinterpret_cast<void**>(&e->d_in[i]), e->in_stride * chunk);
    if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void**>(&e->d_out[i]), round_up(out_bytes, 256) * chunk);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->ev_in[i], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->ev_run[i], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->ev_free[i], cudaEventDisableTiming);
  }
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->ev_start, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&e->s_in, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&e->s_run, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&e->s_out, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    release(e);
    return exec_fail(FKL_ERR_CUDA, "host executor setup: %s", cudaGetErrorString(ce));
  }
  *out = e;
  return FKL_OK;
}

void fkl_host_executor_destroy(fkl_host_executor e) { release(e); }

fkl_status fkl_execute_batch_host(fkl_host_executor e, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                  fkl_tensor* out, void* stream) {
  if (!e) return exec_fail(FKL_ERR_INVALID, "null executor");
  if (n < 0 || (n > 0 && !ins) || !out || !out->data)
    return exec_fail(FKL_ERR_INVALID, "bad batch arguments");
  if (n == 0) return FKL_OK;
  if (out->layout != FKL_LAYOUT_NCHW && out->layout != FKL_LAYOUT_NHWC)
    return exec_fail(FKL_ERR_INVALID, "host output must be NCHW or NHWC");
  if (out->dims[0] < n) return exec_fail(FKL_ERR_INVALID, "host output holds fewer than %d images", n);
  int64_t out_pitch = 0;
  const int64_t out_img = out_image_bytes(*out, out_pitch);
  if (out_img <= 0 || static_cast<size_t>(out_img) > e->out_bytes)
    return exec_fail(FKL_ERR_INVALID, "output image of %lld bytes exceeds the executor's %zu",
                     static_cast<long long>(out_img), e->out_bytes);
  std::vector<HostImage> hi(n);
  for (int i = 0; i < n; ++i) {
    fkl_status st = host_image(ins[i], i, hi[i]);
    if (st != FKL_OK) return st;
    const size_t dev_bytes = static_cast<size_t>(hi[i].rows * round_up(hi[i].row_bytes, 16));
    if (dev_bytes > e->in_stride)
      return exec_fail(FKL_ERR_INVALID, "input %d needs %zu device bytes, the executor holds %zu per image", i,
                       dev_bytes, e->in_stride);
  }
  const cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaError_t ce = cudaEventRecord(e->ev_start, caller);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->s_in, e->ev_start, 0);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->s_out, e->ev_start, 0);
  if (ce != cudaSuccess) return exec_fail(FKL_ERR_CUDA, "host executor: %s", cudaGetErrorString(ce));

  std::vector<fkl_tensor> dev_in(e->chunk);
  int last_slot = 0;
  for (int start = 0, c = 0; start < n; start += e->chunk, ++c) {
    const int k = std::min(e->chunk, n - start);
    const int slot = c % e->depth;
    last_slot = slot;
    if (e->used[slot] && (ce = cudaStreamWaitEvent(e->s_in, e->ev_free[slot], 0)) != cudaSuccess) break;
    // copy-in: contiguous runs of tightly pitched images go as one copy
    for (int j = 0; j < k && ce == cudaSuccess;) {
      const fkl_tensor& t = ins[start + j];
      const HostImage& h = hi[start + j];
      const int64_t dpitch = static_cast<int64_t>(round_up(h.row_bytes, 16));
      uint8_t* dst = e->d_in[slot] + static_cast<size_t>(j) * e->in_stride;
      int run = 1;
      if (h.pitch == dpitch && static_cast<size_t>(h.rows * dpitch) == e->in_stride) {
        while (j + run < k && ins[start + j + run].data ==
                                  static_cast<const uint8_t*>(t.data) + static_cast<size_t>(run) * e->in_stride &&
               hi[start + j + run].pitch == dpitch && hi[start + j + run].rows == h.rows &&
               hi[start + j + run].row_bytes == h.row_bytes)
          ++run;
        ce = cudaMemcpyAsync(dst, t.data, static_cast<size_t>(run) * e->in_stride, cudaMemcpyHostToDevice, e->s_in);
      } else {
        ce = cudaMemcpy2DAsync(dst, dpitch, t.data, h.pitch, h.row_bytes, h.rows, cudaMemcpyHostToDevice, e->s_in);
      }
      for (int r = 0; r < run; ++r) {
        dev_in[j + r] = ins[start + j + r];
        dev_in[j + r].data = e->d_in[slot] + static_cast<size_t>(j + r) * e->in_stride;
        dev_in[j + r].pitch_bytes = dpitch;
      }
      j += run;
    }
    if (ce != cudaSuccess) break;
    if ((ce = cudaEventRecord(e->ev_in[slot], e->s_in)) != cudaSuccess) break;
    if ((ce = cudaStreamWaitEvent(e->s_run, e->ev_in[slot], 0)) != cudaSuccess) break;
    fkl_tensor dev_out = *out;
    dev_out.data = e->d_out[slot];
    dev_out.dims[0] = k;
    dev_out.pitch_bytes = out_pitch;
    const fkl_status st = fkl_execute_batch(e->p, k, dev_in.data(), rois ? rois + 4 * start : nullptr, &dev_out, e->s_run);
    if (st != FKL_OK) {
      const std::string why = fkl_last_error();
      return exec_fail(st, "chunk at image %d: %s", start, why.c_str());
    }
    if ((ce = cudaEventRecord(e->ev_run[slot], e->s_run)) != cudaSuccess) break;
    if ((ce = cudaStreamWaitEvent(e->s_out, e->ev_run[slot], 0)) != cudaSuccess) break;
    uint8_t* host_dst = static_cast<uint8_t*>(out->data) + static_cast<size_t>(start) * out_img;
    if ((ce = cudaMemcpyAsync(host_dst, e->d_out[slot], static_cast<size_t>(k) * out_img, cudaMemcpyDeviceToHost,
                              e->s_out)) != cudaSuccess)
      break;
    if ((ce = cudaEventRecord(e->ev_free[slot], e->s_out)) != cudaSuccess) break;
    e->used[slot] = true;
  }
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(caller, e->ev_free[last_slot], 0);
  if (ce != cudaSuccess) return exec_fail(FKL_ERR_CUDA, "host executor: %s", cudaGetErrorString(ce));
  return FKL_OK;
}

}  // extern "C"
