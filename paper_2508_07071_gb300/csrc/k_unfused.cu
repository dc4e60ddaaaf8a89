// The unfused reference form of the image chains (paper §II Fig. 3A and
// Algorithm 1, "MainFunctionA"): one kernel per operation, each reading its
// input image from device memory and writing its result back. The kernels
// reuse the very Operations of the fused chains, so the two forms agree bit
// for bit; only the data movement differs.
#include <algorithm>
#include <cstring>
#include <vector>

#include "registry.h"

namespace fkl_impl {

namespace {

constexpr int kV = 4;
constexpr int kTX = 32;
constexpr int kTY = 8;

template <class ROp, class W, class Cops>
cudaError_t step(const fkl::ResampleParams& rp, const fkl::OutParams& wp, const Cops& cops, int H,
                 int W_, cudaStream_t st) {
  using RB = fkl::BatchRead<ROp, 1>;
  fkl::Args2D<RB, W, Cops> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = 1;
  a.rp.p[0] = rp;
  a.wp = wp;
  a.cops = cops;
  a.H = H;
  a.W_ = W_;
  return fkl::launch_transform2d<kV, 1>(a, 1, kTX, kTY, st);
}

// A packed float32 H x W x 3 intermediate image in workspace memory.
fkl::ResampleParams f32_image(const void* p, int H, int W) {
  fkl::ResampleParams r;
  std::memset(&r, 0, sizeof(r));
  r.src = static_cast<const uint8_t*>(p);
  r.pitch = W * 12;
  r.rw = r.dw = W;
  r.rh = r.dh = H;
  return r;
}
fkl::OutParams f32_out(void* p, int H, int W) {
  fkl::OutParams o;
  std::memset(&o, 0, sizeof(o));
  o.base = static_cast<uint8_t*>(p);
  o.pitch = W * 12;
  o.img = static_cast<int64_t>(H) * o.pitch;
  o.plane = o.img;
  o.scale_inv = 1.f;
  o.aligned = (o.pitch % 16) == 0 ? 1 : 0;  // workspace bases are 256-byte aligned
  return o;
}
fkl::ResampleParams u8_image(const void* p, int H, int W) {
  fkl::ResampleParams r = f32_image(p, H, W);
  r.pitch = W * 3;
  return r;
}
fkl::OutParams u8_out(void* p, int H, int W) {
  fkl::OutParams o = f32_out(p, H, W);
  o.pitch = W * 3;
  o.img = o.plane = static_cast<int64_t>(H) * o.pitch;
  o.aligned = 0;
  return o;
}

using PackF32 = fkl::WritePacked<float>;

template <class OutT>
cudaError_t final_write(const Spec& s, const void* src, const fkl::OutParams& out, int H, int W,
                        cudaStream_t st) {
  if (s.split)
    return step<fkl::ReadF32C3, fkl::WriteSplit<OutT>>(f32_image(src, H, W), out, fkl::make_tuple(), H, W, st);
  if constexpr (std::is_same_v<OutT, float>)
    return step<fkl::ReadF32C3, fkl::WritePacked<OutT>>(f32_image(src, H, W), out, fkl::make_tuple(), H, W, st);
  return cudaErrorInvalidValue;  // packed outputs are float32 only
}

cudaError_t float_tail(const Spec& s, void* cur, void* other, const fkl::OutParams& out, int H,
                       int W, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  auto swap_bufs = [&] { std::swap(cur, other); };
  if (s.swap) {
    e = step<fkl::ReadF32C3, PackF32>(f32_image(cur, H, W), f32_out(other, H, W),
                                      fkl::make_tuple(fkl::IOp<fkl::SwapRB<fkl::F3>>{}), H, W, st);
    if (e != cudaSuccess) return e;
    swap_bufs();
  }
  if (s.has_mul) {
    fkl::IOp<fkl::Mul3> op;
    std::memcpy(op.params.c, s.mul, sizeof(op.params.c));
    e = step<fkl::ReadF32C3, PackF32>(f32_image(cur, H, W), f32_out(other, H, W), fkl::make_tuple(op), H, W, st);
    if (e != cudaSuccess) return e;
    swap_bufs();
  }
  if (s.has_sub) {
    fkl::IOp<fkl::Sub3> op;
    std::memcpy(op.params.c, s.sub, sizeof(op.params.c));
    e = step<fkl::ReadF32C3, PackF32>(f32_image(cur, H, W), f32_out(other, H, W), fkl::make_tuple(op), H, W, st);
    if (e != cudaSuccess) return e;
    swap_bufs();
  }
  if (s.has_div) {
    fkl::IOp<fkl::Div3> op;
    std::memcpy(op.params.c, s.div, sizeof(op.params.c));
    op.params.on = 1;
    e = step<fkl::ReadF32C3, PackF32>(f32_image(cur, H, W), f32_out(other, H, W), fkl::make_tuple(op), H, W, st);
    if (e != cudaSuccess) return e;
    swap_bufs();
  }
  switch (s.out_dtype) {
    case FKL_F32:
      return final_write<float>(s, cur, out, H, W, st);
    case FKL_F16:
      return final_write<fkl::f16_t>(s, cur, out, H, W, st);
    case FKL_BF16:
      return final_write<fkl::bf16_t>(s, cur, out, H, W, st);
    case FKL_E4M3:
      return final_write<fkl::e4m3_t>(s, cur, out, H, W, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// The per-op form over a batch (paper §II Fig. 3A, Algorithm 1 "MainFunctionA"
// over all images: each operation is one kernel over every image of the
// chunk). Intermediates are packed float32 images, one slot per image.
// ---------------------------------------------------------------------------

// Elementwise COps over packed float32 pixels: every thread takes 4 pixels
// (three 16-byte vectors) per step of a grid-stride loop; slots are
// multiples of 48 bytes, so a vector group never straddles two pixels'
// channels out of phase.
template <class Cops>
__global__ void __launch_bounds__(256) pixels_f32c3_kernel(const float4* __restrict__ in, float4* __restrict__ out,
                                                           int64_t groups, const __grid_constant__ Cops cops) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += stride) {
    const float4 a = __ldcs(in + 3 * g), b = __ldcs(in + 3 * g + 1), c = __ldcs(in + 3 * g + 2);
    fkl::F3 p[4] = {{{a.x, a.y, a.z}}, {{a.w, b.x, b.y}}, {{b.z, b.w, c.x}}, {{c.y, c.z, c.w}}};
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = fkl::apply_chain(p[k], cops);
    __stcs(out + 3 * g, make_float4(p[0].v[0], p[0].v[1], p[0].v[2], p[1].v[0]));
    __stcs(out + 3 * g + 1, make_float4(p[1].v[1], p[1].v[2], p[2].v[0], p[2].v[1]));
    __stcs(out + 3 * g + 2, make_float4(p[2].v[2], p[3].v[0], p[3].v[1], p[3].v[2]));
  }
}

// One group of 4 pixels per thread (a grid-stride loop only past 2^31 - 1
// blocks): a persistent grid of 8 blocks per SM ran 20% slower on 1.26 GB.
template <class Cops>
cudaError_t pixels_step(const void* in, void* out, int64_t bytes, const Cops& cops, cudaStream_t st) {
  const int64_t groups = bytes / 48;
  const int64_t want = (groups + 255) / 256;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, 0x7FFFFFFF)));
  pixels_f32c3_kernel<Cops><<<grid, 256, 0, st>>>(static_cast<const float4*>(in), static_cast<float4*>(out),
                                                  groups, cops);
  return cudaGetLastError();
}

// The per-op form's NV12 decode (source window -> packed float32 RGB) with
// coalesced stores: a warp decodes 128 consecutive pixels of one row, 4 per
// lane (DecodeNV12::exec_span, the same arithmetic as every other decode),
// stages the 1536 bytes in its own shared memory and writes them as 16-byte
// vectors at consecutive lanes, 512 contiguous bytes per store instruction.
// (The generic packed write stores 16 bytes per lane 48 bytes apart; for a
// step that writes 8 bytes per byte it reads, that kept the L1 store path
// the busiest unit and the step at 72% of the copy bandwidth.) Rows must
// start 16-byte aligned: window width a multiple of 4.
constexpr int kDecodePx = 128;  // pixels per warp
struct DecodeArgs {
  fkl::BatchRead<fkl::DecodeNV12, fkl::kBatchCap>::ParamsType rp;
  uint8_t* out;   // image z's row y at out + z * slot + y * 12 W
  int64_t slot;
  int32_t W, H;   // window width and height (equal for every image of the launch)
  int32_t segs;   // warp segments per row: ceil(W / kDecodePx)
};

__global__ void __launch_bounds__(256) decode_rows_kernel(const __grid_constant__ DecodeArgs a) {
  __shared__ __align__(16) float stage[8][3 * kDecodePx];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = blockIdx.y;
  const int item = blockIdx.x * 8 + warp;  // (row, segment) of this warp
  if (z >= a.rp.count || item >= a.H * a.segs) return;  // uniform for the warp
  const int y = item / a.segs;
  const int x0 = (item - y * a.segs) * kDecodePx;
  const int L = min(kDecodePx, a.W - x0);
  const fkl::ResampleParams& q = a.rp.p[z];
  const int xs = x0 + 4 * lane;
  fkl::F3 v[4];
  if (xs + 4 <= a.W) {
    fkl::DecodeNV12::exec_span<4>(fkl::Point{xs, y, z}, q, v);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (xs + k < a.W) v[k] = fkl::DecodeNV12::exec(fkl::Point{xs + k, y, z}, q);
  }
  float* st = stage[warp];
  if (xs + 4 <= a.W) {
    float4* s4 = reinterpret_cast<float4*>(st + 12 * lane);
    s4[0] = make_float4(v[0].v[0], v[0].v[1], v[0].v[2], v[1].v[0]);
    s4[1] = make_float4(v[1].v[1], v[1].v[2], v[2].v[0], v[2].v[1]);
    s4[2] = make_float4(v[2].v[2], v[3].v[0], v[3].v[1], v[3].v[2]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (xs + k < a.W)
#pragma unroll
        for (int c = 0; c < 3; ++c) st[12 * lane + 3 * k + c] = v[k].v[c];
  }
  __syncwarp();
  uint8_t* row = a.out + z * a.slot + (static_cast<int64_t>(y) * a.W + x0) * 12;
  const int nbytes = 12 * L;
  for (int j = lane; 16 * j < nbytes; j += 32) {
    if (16 * j + 16 <= nbytes) {
      __stcs(reinterpret_cast<float4*>(row) + j, reinterpret_cast<const float4*>(st)[j]);
    } else {
      for (int b = 4 * j; 4 * b < nbytes; ++b) reinterpret_cast<float*>(row)[b] = st[b];
    }
  }
}

cudaError_t decode_rows(const fkl::ResampleParams* rp, int n, uint8_t* out, int64_t slot, int H, int W,
                        cudaStream_t st) {
  DecodeArgs a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = n;
  std::memcpy(a.rp.p, rp, sizeof(fkl::ResampleParams) * n);
  a.out = out;
  a.slot = slot;
  a.W = W;
  a.H = H;
  a.segs = (W + kDecodePx - 1) / kDecodePx;
  const int64_t items = int64_t(H) * a.segs;
  decode_rows_kernel<<<dim3(static_cast<unsigned>((items + 7) / 8), n, 1), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One 2-D step over `n` images: ROp per image (params `rp[i]`) to WOp.
constexpr int kBV = 4;  // pixels per thread of the batched 2-D steps
template <class ROp, class W, int V = kBV, int RY = 1>
cudaError_t batch_step(const fkl::ResampleParams* rp, int n, const fkl::OutParams& wp, int H, int W_,
                       cudaStream_t st) {
  using RB = fkl::BatchRead<ROp, fkl::kBatchCap>;
  fkl::Args2D<RB, W, fkl::Tuple<>> a;
  std::memset(&a.rp, 0, sizeof(a.rp));
  a.rp.count = n;
  std::memcpy(a.rp.p, rp, sizeof(fkl::ResampleParams) * n);
  a.wp = wp;
  a.H = H;
  a.W_ = W_;
  return fkl::launch_transform2d<V, RY>(a, n, kTX, kTY, st);
}

template <class OutT>
cudaError_t batch_final_write(const Spec& s, const fkl::ResampleParams* rp, int n, const fkl::OutParams& out,
                              int H, int W, cudaStream_t st) {
  constexpr int V = 8;  // 16-byte runs of 16-bit planes, 8-byte runs of FP8 planes
  if (s.split) return batch_step<fkl::ReadF32C3, fkl::WriteSplit<OutT>, V>(rp, n, out, H, W, st);
  if constexpr (std::is_same_v<OutT, float>) return batch_step<fkl::ReadF32C3, fkl::WritePacked<OutT>>(rp, n, out, H, W, st);
  return cudaErrorInvalidValue;  // packed outputs are float32 only
}

// Distinct source indices the half-pixel taps reference along one axis (a
// tap of weight 0 is not referenced).
int64_t axis_taps(int n_src, int n_dst) {
  if (n_dst <= 0) return 0;
  std::vector<char> used(n_src, 0);
  for (int64_t d = 0; d < n_dst; ++d) {
    const int64_t num = (2 * d + 1) * n_src - n_dst, D = 2 * int64_t(n_dst);
    const int64_t q = num >= 0 ? num / D : -((-num + D - 1) / D);
    const int64_t r = num - q * D;
    const int64_t i0 = std::min<int64_t>(std::max<int64_t>(q, 0), n_src - 1);
    used[i0] = 1;
    if (q >= 0 && q < n_src - 1 && r > 0) used[i0 + 1] = 1;
  }
  int64_t k = 0;
  for (char u : used) k += u;
  return k;
}

}  // namespace

void PerOpLog::begin(const char* name, double bytes, cudaStream_t st) {
  if (!on) return;
  Entry e;
  e.name = name;
  e.bytes = bytes;
  if (cudaEventCreate(&e.start) != cudaSuccess || cudaEventCreate(&e.stop) != cudaSuccess) {
    failed = true;
    return;
  }
  cudaEventRecord(e.start, st);
  entries.push_back(e);
}
void PerOpLog::end(cudaStream_t st) {
  if (on && !entries.empty()) cudaEventRecord(entries.back().stop, st);
}

cudaError_t launch_per_op_chunk(const Spec& s, const fkl::ResampleParams* imgs, int n, const fkl::OutParams& out,
                                int H, int W, uint8_t* ws0, uint8_t* ws1, int64_t slot_in, int64_t slot,
                                PerOpLog& log, cudaStream_t st) {
  const double px = static_cast<double>(n) * H * W;
  std::vector<fkl::ResampleParams> rp(imgs, imgs + n);
  cudaError_t e = cudaSuccess;
  if (s.family == FAM_NV12) {
    // decode each source window at full resolution to unit-range RGB; one
    // launch per run of images with the same window size
    for (int i = 0; i < n && e == cudaSuccess;) {
      int j = i + 1;
      while (j < n && imgs[j].rw == imgs[i].rw && imgs[j].rh == imgs[i].rh) ++j;
      fkl::OutParams o = f32_out(ws0 + i * slot_in, imgs[i].rh, imgs[i].rw);
      o.img = slot_in;
      const double win = static_cast<double>(j - i) * imgs[i].rw * imgs[i].rh;
      log.begin("decode NV12 -> RGB f32", win * (1.5 + 12.0), st);
      e = imgs[i].rw % 4 == 0 ? decode_rows(imgs + i, j - i, ws0 + i * slot_in, slot_in, imgs[i].rh, imgs[i].rw, st)
                              : batch_step<fkl::DecodeNV12, PackF32>(imgs + i, j - i, o, imgs[i].rh, imgs[i].rw, st);
      log.end(st);
      i = j;
    }
    if (e != cudaSuccess) return e;
    // resize / letterbox the decoded images (scaled to 0..255 after the blend)
    double taps = 0.0;
    for (int i = 0; i < n; ++i) {
      fkl::ResampleParams& r = rp[i];
      r.src = ws0 + i * slot_in;
      r.uv = nullptr;
      r.pitch = imgs[i].rw * 12;
      r.rx = r.ry = 0;
      r.flags &= fkl::kExact2x;
      taps += 12.0 * axis_taps(r.rw, r.dw) * axis_taps(r.rh, r.dh);
    }
    fkl::OutParams o = f32_out(ws1, H, W);
    o.img = slot;
    log.begin(s.geom == GEOM_LETTERBOX ? "letterbox f32" : "resize f32", taps + 12.0 * px, st);
    e = batch_step<fkl::ResizeF32C3T<true>, PackF32>(rp.data(), n, o, H, W, st);
    log.end(st);
  } else if (s.family == FAM_PACKED) {
    double taps = 0.0;
    for (int i = 0; i < n; ++i) taps += 3.0 * axis_taps(imgs[i].rw, imgs[i].dw) * axis_taps(imgs[i].rh, imgs[i].dh);
    fkl::OutParams o = f32_out(ws1, H, W);
    o.img = slot;
    log.begin(s.geom == GEOM_NONE ? "crop u8 -> f32" : "crop + resize u8 -> f32", taps + 12.0 * px, st);
    e = batch_step<fkl::ResizeU8C3, PackF32>(imgs, n, o, H, W, st);
    log.end(st);
  } else {
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  // the compute ops, one kernel each over every pixel of the chunk (ws1 -> ws0 -> ...)
  uint8_t* cur = ws1;
  uint8_t* other = ws0;
  const int64_t bytes = n * slot;
  auto ew = [&](const char* name, const auto& cops) {
    if (e != cudaSuccess) return;
    log.begin(name, 24.0 * px, st);
    e = pixels_step(cur, other, bytes, cops, st);
    log.end(st);
    std::swap(cur, other);
  };
  if (s.swap) ew("BGR <-> RGB", fkl::make_tuple(fkl::IOp<fkl::SwapRB<fkl::F3>>{}));
  if (s.has_mul) {
    fkl::IOp<fkl::Mul3> op;
    std::memcpy(op.params.c, s.mul, sizeof(op.params.c));
    ew("multiply", fkl::make_tuple(op));
  }
  if (s.has_sub) {
    fkl::IOp<fkl::Sub3> op;
    std::memcpy(op.params.c, s.sub, sizeof(op.params.c));
    ew("subtract", fkl::make_tuple(op));
  }
  if (s.has_div) {
    fkl::IOp<fkl::Div3> op;
    std::memcpy(op.params.c, s.div, sizeof(op.params.c));
    op.params.on = 1;
    ew("divide", fkl::make_tuple(op));
  }
  if (e != cudaSuccess) return e;
  // the write: packed float32 images -> the output layout and type
  std::vector<fkl::ResampleParams> fin(n);
  for (int i = 0; i < n; ++i) fin[i] = f32_image(cur + i * slot, H, W);
  const int ob = s.out_dtype == FKL_F32 ? 4 : (s.out_dtype == FKL_E4M3 ? 1 : 2);
  log.begin(s.split ? "split + cast" : "write", px * (12.0 + 3.0 * ob), st);
  switch (s.out_dtype) {
    case FKL_F32:
      e = batch_final_write<float>(s, fin.data(), n, out, H, W, st);
      break;
    case FKL_F16:
      e = batch_final_write<fkl::f16_t>(s, fin.data(), n, out, H, W, st);
      break;
    case FKL_BF16:
      e = batch_final_write<fkl::bf16_t>(s, fin.data(), n, out, H, W, st);
      break;
    case FKL_E4M3:
      e = batch_final_write<fkl::e4m3_t>(s, fin.data(), n, out, H, W, st);
      break;
    default:
      e = cudaErrorInvalidValue;
  }
  log.end(st);
  return e;
}

cudaError_t launch_unfused_image(const Spec& s, const fkl::ResampleParams& img,
                                 const fkl::OutParams& out, int z, int H, int W, void* ws0,
                                 void* ws1, cudaStream_t st) {
  fkl::OutParams o = out;
  o.base += z * out.img;
  cudaError_t e = cudaSuccess;
  if (s.family == FAM_PACKED) {
    // resize (u8 -> f32 HWC), then the compute ops, then the write
    e = step<fkl::ResizeU8C3, PackF32>(img, f32_out(ws0, H, W), fkl::make_tuple(), H, W, st);
    if (e != cudaSuccess) return e;
    return float_tail(s, ws0, ws1, o, H, W, st);
  }
  if (s.family == FAM_NV12) {
    // decode the source window to unit-range RGB f32 HWC, resize / letterbox
    // it (scaled to 0..255 after the blend), ...
    fkl::ResampleParams dec = img;
    e = step<fkl::DecodeNV12, PackF32>(dec, f32_out(ws0, img.rh, img.rw), fkl::make_tuple(), img.rh,
                                       img.rw, st);
    if (e != cudaSuccess) return e;
    fkl::ResampleParams rs = img;
    rs.src = static_cast<const uint8_t*>(ws0);
    rs.uv = nullptr;
    rs.pitch = img.rw * 12;
    rs.rx = rs.ry = 0;
    rs.flags = 0;
    e = step<fkl::ResizeF32C3T<true>, PackF32>(rs, f32_out(ws1, H, W), fkl::make_tuple(), H, W, st);
    if (e != cudaSuccess) return e;
    return float_tail(s, ws1, ws0, o, H, W, st);
  }
  if (s.family == FAM_INT) {
    e = step<fkl::CropU8C3, fkl::WriteU8C3<false>>(img, u8_out(ws0, H, W), fkl::make_tuple(), H, W, st);
    if (e != cudaSuccess) return e;
    void* cur = ws0;
    void* other = ws1;
    if (s.swap) {
      e = step<fkl::CropU8C3, fkl::WriteU8C3<false>>(u8_image(cur, H, W), u8_out(other, H, W),
                                                     fkl::make_tuple(fkl::IOp<fkl::SwapRB<fkl::U3>>{}), H, W, st);
      if (e != cudaSuccess) return e;
      std::swap(cur, other);
    }
    if (s.has_addsat) {
      fkl::IOp<fkl::AddSatU8> op;
      std::memcpy(op.params.k, s.addsat, sizeof(op.params.k));
      e = step<fkl::CropU8C3, fkl::WriteU8C3<false>>(u8_image(cur, H, W), u8_out(other, H, W),
                                                     fkl::make_tuple(op), H, W, st);
      if (e != cudaSuccess) return e;
      std::swap(cur, other);
    }
    if (s.split)
      return step<fkl::CropU8C3, fkl::WriteU8C3<true>>(u8_image(cur, H, W), o, fkl::make_tuple(), H, W, st);
    return step<fkl::CropU8C3, fkl::WriteU8C3<false>>(u8_image(cur, H, W), o, fkl::make_tuple(), H, W, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fkl_impl
