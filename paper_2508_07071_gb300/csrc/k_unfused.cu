// The unfused reference form of the image chains (paper §II Fig. 3A and
// Algorithm 1, "MainFunctionA"): one kernel per operation, each reading its
// input image from device memory and writing its result back. The kernels
// reuse the very Operations of the fused chains, so the two forms agree bit
// for bit; only the data movement differs.
#include <cstring>

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

}  // namespace

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
