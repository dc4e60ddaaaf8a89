// Operations of the preprocessing chains: Read (K1), Compute (K2) and Write
// (K3) steps of paper Fig. 3, in the exec forms of paper Table I.
//
// Every floating-point step is written with an explicit rounding intrinsic
// (__fmul_rn, __fadd_rn, __fdiv_rn, ...), so the compiler cannot contract or
// reassociate across Ops. The same Op therefore gives the same bits whether
// it runs inside one fused kernel or alone in a kernel of its own, which is
// what lets the unfused reference form be compared bit for bit.
#pragma once

#include "core.cuh"

namespace fkl {

// ===========================================================================
// Geometry shared by the resampling Read Operations
// ===========================================================================

// Per-image parameters of a resampling ROp. The source window (rx, ry, rw,
// rh) is resized to dw x dh and placed at (ox, oy) in the output; output
// pixels outside the placed window read `pad` (letterbox). A plain resize is
// ox = oy = 0 and dw x dh = the output size; a plain crop is dw = rw, dh = rh.
struct ResampleParams {
  const uint8_t* src;  // packed image base, or NV12 luma plane
  const uint8_t* uv;   // NV12 chroma plane (nullptr otherwise)
  int32_t pitch;       // bytes per source row (both NV12 planes)
  int32_t rx, ry, rw, rh;
  int32_t ox, oy, dw, dh;
  float pad;
  float inv_area;      // fl32(1 / (4 dw dh)), integer-weight bilinear
  int32_t flags;       // kFast2x: exact 2x downscale, rows 16-byte aligned
};
static_assert(sizeof(ResampleParams) == 64, "kernel-parameter table entry");

constexpr int32_t kFast2x = 1;   // exact 2x, even 16-byte aligned window: vector loads
constexpr int32_t kExact2x = 2;  // rw == 2 dw and rh == 2 dh

// Whether the n outputs from (x0, y) of an image placed by resample
// parameters all lie outside its window, in the fill (letterbox) area.
// Only reads that place an image (kPlaced: the pad value outside the
// window) have such an area; the full-frame reads of the unfused chains
// carry the same parameters with another meaning.
FKL_HD bool fill_span(const ResampleParams& p, int x0, int y, int n) {
  const int lx = x0 - p.ox, ly = y - p.oy;
  return ly < 0 || ly >= p.dh || lx + n <= 0 || lx >= p.dw;
}

// Half-pixel sample along one axis for output index d (0 <= d < n_dst):
// u = (d + 1/2) n_src / n_dst - 1/2 = num / D with num = (2d+1) n_src - n_dst
// and D = 2 n_dst, clamped to [0, n_src - 1]. i0 = floor(u), i1 = min(i0 + 1,
// n_src - 1) and the weight of i1 is w1 / D, all in exact integers.
struct AxisTap {
  int i0;
  int i1;
  int w1;  // in units of 1/D
};

// Walks the taps of consecutive outputs d, d+1, ... with one division.
struct AxisWalker {
  int q, r;    // floor(num / D), num mod D of the current output
  int qs, rs;  // divmod of the step 2 n_src by D
  int D, n_src;

  FKL_D AxisWalker(int d, int n_src_, int n_dst) {
    n_src = n_src_;
    D = 2 * n_dst;
    const int num = (2 * d + 1) * n_src - n_dst;  // > -D for every d >= 0
    const int shifted = num + D;                  // > 0
    q = shifted / D - 1;
    r = shifted - (q + 1) * D;
    qs = (2 * n_src) / D;
    rs = 2 * n_src - qs * D;
  }
  FKL_D AxisTap tap() const {
    AxisTap t;
    if (q < 0) {
      t.i0 = 0;
      t.w1 = 0;
    } else if (q >= n_src - 1) {
      t.i0 = n_src - 1;
      t.w1 = 0;
    } else {
      t.i0 = q;
      t.w1 = r;
    }
    t.i1 = min(t.i0 + 1, n_src - 1);
    return t;
  }
  FKL_D void next() {
    q += qs;
    r += rs;
    if (r >= D) {
      r -= D;
      q += 1;
    }
  }
};

// Bilinear blend of four float taps (tRC: row R, column C) with weights
// w / D computed by IEEE division (exact whenever the ratio is representable,
// e.g. 1/2). Each column is blended vertically first, then the two columns
// horizontally; every path of this library uses that order.
FKL_D F3 blend_float(const F3& t00, const F3& t01, const F3& t10, const F3& t11,
                     const AxisTap& tx, int Dx, const AxisTap& ty, int Dy) {
  const float ax1 = __fdiv_rn(static_cast<float>(tx.w1), static_cast<float>(Dx));
  const float ax0 = __fdiv_rn(static_cast<float>(Dx - tx.w1), static_cast<float>(Dx));
  const float ay1 = __fdiv_rn(static_cast<float>(ty.w1), static_cast<float>(Dy));
  const float ay0 = __fdiv_rn(static_cast<float>(Dy - ty.w1), static_cast<float>(Dy));
  F3 o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float left = __fadd_rn(__fmul_rn(ay0, t00.v[c]), __fmul_rn(ay1, t10.v[c]));
    const float right = __fadd_rn(__fmul_rn(ay0, t01.v[c]), __fmul_rn(ay1, t11.v[c]));
    o.v[c] = __fadd_rn(__fmul_rn(ax0, left), __fmul_rn(ax1, right));
  }
  return o;
}

// ===========================================================================
// Read Operations
// ===========================================================================

// Source loads: through the read-only (non-coherent) path by default, or
// L2-only (`ld.global.cg`) for kernels whose source memory is rewritten while
// they run (the persistent serving kernel reuses its device arena), where a
// stale L1 line must never be read.
template <bool kCoherent>
FKL_D uint8_t load_u8(const uint8_t* p) {
  if constexpr (kCoherent) {
    return __ldcg(p);
  } else {
    return __ldg(p);
  }
}

// Packed 3-channel u8 image, crop window, bilinear resize and placement.
// The four taps are u8 integers, so the blend is done exactly in integers:
// N = (Dy - wy)((Dx - wx) S00 + wx S01) + wy((Dx - wx) S10 + wx S11) and the
// value is N / (Dx Dy) with a single float conversion and one multiply.
template <bool kCoherent>
struct ResizeU8C3T {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static constexpr bool kPlaced = true;  // the pad value outside the placed window

  // The blend of four taps' bytes: s[0] = S(x0, y0), s[1] = S(x1, y0),
  // s[2] = S(x0, y1), s[3] = S(x1, y1), each channel exact in integers.
  static FKL_D F3 blend_bytes(const uint32_t (&s)[4][3], const AxisTap& tx, int Dx, const AxisTap& ty, int Dy,
                              float inv_area) {
    const uint32_t wx1 = static_cast<uint32_t>(tx.w1);
    const uint32_t wx0 = static_cast<uint32_t>(Dx - tx.w1);
    const uint32_t wy1 = static_cast<uint32_t>(ty.w1);
    const uint32_t wy0 = static_cast<uint32_t>(Dy - ty.w1);
    F3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint32_t top = wx0 * s[0][c] + wx1 * s[1][c];
      const uint32_t bot = wx0 * s[2][c] + wx1 * s[3][c];
      const uint64_t n = static_cast<uint64_t>(wy0) * top + static_cast<uint64_t>(wy1) * bot;
      o.v[c] = __fmul_rn(__ull2float_rn(n), inv_area);
    }
    return o;
  }

  static FKL_D F3 blend(const uint8_t* row0, const uint8_t* row1, const AxisTap& tx,
                        int Dx, const AxisTap& ty, int Dy, float inv_area) {
    const uint8_t* p00 = row0 + 3 * tx.i0;
    const uint8_t* p01 = row0 + 3 * tx.i1;
    const uint8_t* p10 = row1 + 3 * tx.i0;
    const uint8_t* p11 = row1 + 3 * tx.i1;
    uint32_t s[4][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s[0][c] = load_u8<kCoherent>(p00 + c);
      s[1][c] = load_u8<kCoherent>(p01 + c);
      s[2][c] = load_u8<kCoherent>(p10 + c);
      s[3][c] = load_u8<kCoherent>(p11 + c);
    }
    return blend_bytes(s, tx, Dx, ty, Dy, inv_area);
  }

  static FKL_D F3 exec(const Point& pt, const ParamsType& p) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (lx < 0 || ly < 0 || lx >= p.dw || ly >= p.dh) return F3{{p.pad, p.pad, p.pad}};
    const AxisTap tx = AxisWalker(lx, p.rw, p.dw).tap();
    const AxisTap ty = AxisWalker(ly, p.rh, p.dh).tap();
    const uint8_t* base = p.src + static_cast<int64_t>(p.ry) * p.pitch + 3 * p.rx;
    return blend(base + static_cast<int64_t>(ty.i0) * p.pitch,
                 base + static_cast<int64_t>(ty.i1) * p.pitch, tx, 2 * p.dw, ty, 2 * p.dh,
                 p.inv_area);
  }

  // V consecutive outputs of one row: the row taps are found once and the
  // column taps by an incremental walk.
  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (ly < 0 || ly >= p.dh || lx < 0 || lx + V > p.dw) {
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
      return;
    }
    const AxisTap ty = AxisWalker(ly, p.rh, p.dh).tap();
    const uint8_t* base = p.src + static_cast<int64_t>(p.ry) * p.pitch + 3 * p.rx;
    const uint8_t* row0 = base + static_cast<int64_t>(ty.i0) * p.pitch;
    const uint8_t* row1 = base + static_cast<int64_t>(ty.i1) * p.pitch;
    AxisWalker wx(lx, p.rw, p.dw);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      out[k] = blend(row0, row1, wx.tap(), 2 * p.dw, ty, 2 * p.dh, p.inv_area);
      wx.next();
    }
  }
};

using ResizeU8C3 = ResizeU8C3T<false>;

// BT.601 limited-range decode constants, divided by 255 so that the clamp to
// [0, 255] becomes the free [0, 1] saturation of an add:
//   R = 255 sat(Y'/219 + (1 - Kr) V' / 112), B = 255 sat(Y'/219 + (1 - Kb) U' / 112),
//   G = 255 sat(Y'/219 - (1 - Kb)(Kb/Kg) U'/112 - (1 - Kr)(Kr/Kg) V'/112),
// Kr = 0.299, Kb = 0.114, Kg = 1 - Kr - Kb, Y' = Y - 16, U' = U - 128, V' = V - 128.
struct Bt601 {
  static constexpr double kr = 0.299, kb = 0.114, kg = 1.0 - kr - kb;
  static constexpr float cy = static_cast<float>(1.0 / 219.0);
  static constexpr float crv = static_cast<float>((1.0 - kr) / 112.0);
  static constexpr float cbu = static_cast<float>((1.0 - kb) / 112.0);
  static constexpr float cgu = static_cast<float>((1.0 - kb) * kb / kg / 112.0);
  static constexpr float cgv = static_cast<float>((1.0 - kr) * kr / kg / 112.0);
};

FKL_D float add_sat(float a, float b) {
  float d;
  asm("add.rn.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
FKL_D float sub_sat(float a, float b) {
  float d;
  asm("sub.rn.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}

// Chroma terms of one (U, V) sample, shared by the luma samples that use it.
struct ChromaTerms {
  float rv, guv, bu;
};
FKL_D ChromaTerms chroma_terms(float uf, float vf) {
  ChromaTerms t;
  t.rv = __fmul_rn(Bt601::crv, vf);
  t.guv = __fmaf_rn(Bt601::cgu, uf, __fmul_rn(Bt601::cgv, vf));
  t.bu = __fmul_rn(Bt601::cbu, uf);
  return t;
}
// BT.601 RGB of one luma sample yf = Y - 16 with its chroma terms, in
// [0, 1]: each channel's saturating add is its clamp. The resampling read ops
// interpolate these unit values and scale the result to 0..255 once per
// output (scale255); interpolation and the scale commute in exact arithmetic.
FKL_D F3 yuv_to_unit(float yf, const ChromaTerms& t) {
  const float l = __fmul_rn(Bt601::cy, yf);
  return F3{{add_sat(l, t.rv), sub_sat(l, t.guv), add_sat(l, t.bu)}};
}
FKL_D F3 scale255(const F3& u) {
  return F3{{__fmul_rn(u.v[0], 255.f), __fmul_rn(u.v[1], 255.f), __fmul_rn(u.v[2], 255.f)}};
}

constexpr float k2p23 = 8388608.f;

// The 2x span's constants as packed pairs in constant memory (both lanes
// equal): the packed instructions read them from the constant bank rather
// than from registers rebuilt for every use.
static __constant__ __align__(8) float kNv12Pairs[16] = {
    k2p23 + 16.f, k2p23 + 16.f,   k2p23 + 128.f, k2p23 + 128.f, Bt601::cy,  Bt601::cy,  Bt601::crv, Bt601::crv,
    Bt601::cgu,   Bt601::cgu,     Bt601::cgv,    Bt601::cgv,    Bt601::cbu, Bt601::cbu, 63.75f,     63.75f};

// 2^23 + (byte k of w), exactly, as a float: the byte is placed in the
// mantissa of 2^23 by one byte permute; subtracting 2^23 + bias later gives
// byte - bias exactly.
FKL_D float byte_as_float(uint32_t w, int k) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | static_cast<uint32_t>(k)));
}

// yuv_to_unit on a pair of luma samples (one per lane) with their chroma terms.
FKL_D void unit_pair(F2 yf, F2 cy, F2 rv, F2 guv, F2 bu, F2 (&o)[3]) {
  float l0, l1, r0, r1, g0, g1, b0, b1;
  f2split(f2mul(cy, yf), l0, l1);
  f2split(rv, r0, r1);
  f2split(guv, g0, g1);
  f2split(bu, b0, b1);
  o[0] = f2(add_sat(l0, r0), add_sat(l1, r1));
  o[1] = f2(sub_sat(l0, g0), sub_sat(l1, g1));
  o[2] = f2(add_sat(l0, b0), add_sat(l1, b1));
}

// One decoded NV12 sample in [0, 1] at absolute source coordinates (sx, sy):
// nearest (co-sited) chroma sample (sx/2, sy/2), U then V.
FKL_D F3 nv12_unit(const ResampleParams& p, int sx, int sy) {
  const float yf = static_cast<float>(__ldg(p.src + static_cast<int64_t>(sy) * p.pitch + sx)) - 16.f;
  const uint8_t* c = p.uv + static_cast<int64_t>(sy >> 1) * p.pitch + (sx & ~1);
  const float uf = static_cast<float>(__ldg(c)) - 128.f;
  const float vf = static_cast<float>(__ldg(c + 1)) - 128.f;
  return yuv_to_unit(yf, chroma_terms(uf, vf));
}

// NV12 frame -> BT.601 RGB -> crop window -> bilinear resize -> placement.
// Every tap is decoded (and clamped) first, then interpolated ("YUV->RGB,
// then resize" order); taps stay in [0, 1] and the interpolated value is
// scaled to 0..255.
struct ResizeNV12 {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static constexpr bool kPlaced = true;  // the pad value outside the placed window

  static FKL_D F3 exec(const Point& pt, const ParamsType& p) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (lx < 0 || ly < 0 || lx >= p.dw || ly >= p.dh) return F3{{p.pad, p.pad, p.pad}};
    const AxisTap tx = AxisWalker(lx, p.rw, p.dw).tap();
    const AxisTap ty = AxisWalker(ly, p.rh, p.dh).tap();
    const F3 t00 = nv12_unit(p, p.rx + tx.i0, p.ry + ty.i0);
    const F3 t01 = nv12_unit(p, p.rx + tx.i1, p.ry + ty.i0);
    const F3 t10 = nv12_unit(p, p.rx + tx.i0, p.ry + ty.i1);
    const F3 t11 = nv12_unit(p, p.rx + tx.i1, p.ry + ty.i1);
    return scale255(blend_float(t00, t01, t10, t11, tx, 2 * p.dw, ty, 2 * p.dh));
  }

  // Exact 2x downscale of an even-aligned window: output k of the span is
  // the mean of the 2x2 block that shares chroma sample k, so the span reads
  // 2V luma bytes from each of two rows and 2V chroma bytes, all as 16-byte
  // vectors. Outputs are processed in pairs, one per lane of the packed
  // f32x2 instructions; only the saturating adds are scalar. The result
  // equals exec() bit for bit: per lane the same IEEE operations run in the
  // same order. With weights 1/2 the blend of unit taps is exactly
  // fl(fl(u00 + u10) + fl(u01 + u11)) / 4, and scaled by 255 that is
  // fl(fl(fl(u00 + u10) + fl(u01 + u11)) * 63.75). No packed multiply feeds
  // a packed add in this sequence, so nothing can be fused into a
  // multiply-add that would round differently from the scalar form.
  template <int V>
  static FKL_D void span_fast2x(const ParamsType& p, int lx, int ly, F3 (&out)[V]) {
    uint4 a[V / 8], b[V / 8], c[V / 8];
    load2x<V>(p, lx, ly, a, b, c);
    compute2x<V>(a, b, c, out);
  }

  // Whether the V outputs from window position (lx, ly) take the 2x span
  // path (exact 2x, inside the window, 16-byte aligned source).
  template <int V>
  static FKL_D bool fast2x(const ParamsType& p, int lx, int ly) {
    return V % 8 == 0 && (p.flags & kFast2x) && ly >= 0 && ly < p.dh && lx >= 0 && lx + V <= p.dw &&
           ((2 * lx) & 15) == 0;
  }

  // The 16-byte words of the 2x span: two luma rows and the chroma row.
  template <int V>
  static FKL_D void load2x(const ParamsType& p, int lx, int ly, uint4 (&a)[V / 8], uint4 (&b)[V / 8],
                           uint4 (&c)[V / 8]) {
    static_assert(V % 8 == 0, "2x path reads 16-byte vectors");
    const int64_t y0 = p.ry + 2 * ly;
    const uint4* r0 = reinterpret_cast<const uint4*>(p.src + y0 * p.pitch + p.rx + 2 * lx);
    const uint4* r1 = reinterpret_cast<const uint4*>(p.src + (y0 + 1) * p.pitch + p.rx + 2 * lx);
    const uint4* rc = reinterpret_cast<const uint4*>(p.uv + (y0 >> 1) * p.pitch + p.rx + 2 * lx);
#pragma unroll
    for (int i = 0; i < V / 8; ++i) {
      a[i] = __ldg(r0 + i);
      b[i] = __ldg(r1 + i);
      c[i] = __ldg(rc + i);
    }
  }

  // The tap sums of outputs k, k+1 of the 2x span, one output per lane:
  // per channel fl(fl(u00 + u10) + fl(u01 + u11)) of the four unit taps,
  // before the scale to 0..255. wa, wb: word k/2 of the two luma rows'
  // 16-byte vectors, [left(k), right(k), left(k+1), right(k+1)]; wc: the
  // chroma word [U(k), V(k), U(k+1), V(k+1)].
  static FKL_D void pair_sums2x(uint32_t wa, uint32_t wb, uint32_t wc, F2 (&sum)[3]) {
    const F2* kp = reinterpret_cast<const F2*>(kNv12Pairs);
    const F2 kY = kp[0], kC = kp[1], cy = kp[2], crv = kp[3], cgu = kp[4], cgv = kp[5], cbu = kp[6];
    const F2 u = f2sub(f2(byte_as_float(wc, 0), byte_as_float(wc, 2)), kC);
    const F2 v = f2sub(f2(byte_as_float(wc, 1), byte_as_float(wc, 3)), kC);
    const F2 rv = f2mul(crv, v), guv = f2fma(cgu, u, f2mul(cgv, v)), bu = f2mul(cbu, u);
    F2 t[4][3];  // taps row 0 left, row 0 right, row 1 left, row 1 right
    unit_pair(f2sub(f2(byte_as_float(wa, 0), byte_as_float(wa, 2)), kY), cy, rv, guv, bu, t[0]);
    unit_pair(f2sub(f2(byte_as_float(wa, 1), byte_as_float(wa, 3)), kY), cy, rv, guv, bu, t[1]);
    unit_pair(f2sub(f2(byte_as_float(wb, 0), byte_as_float(wb, 2)), kY), cy, rv, guv, bu, t[2]);
    unit_pair(f2sub(f2(byte_as_float(wb, 1), byte_as_float(wb, 3)), kY), cy, rv, guv, bu, t[3]);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) sum[ch] = f2add(f2add(t[0][ch], t[2][ch]), f2add(t[1][ch], t[3][ch]));
  }

  // The arithmetic of the 2x span from the 16-byte words of the two luma
  // rows (a, b) and the chroma row (c), wherever they were loaded from.
  template <int V>
  static FKL_D void compute2x(const uint4 (&a)[V / 8], const uint4 (&b)[V / 8], const uint4 (&c)[V / 8],
                              F3 (&out)[V]) {
    const F2 c6375 = reinterpret_cast<const F2*>(kNv12Pairs)[7];
#pragma unroll
    for (int k = 0; k < V; k += 2) {
      // outputs k, k+1 use bytes 2k .. 2k+3 of each row: word (k % 8) / 2 of
      // vector k / 8
      const int vi = k / 8, wi = (k % 8) / 2;
      F2 sum[3];
      pair_sums2x(reinterpret_cast<const uint32_t*>(&a[vi])[wi], reinterpret_cast<const uint32_t*>(&b[vi])[wi],
                  reinterpret_cast<const uint32_t*>(&c[vi])[wi], sum);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) f2split(f2mul(sum[ch], c6375), out[k].v[ch], out[k + 1].v[ch]);
    }
  }

  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (ly < 0 || ly >= p.dh) {  // whole span in the letterbox band
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = F3{{p.pad, p.pad, p.pad}};
      return;
    }
    if constexpr (V % 8 == 0) {
      if ((p.flags & kFast2x) && lx >= 0 && lx + V <= p.dw && ((2 * lx) & 15) == 0) {
        span_fast2x<V>(p, lx, ly, out);
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
  }
};

// NV12 -> RGB -> exact 2x downscale (rw = 2 dw, rh = 2 dh) -> placement: a
// specialisation of ResizeNV12 with no division in it. Every output is the
// mean of one 2x2 block of unit taps scaled to 0..255,
// fl(fl(fl(u00 + u10) + fl(u01 + u11)) * 63.75), which is what the general
// bilinear blend and scale255 compute bit for bit when all weights are 1/2.
struct ResizeNV12x2 {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static constexpr bool kPlaced = true;  // the pad value outside the placed window

  static FKL_D F3 exec(const Point& pt, const ParamsType& p) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (lx < 0 || ly < 0 || lx >= p.dw || ly >= p.dh) return F3{{p.pad, p.pad, p.pad}};
    const int sx = p.rx + 2 * lx, sy = p.ry + 2 * ly;
    const F3 t00 = nv12_unit(p, sx, sy);
    const F3 t01 = nv12_unit(p, sx + 1, sy);
    const F3 t10 = nv12_unit(p, sx, sy + 1);
    const F3 t11 = nv12_unit(p, sx + 1, sy + 1);
    F3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      o.v[c] = __fmul_rn(__fadd_rn(__fadd_rn(t00.v[c], t10.v[c]), __fadd_rn(t01.v[c], t11.v[c])), 63.75f);
    return o;
  }

  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (ly < 0 || ly >= p.dh) {
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = F3{{p.pad, p.pad, p.pad}};
      return;
    }
    if constexpr (V % 8 == 0) {
      if ((p.flags & kFast2x) && lx >= 0 && lx + V <= p.dw && ((2 * lx) & 15) == 0) {
        ResizeNV12::span_fast2x<V>(p, lx, ly, out);
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
  }
};

// NV12 decode at full resolution to unit-range RGB (the first kernel of the
// unfused NV12 chain; its resize kernel scales to 0..255).
struct DecodeNV12 {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static FKL_D F3 exec(const Point& pt, const ParamsType& p) { return nv12_unit(p, p.rx + pt.x, p.ry + pt.y); }

  // V consecutive pixels of one row, from 4-byte words of the luma and the
  // chroma row when the first pixel's column is a multiple of 4 and the
  // pitch too (the same arithmetic as exec, one chroma term per pixel pair).
  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int sx = p.rx + pt.x, sy = p.ry + pt.y;
    if constexpr (V % 4 == 0) {
      if ((sx & 3) == 0 && (p.pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(p.src) & 3) == 0 &&
          (reinterpret_cast<uintptr_t>(p.uv) & 3) == 0) {
        const uint32_t* yw = reinterpret_cast<const uint32_t*>(p.src + static_cast<int64_t>(sy) * p.pitch + sx);
        const uint32_t* cw = reinterpret_cast<const uint32_t*>(p.uv + static_cast<int64_t>(sy >> 1) * p.pitch + sx);
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
          const uint32_t wy = __ldg(yw + i), wc = __ldg(cw + i);
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // chroma sample h serves pixels 2h, 2h + 1
            const float uf = static_cast<float>((wc >> (16 * h)) & 0xFFu) - 128.f;
            const float vf = static_cast<float>((wc >> (16 * h + 8)) & 0xFFu) - 128.f;
            const ChromaTerms t = chroma_terms(uf, vf);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const float yf = static_cast<float>((wy >> (8 * (2 * h + j))) & 0xFFu) - 16.f;
              out[4 * i + 2 * h + j] = yuv_to_unit(yf, t);
            }
          }
        }
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
  }
};

// Packed float32 3-channel image (an intermediate of the unfused chains),
// read through the same resampling geometry with float taps. kUnit: the
// image holds unit-range RGB (the unfused NV12 decode) and the blend is scaled
// to 0..255, the rounding points of the fused NV12 read.
template <bool kUnit>
struct ResizeF32C3T {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static constexpr bool kPlaced = true;  // the pad value outside the placed window
  static FKL_D F3 load(const ParamsType& p, int sx, int sy) {
    const float* q = reinterpret_cast<const float*>(p.src + static_cast<int64_t>(sy) * p.pitch) + 3 * sx;
    return F3{{__ldg(q), __ldg(q + 1), __ldg(q + 2)}};
  }
  static FKL_D F3 exec(const Point& pt, const ParamsType& p) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if (lx < 0 || ly < 0 || lx >= p.dw || ly >= p.dh) return F3{{p.pad, p.pad, p.pad}};
    const AxisTap tx = AxisWalker(lx, p.rw, p.dw).tap();
    const AxisTap ty = AxisWalker(ly, p.rh, p.dh).tap();
    const F3 b = blend_float(load(p, p.rx + tx.i0, p.ry + ty.i0), load(p, p.rx + tx.i1, p.ry + ty.i0),
                             load(p, p.rx + tx.i0, p.ry + ty.i1), load(p, p.rx + tx.i1, p.ry + ty.i1), tx,
                             2 * p.dw, ty, 2 * p.dh);
    if constexpr (kUnit) return scale255(b);
    return b;
  }

  // V outputs of one row of an exact 2x downscale, inside the window: the
  // taps of output k are source pixels 2k, 2k + 1 of two rows, read as
  // 16-byte vectors (the 24 V bytes of each row start 16-byte aligned); the
  // blend is blend_float's with its weights, which are exactly 1/2 here, so
  // the bits are exec's. Other spans take exec pixel by pixel.
  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int lx = pt.x - p.ox, ly = pt.y - p.oy;
    if constexpr (V % 2 == 0) {
      const int sx = p.rx + 2 * lx;
      if ((p.flags & kExact2x) && ly >= 0 && ly < p.dh && lx >= 0 && lx + V <= p.dw && (sx & 3) == 0 &&
          (p.pitch & 15) == 0 && (reinterpret_cast<uintptr_t>(p.src) & 15) == 0) {
        const int64_t y0 = p.ry + 2 * ly;
        const float4* r0 = reinterpret_cast<const float4*>(p.src + y0 * p.pitch) + 3 * sx / 4;
        const float4* r1 = reinterpret_cast<const float4*>(p.src + (y0 + 1) * p.pitch) + 3 * sx / 4;
        float a[6 * V], b[6 * V];  // 2 V source pixels x 3 channels of each row
#pragma unroll
        for (int i = 0; i < 3 * V / 2; ++i) {
          const float4 u = __ldg(r0 + i), w = __ldg(r1 + i);
          a[4 * i] = u.x, a[4 * i + 1] = u.y, a[4 * i + 2] = u.z, a[4 * i + 3] = u.w;
          b[4 * i] = w.x, b[4 * i + 1] = w.y, b[4 * i + 2] = w.z, b[4 * i + 3] = w.w;
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float left = __fadd_rn(__fmul_rn(0.5f, a[6 * k + c]), __fmul_rn(0.5f, b[6 * k + c]));
            const float right = __fadd_rn(__fmul_rn(0.5f, a[6 * k + 3 + c]), __fmul_rn(0.5f, b[6 * k + 3 + c]));
            const float o = __fadd_rn(__fmul_rn(0.5f, left), __fmul_rn(0.5f, right));
            out[k].v[c] = kUnit ? __fmul_rn(o, 255.f) : o;
          }
        }
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
  }
};
using ResizeF32C3 = ResizeF32C3T<false>;

// Packed float32 3-channel image, pixel for pixel (unfused per-op kernels).
struct ReadF32C3 {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = F3;
  static FKL_D F3 exec(const Point& pt, const ParamsType& p) {
    return ResizeF32C3::load(p, p.rx + pt.x, p.ry + pt.y);
  }
  // V pixels (12 V bytes) as 16-byte vectors when they start 16-byte aligned.
  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& p, F3 (&out)[V]) {
    const int sx = p.rx + pt.x;
    if constexpr (V % 4 == 0) {
      if ((sx & 3) == 0 && (p.pitch & 15) == 0 && (reinterpret_cast<uintptr_t>(p.src) & 15) == 0) {
        const float4* q =
            reinterpret_cast<const float4*>(p.src + static_cast<int64_t>(p.ry + pt.y) * p.pitch) + 3 * sx / 4;
        float f[3 * V];
#pragma unroll
        for (int i = 0; i < 3 * V / 4; ++i) {
          const float4 u = __ldcs(q + i);
          f[4 * i] = u.x, f[4 * i + 1] = u.y, f[4 * i + 2] = u.z, f[4 * i + 3] = u.w;
        }
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = F3{{f[3 * k], f[3 * k + 1], f[3 * k + 2]}};
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = exec(Point{pt.x + k, pt.y, pt.z}, p);
  }
};

// Packed u8 3-channel crop (integer chains): no resampling.
struct CropU8C3 {
  using InstanceType = ReadType;
  using ParamsType = ResampleParams;
  using OutputType = U3;
  static FKL_D U3 exec(const Point& pt, const ParamsType& p) {
    const uint8_t* q = p.src + static_cast<int64_t>(p.ry + pt.y) * p.pitch + 3 * (p.rx + pt.x);
    return U3{{__ldg(q), __ldg(q + 1), __ldg(q + 2)}};
  }
};

// Whether a read places its image in the output with a fill around it.
template <class R, class = void>
struct Placed : std::false_type {};
template <class R>
struct Placed<R, std::enable_if_t<R::kPlaced>> : std::true_type {};

// Horizontal fusion (paper §IV-B, BatchRead): an array of per-image params
// indexed by thread.z; `count` disables the unused entries.
template <class ROp, int CAP>
struct BatchRead {
  using InstanceType = ReadType;
  using OutputType = typename ROp::OutputType;
  using Op = ROp;
  struct ParamsType {
    int32_t count;
    int32_t _pad[3];
    typename ROp::ParamsType p[CAP];
  };

  static FKL_D OutputType exec(const Point& pt, const ParamsType& bp) {
    return ROp::exec(pt, bp.p[pt.z]);
  }

  // Whether the n outputs from pt are all the fill value of their image
  // (then `v` is that value): placing reads only.
  static FKL_D bool fill(const Point& pt, int n, const ParamsType& bp, OutputType& v) {
    if constexpr (Placed<ROp>::value && std::is_same_v<OutputType, F3>) {
      const ResampleParams& p = bp.p[pt.z];
      if (fill_span(p, pt.x, pt.y, n)) {
        v = F3{{p.pad, p.pad, p.pad}};
        return true;
      }
    }
    return false;
  }

  template <class R, int V, class = void>
  struct HasSpan : std::false_type {};
  template <class R, int V>
  struct HasSpan<R, V, std::void_t<decltype(&R::template exec_span<V>)>> : std::true_type {};

  template <int V>
  static FKL_D void exec_span(const Point& pt, const ParamsType& bp, OutputType (&out)[V]) {
    const typename ROp::ParamsType& p = bp.p[pt.z];
    if constexpr (HasSpan<ROp, V>::value) {
      ROp::template exec_span<V>(pt, p, out);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) out[k] = ROp::exec(Point{pt.x + k, pt.y, pt.z}, p);
    }
  }
};

// ===========================================================================
// Compute Operations
// ===========================================================================

// Two pixels' channels, one pixel per lane of a packed pair (f32x2): the
// form in which a DPP may run elementwise COps on Blackwell's packed FP32
// instructions. An Op that offers `exec_pair` computes exactly `exec` on
// each lane.
struct F3x2 {
  F2 v[3];
};
FKL_D F3x2 pack_pair(const F3& a, const F3& b) {
  return F3x2{{f2(a.v[0], b.v[0]), f2(a.v[1], b.v[1]), f2(a.v[2], b.v[2])}};
}
FKL_D void unpack_pair(const F3x2& p, F3& a, F3& b) {
#pragma unroll
  for (int c = 0; c < 3; ++c) f2split(p.v[c], a.v[c], b.v[c]);
}

// ColorConvert BGR <-> RGB: a register permutation.
template <class P>
struct SwapRB {
  using InstanceType = UnaryType;
  using InputType = P;
  using OutputType = P;
  static FKL_D P exec(const P& x) {
    P o = x;
    o.v[0] = x.v[2];
    o.v[2] = x.v[0];
    return o;
  }
  static FKL_D F3x2 exec_pair(const F3x2& x) { return F3x2{{x.v[2], x.v[1], x.v[0]}}; }
};

struct C3Params {
  float c[3];
};

struct Mul3 {
  using InstanceType = BinaryType;
  using InputType = F3;
  using OutputType = F3;
  using ParamsType = C3Params;
  static FKL_D F3 exec(const F3& x, const ParamsType& p) {
    return F3{{__fmul_rn(x.v[0], p.c[0]), __fmul_rn(x.v[1], p.c[1]), __fmul_rn(x.v[2], p.c[2])}};
  }
  static FKL_D F3x2 exec_pair(const F3x2& x, const ParamsType& p) {
    return F3x2{{f2mul(x.v[0], f2s(p.c[0])), f2mul(x.v[1], f2s(p.c[1])), f2mul(x.v[2], f2s(p.c[2]))}};
  }
};
struct Sub3 {
  using InstanceType = BinaryType;
  using InputType = F3;
  using OutputType = F3;
  using ParamsType = C3Params;
  static FKL_D F3 exec(const F3& x, const ParamsType& p) {
    return F3{{__fsub_rn(x.v[0], p.c[0]), __fsub_rn(x.v[1], p.c[1]), __fsub_rn(x.v[2], p.c[2])}};
  }
  // Per lane (scalar sub.rn): a packed subtract of the product of a packed
  // multiply (Mul3 before it) can be fused into one multiply-add by the
  // assembler, which would round once where the two ops round twice.
  static FKL_D F3x2 exec_pair(const F3x2& x, const ParamsType& p) {
    F3x2 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float a, b;
      f2split(x.v[c], a, b);
      o.v[c] = f2(__fsub_rn(a, p.c[c]), __fsub_rn(b, p.c[c]));
    }
    return o;
  }
};
// IEEE division. `on` = 0 passes the value through untouched (a chain
// without a Divide), which skips the cost of dividing by one.
struct Div3Params {
  float c[3];
  int32_t on;
};
struct Div3 {
  using InstanceType = BinaryType;
  using InputType = F3;
  using OutputType = F3;
  using ParamsType = Div3Params;
  static FKL_D F3 exec(const F3& x, const ParamsType& p) {
    if (!p.on) return x;
    return F3{{__fdiv_rn(x.v[0], p.c[0]), __fdiv_rn(x.v[1], p.c[1]), __fdiv_rn(x.v[2], p.c[2])}};
  }
};

struct I3Params {
  int32_t k[3];
};
// Saturating u8 add of an integer per channel: clamp(x + k, 0, 255).
struct AddSatU8 {
  using InstanceType = BinaryType;
  using InputType = U3;
  using OutputType = U3;
  using ParamsType = I3Params;
  static FKL_D U3 exec(const U3& x, const ParamsType& p) {
    U3 o;
#pragma unroll
    for (int c = 0; c < 3; ++c) o.v[c] = static_cast<uint8_t>(min(255, max(0, static_cast<int>(x.v[c]) + p.k[c])));
    return o;
  }
};

// ===========================================================================
// Write Operations
// ===========================================================================

// Output tensor of a batch of images: element (z, c, y, x) of a planar
// tensor lives at base + z*img + c*plane + y*pitch + x*bytes; a packed
// tensor uses (z, y, x, c) at base + z*img + y*pitch + (x*C + c)*bytes.
struct OutParams {
  uint8_t* base;
  int64_t img;
  int64_t plane;
  int64_t pitch;
  float scale_inv;  // FP8: the stored value is x * scale_inv
  int32_t aligned;  // 1: every run start is aligned for vector stores
  const float* scale_inv_dev;  // FP8: if set, scale_inv is read from here (dynamic scaling)
};

template <class OutT>
FKL_D float prescale(float x, const OutParams& p) {
  if constexpr (std::is_same_v<OutT, e4m3_t>) {
    const float inv = p.scale_inv_dev ? __ldg(p.scale_inv_dev) : p.scale_inv;
    return __fmul_rn(x, inv);
  }
  return x;
}

// Split (paper Fig. 9): packed pixel -> C planes.
template <class OutT, int C = 3>
struct WriteSplit {
  using InstanceType = WriteType;
  using InputType = Pix<float, C>;
  using ParamsType = OutParams;
  static constexpr int B = Format<OutT>::bytes;

  static FKL_D void exec(const Point& pt, const InputType& v, const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch + static_cast<int64_t>(pt.x) * B;
#pragma unroll
    for (int c = 0; c < C; ++c) store_one<OutT>(q + c * p.plane, prescale<OutT>(v.v[c], p));
  }

  // The parameters a thread writes with: a dynamic FP8 scale is read from
  // device memory once, when the thread starts, so that its latency overlaps
  // the thread's source loads instead of stalling the write.
  static FKL_D ParamsType prepare(const ParamsType& p) {
    ParamsType q = p;
    if constexpr (std::is_same_v<OutT, e4m3_t>) {
      if (q.scale_inv_dev) {
        q.scale_inv = __ldg(q.scale_inv_dev);
        q.scale_inv_dev = nullptr;
      }
    }
    return q;
  }

  // n <= V valid pixels starting at pt.x.
  template <int V>
  static FKL_D void exec_span(const Point& pt, int n, const InputType (&v)[V], const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch + static_cast<int64_t>(pt.x) * B;
    if (n == V && p.aligned) {
      if constexpr (std::is_same_v<OutT, e4m3_t> && V % 2 == 0) {
        // FP8 scaling two values per packed multiply (same bits as prescale)
        const float inv = p.scale_inv_dev ? __ldg(p.scale_inv_dev) : p.scale_inv;
        const F2 inv2 = f2s(inv);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float run[V];
#pragma unroll
          for (int k = 0; k < V; k += 2) f2split(f2mul(f2(v[k].v[c], v[k + 1].v[c]), inv2), run[k], run[k + 1]);
          store_run<OutT, V>(q + c * p.plane, run);
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float run[V];
#pragma unroll
          for (int k = 0; k < V; ++k) run[k] = prescale<OutT>(v[k].v[c], p);
          store_run<OutT, V>(q + c * p.plane, run);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        if (k < n) {
#pragma unroll
          for (int c = 0; c < C; ++c) store_one<OutT>(q + c * p.plane + k * B, prescale<OutT>(v[k].v[c], p));
        }
      }
    }
  }
};

// Packed store: C consecutive values per pixel.
template <class OutT, int C = 3>
struct WritePacked {
  using InstanceType = WriteType;
  using InputType = Pix<float, C>;
  using ParamsType = OutParams;
  static constexpr int B = Format<OutT>::bytes;

  static FKL_D void exec(const Point& pt, const InputType& v, const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch + static_cast<int64_t>(pt.x) * C * B;
#pragma unroll
    for (int c = 0; c < C; ++c) store_one<OutT>(q + c * B, prescale<OutT>(v.v[c], p));
  }
  template <int V>
  static FKL_D void exec_span(const Point& pt, int n, const InputType (&v)[V], const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch + static_cast<int64_t>(pt.x) * C * B;
    if constexpr ((V * C) % 4 == 0) {
      if (n == V && p.aligned) {
        float run[V * C];
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
          for (int c = 0; c < C; ++c) run[k * C + c] = prescale<OutT>(v[k].v[c], p);
        store_run<OutT, V * C>(q, run);
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      if (k < n) {
#pragma unroll
        for (int c = 0; c < C; ++c) store_one<OutT>(q + (k * C + c) * B, prescale<OutT>(v[k].v[c], p));
      }
    }
  }
};

// u8 outputs of the integer chains.
template <bool kSplit>
struct WriteU8C3 {
  using InstanceType = WriteType;
  using InputType = U3;
  using ParamsType = OutParams;
  static FKL_D void exec(const Point& pt, const U3& v, const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch;
    if constexpr (kSplit) {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c * p.plane + pt.x] = v.v[c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[3 * pt.x + c] = v.v[c];
    }
  }
  template <int V>
  static FKL_D void exec_span(const Point& pt, int n, const U3 (&v)[V], const ParamsType& p) {
    uint8_t* q = p.base + pt.z * p.img + pt.y * p.pitch;
    if constexpr (kSplit && V % 4 == 0) {
      if (n == V && p.aligned) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uint32_t w[V / 4];
#pragma unroll
          for (int i = 0; i < V / 4; ++i)
            w[i] = v[4 * i].v[c] | (v[4 * i + 1].v[c] << 8) | (v[4 * i + 2].v[c] << 16) |
                   (static_cast<uint32_t>(v[4 * i + 3].v[c]) << 24);
          store_words<V / 4>(q + c * p.plane + pt.x, w);
        }
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (k < n) exec(Point{pt.x + k, pt.y, pt.z}, v[k], p);
  }
};

}  // namespace fkl
