// The C ABI (include/fkl.h): chain parsing, argument validation, the table
// of compiled chain families, and the launch of fused and unfused forms.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "fkl/reduce.cuh"
#include "registry.h"

namespace fkl_impl {

namespace {

// The last error message of this thread: a fixed buffer, so that reporting a
// failure never allocates.
thread_local char t_error[512];

fkl_status fail(fkl_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(t_error, sizeof(t_error), fmt, ap);
  va_end(ap);
  return s;
}

fkl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FKL_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr int kMaxDim = 16384;

int dtype_bytes(int dt) {
  switch (dt) {
    case FKL_U8:
    case FKL_E4M3:
      return 1;
    case FKL_F16:
    case FKL_BF16:
      return 2;
    case FKL_F32:
      return 4;
    case FKL_U16:
      return 2;
    case FKL_F64:
      return 8;
    default:
      return 0;
  }
}

const char* dtype_name(int dt) {
  switch (dt) {
    case FKL_U8:
      return "u8";
    case FKL_F32:
      return "f32";
    case FKL_F16:
      return "f16";
    case FKL_BF16:
      return "bf16";
    case FKL_E4M3:
      return "e4m3";
    case FKL_U16:
      return "u16";
    case FKL_F64:
      return "f64";
    default:
      return "?";
  }
}

bool is_linear_read(int op) {
  return op == FKL_OP_READ_F32 || op == FKL_OP_READ_U8 || op == FKL_OP_READ_U16 || op == FKL_OP_READ_F64;
}
bool is_read(int op) { return op == FKL_OP_READ_U8C3 || op == FKL_OP_READ_NV12 || is_linear_read(op); }
bool is_write(int op) { return op == FKL_OP_WRITE_PACKED || op == FKL_OP_WRITE_SPLIT; }
bool is_modifier(int op) { return op == FKL_OP_CROP || op == FKL_OP_RESIZE || op == FKL_OP_LETTERBOX; }
bool is_compute(int op) {
  return op == FKL_OP_SWAP_RB || op == FKL_OP_MUL || op == FKL_OP_ADD || op == FKL_OP_SUB ||
         op == FKL_OP_DIV || op == FKL_OP_ADD_SAT_U8;
}

// Typed chains: READ_{U8,U16,F32,F64} [MUL] [ADD|SUB] [DIV] WRITE_PACKED(F32|F64|F16|BF16|E4M3).
fkl_status parse_typed(const fkl_op_desc* ops, int n, int src, Spec& s) {
  s.family = FAM_CAST;
  s.in_dtype = src == FKL_OP_READ_U8 ? FKL_U8 : src == FKL_OP_READ_U16 ? FKL_U16
               : src == FKL_OP_READ_F32 ? FKL_F32 : FKL_F64;
  if (ops[n - 1].op != FKL_OP_WRITE_PACKED || s.out_dtype == FKL_U8 || s.out_dtype == FKL_U16)
    return fail(FKL_ERR_UNSUPPORTED, "typed tensor chains write packed F32, F64, F16, BF16 or E4M3");
  int stage = 0;  // compiled order: MUL, ADD|SUB, DIV
  for (int k = 1; k < n - 1; ++k) {
    const fkl_op_desc& d = ops[k];
    int want;
    if (d.op == FKL_OP_MUL) {
      want = 1;
      s.has_mul = true;
      s.mul[0] = d.f[0];
    } else if (d.op == FKL_OP_ADD || d.op == FKL_OP_SUB) {
      want = 2;
      s.has_sub = true;
      s.sub[0] = d.op == FKL_OP_SUB ? d.f[0] : -d.f[0];  // x + c == x - (-c), bit for bit
    } else if (d.op == FKL_OP_DIV) {
      want = 3;
      s.has_div = true;
      s.div[0] = d.f[0];
    } else if (is_modifier(d.op)) {
      return fail(FKL_ERR_INVALID, "op %d: read modifiers apply to image reads only", k);
    } else {
      return fail(FKL_ERR_UNSUPPORTED, "op %d: typed tensor chains take [MUL] [ADD|SUB] [DIV]", k);
    }
    if (want <= stage)
      return fail(FKL_ERR_UNSUPPORTED, "op %d: typed tensor chains take MUL, then ADD|SUB, then DIV", k);
    stage = want;
  }
  return FKL_OK;
}

// ROp -> COp* -> WOp grammar, then the compiled-family table.
fkl_status parse(const fkl_op_desc* ops, int n, Spec& s) {
  if (n < 2) return fail(FKL_ERR_INVALID, "a chain needs at least a read and a write op (got %d ops)", n);
  const int src = ops[0].op;
  const int wop = ops[n - 1].op;
  if (!is_read(src)) return fail(FKL_ERR_INVALID, "op 0 must be a READ_* op (got code %d)", src);
  if (!is_write(wop)) return fail(FKL_ERR_INVALID, "the last op must be a WRITE_* op (got code %d)", wop);
  for (int k = 1; k < n - 1; ++k) {
    const int op = ops[k].op;
    if (is_read(op)) return fail(FKL_ERR_INVALID, "op %d: a read op may only come first", k);
    if (is_write(op)) return fail(FKL_ERR_INVALID, "op %d: a write op may only come last", k);
    if (!is_modifier(op) && !is_compute(op)) return fail(FKL_ERR_INVALID, "op %d: unknown op code %d", k, op);
  }
  const int odt = ops[n - 1].i[0];
  if (dtype_bytes(odt) == 0) return fail(FKL_ERR_INVALID, "write op: unknown dtype %d", odt);
  s.split = wop == FKL_OP_WRITE_SPLIT;
  s.out_dtype = odt;
  if (odt == FKL_E4M3) {
    const float sc = ops[n - 1].f[0];
    if (!(sc > 0.f) || !std::isfinite(sc))
      return fail(FKL_ERR_INVALID, "E4M3 output needs a finite per-tensor scale > 0 in f[0]");
    s.fp8_scale = sc;
  }

  if (is_linear_read(src)) {
    bool mul_add_only = true;
    for (int k = 1; k < n - 1; ++k) {
      if (is_modifier(ops[k].op)) return fail(FKL_ERR_INVALID, "op %d: read modifiers apply to image reads only", k);
      mul_add_only = mul_add_only && (ops[k].op == FKL_OP_MUL || ops[k].op == FKL_OP_ADD);
    }
    const bool vertical = (src == FKL_OP_READ_F32 || src == FKL_OP_READ_U8) && mul_add_only &&
                          wop == FKL_OP_WRITE_PACKED && odt == FKL_F32;
    if (!vertical) return parse_typed(ops, n, src, s);
    s.family = FAM_VCHAIN;
    s.vinput_u8 = src == FKL_OP_READ_U8;
    for (int k = 1; k < n - 1; ++k) {
      const int op = ops[k].op;
      if (op == FKL_OP_MUL || op == FKL_OP_ADD) {
        s.vkinds.push_back(op == FKL_OP_ADD ? 1 : 0);
        s.vconsts.push_back(ops[k].f[0]);
      } else if (is_modifier(op)) {
        return fail(FKL_ERR_INVALID, "op %d: read modifiers apply to image reads only", k);
      } else {
        return fail(FKL_ERR_UNSUPPORTED, "op %d: float32 tensor chains take MUL and ADD only", k);
      }
    }
    if (wop != FKL_OP_WRITE_PACKED || odt != FKL_F32)
      return fail(FKL_ERR_UNSUPPORTED, "float32 tensor chains write packed F32 only");
    if (s.vkinds.size() > 65536) return fail(FKL_ERR_UNSUPPORTED, "vertical chains are limited to 65536 ops");
    return FKL_OK;
  }

  int k = 1;
  if (ops[k].op == FKL_OP_CROP) {
    const int32_t* c = ops[k].i;
    if (c[0] < 0 || c[1] < 0 || c[2] <= 0 || c[3] <= 0 || c[2] > kMaxDim || c[3] > kMaxDim)
      return fail(FKL_ERR_INVALID, "CROP (%d,%d,%d,%d): need x, y >= 0 and 0 < w, h <= %d", c[0], c[1], c[2], c[3], kMaxDim);
    s.has_crop = true;
    std::memcpy(s.crop, c, sizeof(s.crop));
    ++k;
  }
  if (ops[k].op == FKL_OP_RESIZE || ops[k].op == FKL_OP_LETTERBOX) {
    s.geom = ops[k].op == FKL_OP_RESIZE ? GEOM_RESIZE : GEOM_LETTERBOX;
    s.out_w = ops[k].i[0];
    s.out_h = ops[k].i[1];
    if (s.out_w <= 0 || s.out_h <= 0 || s.out_w > kMaxDim || s.out_h > kMaxDim)
      return fail(FKL_ERR_INVALID, "RESIZE/LETTERBOX size %dx%d outside 1..%d", s.out_w, s.out_h, kMaxDim);
    s.pad = s.geom == GEOM_LETTERBOX ? ops[k].f[0] : 0.f;
    ++k;
  }
  int stage = 0;  // compiled order: SWAP_RB, MUL, ADD|SUB, DIV, ADD_SAT_U8
  for (; k < n - 1; ++k) {
    const fkl_op_desc& d = ops[k];
    int want;
    switch (d.op) {
      case FKL_OP_SWAP_RB:
        want = 1;
        s.swap = true;
        break;
      case FKL_OP_MUL:
        want = 2;
        s.has_mul = true;
        std::memcpy(s.mul, d.f, sizeof(s.mul));
        break;
      case FKL_OP_ADD:
      case FKL_OP_SUB:
        want = 3;
        s.has_sub = true;
        for (int c = 0; c < 3; ++c) s.sub[c] = d.op == FKL_OP_SUB ? d.f[c] : -d.f[c];
        break;
      case FKL_OP_DIV:
        want = 4;
        s.has_div = true;
        std::memcpy(s.div, d.f, sizeof(s.div));
        break;
      case FKL_OP_ADD_SAT_U8:
        want = 5;
        s.has_addsat = true;
        std::memcpy(s.addsat, d.i, sizeof(s.addsat));
        break;
      default:
        return fail(FKL_ERR_INVALID, "op %d: read modifiers must directly follow the read op", k);
    }
    if (want <= stage)
      return fail(FKL_ERR_UNSUPPORTED,
                  "op %d: no compiled chain has this op order (compiled: SWAP_RB, MUL, ADD|SUB, DIV, ADD_SAT_U8)", k);
    stage = want;
  }
  const bool float_ops = s.has_mul || s.has_sub || s.has_div;
  if (s.has_addsat || odt == FKL_U8) {
    if (src != FKL_OP_READ_U8C3 || s.geom != GEOM_NONE || float_ops || odt != FKL_U8)
      return fail(FKL_ERR_UNSUPPORTED, "u8 chains are READ_U8C3 [CROP] [SWAP_RB] [ADD_SAT_U8] WRITE_* (U8)");
    s.family = FAM_INT;
    return FKL_OK;
  }
  s.family = src == FKL_OP_READ_U8C3 ? FAM_PACKED : FAM_NV12;
  if (odt == FKL_U16 || odt == FKL_F64)
    return fail(FKL_ERR_UNSUPPORTED, "image chains write U8, F32, F16, BF16 or E4M3");
  if (!s.split && odt != FKL_F32) return fail(FKL_ERR_UNSUPPORTED, "packed float outputs are F32 only");
  return FKL_OK;
}

// ------------------------------------------------------------------ tensors

struct OutDesc {
  fkl::OutParams p;
  int N, H, W;
};

fkl_status check_out(const Spec& s, const fkl_tensor* t, int n, OutDesc& o) {
  if (!t || !t->data) return fail(FKL_ERR_INVALID, "output tensor missing");
  if (t->dtype != s.out_dtype)
    return fail(FKL_ERR_INVALID, "output dtype %s, chain writes %s", dtype_name(t->dtype), dtype_name(s.out_dtype));
  const int B = dtype_bytes(s.out_dtype);
  int64_t N, H, W, C;
  if (s.split) {
    if (t->layout != FKL_LAYOUT_NCHW) return fail(FKL_ERR_INVALID, "WRITE_SPLIT needs an NCHW output");
    N = t->dims[0];
    C = t->dims[1];
    H = t->dims[2];
    W = t->dims[3];
  } else {
    if (t->layout != FKL_LAYOUT_NHWC) return fail(FKL_ERR_INVALID, "WRITE_PACKED needs an NHWC output");
    N = t->dims[0];
    H = t->dims[1];
    W = t->dims[2];
    C = t->dims[3];
  }
  if (C != 3) return fail(FKL_ERR_INVALID, "output must have 3 channels (got %lld)", (long long)C);
  if (N < n) return fail(FKL_ERR_INVALID, "output holds %lld images, batch has %d", (long long)N, n);
  if (H <= 0 || W <= 0 || H > kMaxDim || W > kMaxDim)
    return fail(FKL_ERR_INVALID, "output size %lldx%lld outside 1..%d", (long long)W, (long long)H, kMaxDim);
  if (s.geom != GEOM_NONE && (H != s.out_h || W != s.out_w))
    return fail(FKL_ERR_INVALID, "output is %lldx%lld, chain resizes to %dx%d", (long long)W, (long long)H, s.out_w, s.out_h);
  const int64_t row = s.split ? W * B : W * 3 * B;
  const int64_t pitch = t->pitch_bytes ? t->pitch_bytes : row;
  if (pitch < row) return fail(FKL_ERR_INVALID, "output pitch %lld < row bytes %lld", (long long)pitch, (long long)row);
  std::memset(&o, 0, sizeof(o));
  o.p.base = static_cast<uint8_t*>(t->data);
  o.p.pitch = pitch;
  o.p.plane = H * pitch;
  o.p.img = s.split ? 3 * H * pitch : H * pitch;
  o.p.scale_inv = s.out_dtype == FKL_E4M3 ? static_cast<float>(1.0 / s.fp8_scale) : 1.f;
  o.p.aligned = (reinterpret_cast<uintptr_t>(t->data) % 16 == 0 && pitch % 16 == 0) ? 1 : 0;
  o.N = static_cast<int>(N);
  o.H = static_cast<int>(H);
  o.W = static_cast<int>(W);
  return FKL_OK;
}

// Per-image ROp parameters from the input tensor, the ROI and the geometry.
fkl_status image_params(const Spec& s, const fkl_tensor* t, const int32_t* roi_in, int i,
                        const OutDesc& od, fkl::ResampleParams& r) {
  if (!t || !t->data) return fail(FKL_ERR_INVALID, "input %d missing", i);
  if (t->dtype != FKL_U8) return fail(FKL_ERR_INVALID, "input %d: image sources are U8", i);
  int64_t H, W, row;
  if (s.family == FAM_NV12) {
    if (t->layout != FKL_LAYOUT_NV12) return fail(FKL_ERR_INVALID, "input %d: READ_NV12 needs an NV12 tensor", i);
    H = t->dims[0];
    W = t->dims[1];
    if (H % 2 || W % 2) return fail(FKL_ERR_INVALID, "input %d: NV12 needs even width and height", i);
    row = W;
  } else {
    if (t->layout != FKL_LAYOUT_HWC || t->dims[2] != 3)
      return fail(FKL_ERR_INVALID, "input %d: READ_U8C3 needs an HWC tensor with 3 channels", i);
    H = t->dims[0];
    W = t->dims[1];
    row = 3 * W;
  }
  if (H <= 0 || W <= 0 || H > kMaxDim || W > kMaxDim)
    return fail(FKL_ERR_INVALID, "input %d: size %lldx%lld outside 1..%d", i, (long long)W, (long long)H, kMaxDim);
  const int64_t pitch = t->pitch_bytes ? t->pitch_bytes : row;
  if (pitch < row || pitch > (int64_t(1) << 30))
    return fail(FKL_ERR_INVALID, "input %d: pitch %lld invalid for rows of %lld bytes", i, (long long)pitch, (long long)row);
  int32_t roi[4] = {0, 0, static_cast<int32_t>(W), static_cast<int32_t>(H)};
  if (roi_in) {
    std::memcpy(roi, roi_in + 4 * i, sizeof(roi));
  } else if (s.has_crop) {
    std::memcpy(roi, s.crop, sizeof(roi));
  }
  if (roi[0] < 0 || roi[1] < 0 || roi[2] <= 0 || roi[3] <= 0 || roi[0] + int64_t(roi[2]) > W ||
      roi[1] + int64_t(roi[3]) > H)
    return fail(FKL_ERR_INVALID, "input %d: ROI (%d,%d,%d,%d) not inside the %lldx%lld image", i, roi[0], roi[1],
                roi[2], roi[3], (long long)W, (long long)H);
  std::memset(&r, 0, sizeof(r));
  r.src = static_cast<const uint8_t*>(t->data);
  r.uv = s.family == FAM_NV12 ? r.src + H * pitch : nullptr;
  r.pitch = static_cast<int32_t>(pitch);
  r.rx = roi[0];
  r.ry = roi[1];
  r.rw = roi[2];
  r.rh = roi[3];
  if (s.geom == GEOM_NONE && (r.rw != od.W || r.rh != od.H))
    return fail(FKL_ERR_INVALID, "input %d: ROI %dx%d must equal the %dx%d output when the chain has no resize", i,
                r.rw, r.rh, od.W, od.H);
  place(s, od.W, od.H, r);
  if (s.family == FAM_NV12 && (r.flags & fkl::kExact2x) && r.rx % 16 == 0 && r.ry % 2 == 0 &&
      pitch % 16 == 0 && reinterpret_cast<uintptr_t>(r.src) % 16 == 0)
    r.flags |= fkl::kFast2x;
  return FKL_OK;
}

std::mutex g_sm_mu;
int g_sm[64] = {0};

}  // namespace

void place(const Spec& s, int out_w, int out_h, fkl::ResampleParams& r) {
  if (s.geom == GEOM_NONE) {
    r.dw = r.rw;
    r.dh = r.rh;
  } else if (s.geom == GEOM_RESIZE) {
    r.dw = out_w;
    r.dh = out_h;
  } else {
    const double sc = std::min(static_cast<double>(out_w) / r.rw, static_cast<double>(out_h) / r.rh);
    r.dw = std::max(1, std::min(out_w, static_cast<int>(std::floor(r.rw * sc + 0.5))));
    r.dh = std::max(1, std::min(out_h, static_cast<int>(std::floor(r.rh * sc + 0.5))));
    r.ox = (out_w - r.dw) / 2;
    r.oy = (out_h - r.dh) / 2;
  }
  r.pad = s.pad;
  r.inv_area = static_cast<float>(1.0 / (4.0 * r.dw * r.dh));
  if (r.rw == 2 * r.dw && r.rh == 2 * r.dh) r.flags |= fkl::kExact2x;
}

void set_last_error(const char* msg) { std::snprintf(t_error, sizeof(t_error), "%s", msg ? msg : ""); }

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(g_sm_mu);
  if (g_sm[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    g_sm[dev] = v;
  }
  return g_sm[dev];
}

namespace {
const int kBlocks[][2] = {{8, 16}, {16, 8}, {16, 16}, {32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1}, {128, 2}};
// Row-staged NV12 shapes {threads, rows per job, stages}: the fastest of a
// 24-point sweep (threads 128/256, rows 2/4/8, stages 2/3/4/6) on 256 frames
// 1280x720 -> 640x640; deeper rings and longer jobs only lowered occupancy.
const int kStaged[][3] = {{128, 4, 2}, {128, 2, 2}, {128, 4, 3}, {256, 8, 2}};
// Tile-staged packed shapes {threads x, threads y}: tiles of (x * vec) x y outputs.
const int kTiles[][2] = {{16, 8}, {32, 8}, {16, 16}, {32, 4}, {8, 16}};
}
// ---------------------------------------------------------------------------
// Scratch for fkl_execute_batch_unfused_static: a fixed device array that
// every GPU loading this library holds until the process exits. Host code
// must not pass `g_unfused_scratch` itself to a kernel (on the host that name
// is only a stand-in); it asks the runtime for the device address instead.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) uint8_t g_unfused_scratch[kStaticScratchBytes];

// Set to 1 by a bounded device wait that gave up (fkl_device_check).
static __device__ int g_device_error;

namespace {
constexpr unsigned long long kDefaultWaitNs = 1000ull * 1000 * 1000;  // 1 s
constexpr unsigned long long kMaxWaitNs = 10ull * kDefaultWaitNs;
std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
}  // namespace

unsigned long long device_wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

namespace {
std::mutex g_scratch_mu;
void* g_error_ptr[64] = {nullptr};
void* g_scratch_ptr[64] = {nullptr};

// Device address of g_unfused_scratch on the current device, looked up once
// per device (the lookup also loads this library's module on that device).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_unfused_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t device_error_flag(int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_error_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_device_error);
    if (e != cudaSuccess) return e;
    g_error_ptr[dev] = ptr;
  }
  *out = static_cast<int*>(g_error_ptr[dev]);
  return cudaSuccess;
}


std::vector<fkl_launch_shape> shapes_for(const Spec& s) {
  std::vector<int> vecs;
  if (s.family == FAM_CAST) {  // {elements per thread, threads, 1, 1}
    std::vector<fkl_launch_shape> out;
    for (int v : {8, 16})
      for (int tx : {128, 256}) out.push_back(fkl_launch_shape{v, tx, 1, 1});
    return out;
  }
  if (s.family == FAM_INT) {
    vecs = {16};
  } else if (s.family == FAM_PACKED || s.family == FAM_NV12) {
    const bool packed = s.family == FAM_PACKED;  // the packed reader also runs 1-2 pixels per thread
    if (s.out_dtype == FKL_F32)
      vecs = !s.split ? std::vector<int>{4} : packed ? std::vector<int>{1, 2, 4, 8} : std::vector<int>{4, 8};
    else if (packed && (s.out_dtype == FKL_F16 || s.out_dtype == FKL_BF16))
      vecs = {2, 8, 16};
    else
      vecs = {8, 16};
  } else {
    std::vector<fkl_launch_shape> out;
    // 2 or 4 elements per thread spread a small tensor over more warps: an
    // ALU-bound chain ends when the most loaded warp scheduler (4 per SM)
    // does, so finer warps balance better
    for (int v : {2, 4, 8, 16, 32})
      for (int tx : {128, 256, 512})
        for (int ry : {1, 0}) out.push_back(fkl_launch_shape{v, tx, 1, ry});
    return out;
  }
  std::vector<fkl_launch_shape> out;
  for (int v : vecs)
    for (int ry : {1, 2}) {
      if (v > 8 && ry > 1) continue;  // not compiled (register budget)
      for (const auto& b : kBlocks) out.push_back(fkl_launch_shape{v, b[0], b[1], ry});
    }
  if (s.family == FAM_PACKED)  // tile-staged packed reader: {vec, tile threads x, y, -1}
    for (int v : vecs) {
      if (v > 4) continue;
      for (const auto& b : kTiles) out.push_back(fkl_launch_shape{v, b[0], b[1], -1});
    }
  if (s.family == FAM_NV12 && s.split)  // row-staged kernel: {vec, threads, rows per job, -stages}
    for (int v : vecs) {
      if (v % 8) continue;
      for (const auto& st : kStaged) out.push_back(fkl_launch_shape{v, st[0], st[1], -st[2]});
    }
  return out;
}

fkl_launch_shape default_shape(const Spec& s) {
  if (s.family == FAM_INT) return {16, 16, 8, 1};
  if (s.family == FAM_VCHAIN) return {16, 256, 1, 1};
  if (s.family == FAM_CAST) return {8, 256, 1, 1};
  return {s.out_dtype == FKL_F32 ? 4 : 8, 16, 8, 1};
}

}  // namespace fkl_impl

using namespace fkl_impl;

namespace {

std::string make_name(const Spec& s) {
  std::string n = "fused:";
  switch (s.family) {
    case FAM_PACKED:
      n += "ResizeU8C3";
      break;
    case FAM_NV12:
      n += "ResizeNV12";
      break;
    case FAM_INT:
      n += "CropU8C3";
      break;
    case FAM_VCHAIN:
      n += "ReadF32";
      break;
    case FAM_CAST:
      n = std::string("fused:Read<") + dtype_name(s.in_dtype) + ">>Cast<" + dtype_name(s.out_dtype) + ">";
      if (s.has_mul) n += ">Mul";
      if (s.has_sub) n += ">Sub";
      if (s.has_div) n += ">Div";
      return n + ">Write<" + dtype_name(s.out_dtype) + ">";
  }
  if (s.family == FAM_VCHAIN) {
    if (s.vinput_u8) n = "fused:ReadU8";
    n += ">(Mul|Add)x" + std::to_string(s.vkinds.size()) + ">WriteF32";
    return n;
  }
  if (s.swap) n += ">SwapRB";
  if (s.family == FAM_INT) {
    n += ">AddSatU8>WriteU8";
  } else {
    n += ">Mul>Sub>Div";
    n += s.split ? ">WriteSplit<" : ">WritePacked<";
    n += dtype_name(s.out_dtype);
    n += ">";
  }
  return n;
}

cudaError_t launch_family(const LaunchCtx& c) {
  const Spec& s = *c.spec;
  if (s.family == FAM_INT) return launch_int(c);
  const bool packed = s.family == FAM_PACKED;
  switch (s.out_dtype) {
    case FKL_F32:
      return packed ? launch_packed_f32(c) : launch_nv12_f32(c);
    case FKL_F16:
      return packed ? launch_packed_f16(c) : launch_nv12_f16(c);
    case FKL_BF16:
      return packed ? launch_packed_bf16(c) : launch_nv12_bf16(c);
    case FKL_E4M3:
      return packed ? launch_packed_e4m3(c) : launch_nv12_e4m3(c);
    default:
      return cudaErrorInvalidValue;
  }
}

// Tensor chains (vertical and typed): n LINEAR inputs of the read's type and
// one length, one LINEAR output of n * length elements of the write's type
// (tensor i at elements [i * length, (i + 1) * length)).
fkl_status check_linear(const Spec& s, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                        const fkl_tensor* out, int64_t& len) {
  const int in_dt = s.family == FAM_CAST ? s.in_dtype : (s.vinput_u8 ? FKL_U8 : FKL_F32);
  const int out_dt = s.family == FAM_CAST ? s.out_dtype : FKL_F32;
  if (n < 0) return fail(FKL_ERR_INVALID, "negative batch size");
  if (rois) return fail(FKL_ERR_INVALID, "tensor chains take no ROIs");
  if (n > 0 && !ins) return fail(FKL_ERR_INVALID, "inputs missing");
  if (!out) return fail(FKL_ERR_INVALID, "output tensor missing");
  if (out->layout != FKL_LAYOUT_LINEAR || out->dtype != out_dt)
    return fail(FKL_ERR_INVALID, "tensor chains need a LINEAR %s output", dtype_name(out_dt));
  len = n > 0 ? ins[0].dims[0] : 0;
  for (int i = 0; i < n; ++i) {
    const fkl_tensor& t = ins[i];
    if (t.layout != FKL_LAYOUT_LINEAR || t.dtype != in_dt)
      return fail(FKL_ERR_INVALID, "input %d must be LINEAR %s", i, dtype_name(in_dt));
    if (t.dims[0] != len || len < 0)
      return fail(FKL_ERR_INVALID, "input %d has %lld elements, input 0 has %lld", i, (long long)t.dims[0],
                  (long long)len);
    if (!t.data && len > 0) return fail(FKL_ERR_INVALID, "input %d: data is NULL", i);
  }
  if (len > (int64_t(1) << 40) || out->dims[0] != int64_t(n) * len)
    return fail(FKL_ERR_INVALID, "output must hold n x length = %lld elements (has %lld)",
                (long long)(int64_t(n) * len), (long long)out->dims[0]);
  if (!out->data && n * len > 0) return fail(FKL_ERR_INVALID, "output tensor missing");
  return FKL_OK;
}

// Device workspace of the unfused form of a tensor chain: a float32 copy of
// one tensor for typed chains writing F16/BF16/E4M3, nothing otherwise.
size_t linear_workspace_bytes(const Spec& s, int64_t len) {
  const bool narrow = s.family == FAM_CAST && s.out_dtype != FKL_F32 && s.out_dtype != FKL_F64;
  return narrow ? static_cast<size_t>((len * 4 + 255) / 256 * 256) : 0;
}

// Runs a validated tensor chain (check_linear gave `len`): typed chains in
// one launch per 256 tensors, vertical chains one launch per tensor (and per
// 4096 ops); unfused: one kernel per op, with `ws` (linear_workspace_bytes)
// when the chain needs one. The input pointers travel in a stack array of
// one launch's tensors, so the call allocates no host memory.
constexpr int kLinearChunk = 256;  // tensors per typed-chain launch

fkl_status run_linear(fkl_pipeline p, int32_t n, const fkl_tensor* ins, fkl_tensor* out, int64_t len,
                      bool unfused, void* stream, void* ws = nullptr, size_t ws_bytes = 0) {
  if (n == 0 || len == 0) return FKL_OK;
  const size_t need = unfused ? linear_workspace_bytes(p->spec, len) : 0;
  if (need && (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256))
    return fail(FKL_ERR_INVALID, "workspace must be >= %zu bytes and 256-byte aligned", need);
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int64_t esz = dtype_bytes(out->dtype);
  const void* ptrs[kLinearChunk];
  cudaError_t e = cudaSuccess;
  for (int start = 0; start < n && e == cudaSuccess; start += kLinearChunk) {
    const int m = std::min(kLinearChunk, n - start);
    for (int i = 0; i < m; ++i) ptrs[i] = ins[start + i].data;
    uint8_t* o = static_cast<uint8_t*>(out->data) + start * len * esz;
    if (p->spec.family == FAM_CAST) {
      e = unfused ? launch_unfused_cast(p->spec, m, ptrs, o, len, ws, cs)
                  : launch_cast(p->spec, p->shape, m, ptrs, o, len, cs);
    } else {
      for (int i = 0; i < m && e == cudaSuccess; ++i) {
        float* oi = reinterpret_cast<float*>(o) + i * len;
        e = unfused ? launch_unfused_vchain(p->spec, ptrs[i], oi, len, cs)
                    : launch_vchain(p->spec, p->shape, ptrs[i], oi, len, cs);
      }
    }
  }
  return e == cudaSuccess ? FKL_OK : cuda_fail(e, unfused ? "unfused launch" : "tensor chain launch");
}

// check_linear, then run_linear.
fkl_status exec_linear(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois, fkl_tensor* out,
                       bool unfused, void* stream, void* ws = nullptr, size_t ws_bytes = 0) {
  int64_t len = 0;
  const fkl_status st = check_linear(p->spec, n, ins, rois, out, len);
  if (st != FKL_OK) return st;
  return run_linear(p, n, ins, out, len, unfused, stream, ws, ws_bytes);
}

bool is_tensor_chain(const Spec& s) { return s.family == FAM_VCHAIN || s.family == FAM_CAST; }

// Sizing of the unfused image chains' intermediates, shared by every unfused
// entry point: each intermediate holds one image's pixels, packed (3 bytes
// per pixel in the integer chains, 3 float32 otherwise), at the output size,
// or for NV12 chains at least the source window (the decode runs at full
// resolution); slots are rounded up to 256 bytes.
int64_t unfused_min_px(const OutDesc& od) { return static_cast<int64_t>(od.H) * od.W; }
int64_t unfused_image_px(const Spec& s, const OutDesc& od, const fkl::ResampleParams& r) {
  const int64_t px = unfused_min_px(od);
  return s.family == FAM_NV12 ? std::max<int64_t>(px, static_cast<int64_t>(r.rw) * r.rh) : px;
}
int64_t unfused_slot_bytes(const Spec& s, int64_t px) {
  const int64_t elem = s.family == FAM_INT ? 3 : 12;
  return (px * elem + 255) / 256 * 256;
}

fkl_status validate_batch(const fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                          const fkl_tensor* out, OutDesc& od, std::vector<fkl::ResampleParams>& imgs) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (is_tensor_chain(p->spec)) return fail(FKL_ERR_INVALID, "tensor chains take LINEAR tensors");
  if (n < 0) return fail(FKL_ERR_INVALID, "negative batch size");
  if (n > 0 && !ins) return fail(FKL_ERR_INVALID, "inputs missing");
  fkl_status st = check_out(p->spec, out, n, od);
  if (st != FKL_OK) return st;
  try {
    imgs.resize(n);
  } catch (...) {
    return fail(FKL_ERR_OOM, "host allocation failed");
  }
  for (int i = 0; i < n; ++i) {
    st = image_params(p->spec, &ins[i], rois, i, od, imgs[i]);
    if (st != FKL_OK) return st;
  }
  return FKL_OK;
}

}  // namespace

namespace {

// fkl_execute_batch with an optional device-side FP8 scale.
fkl_status execute_batch_impl(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                              fkl_tensor* out, const float* scale_inv_dev, void* stream) {
  if (p && is_tensor_chain(p->spec)) return exec_linear(p, n, ins, rois, out, false, stream);
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  fkl_status st = validate_batch(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  od.p.scale_inv_dev = scale_inv_dev;
  int* err_flag = nullptr;
  if (n > 0 && p->shape.ry <= 0 && p->spec.family == FAM_NV12) {
    const cudaError_t e = device_error_flag(&err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "device flag lookup");
  }
  for (int start = 0; start < n; start += kBatchCap) {
    LaunchCtx c;
    c.spec = &p->spec;
    c.shape = p->shape;
    c.imgs = imgs.data() + start;
    c.n = std::min(kBatchCap, n - start);
    c.out = od.p;
    c.out.base += start * od.p.img;
    c.H = od.H;
    c.W = od.W;
    c.stream = static_cast<cudaStream_t>(stream);
    c.all_exact2x = true;
    for (int i = 0; i < c.n; ++i) c.all_exact2x = c.all_exact2x && (c.imgs[i].flags & fkl::kExact2x);
    c.device_error = err_flag;
    c.wait_ns = device_wait_limit_ns();
    const cudaError_t e = launch_family(c);
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  }
  return FKL_OK;
}

}  // namespace

extern "C" {

fkl_status fkl_pipeline_create(const fkl_op_desc* ops, int32_t n_ops, fkl_pipeline* out) {
  if (!out) return fail(FKL_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ops) return fail(FKL_ERR_INVALID, "ops is NULL");
  Spec s;
  try {
    const fkl_status st = parse(ops, n_ops, s);
    if (st != FKL_OK) return st;
    auto* p = new (std::nothrow) fkl_pipeline_s;
    if (!p) return fail(FKL_ERR_OOM, "host allocation failed");
    p->spec = std::move(s);
    p->shape = default_shape(p->spec);
    p->name = make_name(p->spec);
    *out = p;
  } catch (const std::bad_alloc&) {
    return fail(FKL_ERR_OOM, "host allocation failed");
  }
  return FKL_OK;
}

void fkl_pipeline_destroy(fkl_pipeline p) { delete p; }

const char* fkl_last_error(void) { return t_error; }

fkl_status fkl_set_device_wait_limit(uint64_t ns) {
  if (ns > kMaxWaitNs) return fail(FKL_ERR_INVALID, "wait limit above 10 s");
  g_wait_ns.store(ns ? ns : kDefaultWaitNs, std::memory_order_relaxed);
  return FKL_OK;
}

fkl_status fkl_device_check(void) {
  int* flag = nullptr;
  cudaError_t e = device_error_flag(&flag);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(flag, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "device check");
  if (v) return fail(FKL_ERR_TIMEOUT, "a bounded device wait gave up; outputs of that launch are incomplete");
  return FKL_OK;
}

const char* fkl_version(void) { return "fkl-gb300 0.1 (sm_103a)"; }

const char* fkl_pipeline_kernel_name(fkl_pipeline p) { return p ? p->name.c_str() : ""; }

fkl_status fkl_execute_batch(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                             fkl_tensor* out, void* stream) {
  return execute_batch_impl(p, n, ins, rois, out, nullptr, stream);
}

fkl_status fkl_execute_batch_mapped(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                    fkl_tensor* out, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (n < 0 || (n > 0 && !ins) || !out) return fail(FKL_ERR_INVALID, "bad batch arguments");
  // the device address of a pinned host or device buffer; pageable memory is refused
  auto device_address = [](void* ptr, void** dev, const char* what, int i) -> fkl_status {
    if (!ptr) {
      *dev = nullptr;
      return FKL_OK;
    }
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) return cuda_fail(e, "pointer attributes");
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
      *dev = ptr;
      return FKL_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
      *dev = a.devicePointer;
      return FKL_OK;
    }
    return fail(FKL_ERR_INVALID, "%s %d: not pinned host memory or device memory", what, i);
  };
  std::vector<fkl_tensor> dins;
  try {
    dins.assign(ins, ins + n);
  } catch (...) {
    return fail(FKL_ERR_OOM, "host allocation failed");
  }
  for (int i = 0; i < n; ++i) {
    const fkl_status st = device_address(ins[i].data, &dins[i].data, "input", i);
    if (st != FKL_OK) return st;
  }
  fkl_tensor dout = *out;
  const fkl_status st = device_address(out->data, &dout.data, "output", 0);
  if (st != FKL_OK) return st;
  return fkl_execute_batch(p, n, dins.data(), rois, &dout, stream);
}

fkl_status fkl_execute_batch_scaled(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                    fkl_tensor* out, const float* scale_inv_dev, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (p->spec.out_dtype != FKL_E4M3) return fail(FKL_ERR_INVALID, "scaled execution needs an E4M3 output");
  if (!scale_inv_dev) return fail(FKL_ERR_INVALID, "scale pointer missing");
  return execute_batch_impl(p, n, ins, rois, out, scale_inv_dev, stream);
}

fkl_status fkl_reduce_batch(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                            const fkl_tensor* out, float* stats, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (p->spec.family != FAM_PACKED && p->spec.family != FAM_NV12)
    return fail(FKL_ERR_UNSUPPORTED, "reductions run on float image chains");
  if (!stats || reinterpret_cast<uintptr_t>(stats) % 16) return fail(FKL_ERR_INVALID, "stats must be 16-byte aligned");
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  fkl_status st = validate_batch(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* acc = reinterpret_cast<fkl::ReduceAcc*>(reinterpret_cast<uint8_t*>(stats) + 64);
  static_assert(sizeof(fkl::ReduceAcc) <= 64, "accumulator fits the stats buffer");
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(fkl::ReduceAcc), s);
  double fill = 0.0;  // output pixels outside the placed windows: the pad value
  for (const auto& r : imgs) fill += static_cast<double>(od.H) * od.W - static_cast<double>(r.dw) * r.dh;
  // every chunk's launch is sized first: the block that completes the
  // blocks of all of them writes the statistics
  std::vector<LaunchCtx> chunks;
  std::vector<ReducePlan> plans;
  int64_t jobs = 0, blocks = 0;
  int grid = 0;
  for (int start = 0; start < n && e == cudaSuccess; start += kBatchCap) {
    LaunchCtx c;
    c.spec = &p->spec;
    c.shape = p->shape;
    c.imgs = imgs.data() + start;
    c.n = std::min(kBatchCap, n - start);
    c.out = od.p;
    c.H = od.H;
    c.W = od.W;
    c.stream = s;
    c.all_exact2x = true;
    for (int i = 0; i < c.n; ++i) c.all_exact2x = c.all_exact2x && (c.imgs[i].flags & fkl::kExact2x);
    ReducePlan pl;
    e = plan_reduce(c, pl);
    jobs += pl.jobs;
    blocks += pl.grid;
    grid = std::max(grid, pl.grid);
    chunks.push_back(c);
    plans.push_back(pl);
  }
  if (e == cudaSuccess) {
    const fkl::ReduceFinal fin =
        reduce_final(p->spec, stats, static_cast<double>(n) * od.H * od.W, fill, jobs, grid, blocks);
    if (blocks == 0) e = finish_reduce(acc, fin, s);
    for (size_t i = 0; i < chunks.size() && e == cudaSuccess; ++i) e = launch_reduce(chunks[i], plans[i], acc, fin);
  }
  return e == cudaSuccess ? FKL_OK : cuda_fail(e, "reduction");
}

fkl_status fkl_execute(fkl_pipeline p, const fkl_tensor* in, fkl_tensor* out, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  return fkl_execute_batch(p, 1, in, nullptr, out, stream);
}

fkl_status fkl_unfused_workspace_bytes(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                       const fkl_tensor* out, size_t* bytes) {
  if (!bytes) return fail(FKL_ERR_INVALID, "bytes is NULL");
  *bytes = 0;
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (is_tensor_chain(p->spec)) {
    int64_t len = 0;
    const fkl_status st = check_linear(p->spec, n, ins, rois, out, len);
    if (st != FKL_OK) return st;
    *bytes = linear_workspace_bytes(p->spec, len);
    return FKL_OK;
  }
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  const fkl_status st = validate_batch(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  int64_t px = 0;
  for (const auto& r : imgs) px = std::max(px, unfused_image_px(p->spec, od, r));
  *bytes = static_cast<size_t>(2 * unfused_slot_bytes(p->spec, std::max(px, unfused_min_px(od))));
  return FKL_OK;
}

fkl_status fkl_execute_batch_unfused(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                     fkl_tensor* out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (is_tensor_chain(p->spec)) return exec_linear(p, n, ins, rois, out, true, stream, workspace, workspace_bytes);
  size_t need = 0;
  fkl_status st = fkl_unfused_workspace_bytes(p, n, ins, rois, out, &need);
  if (st != FKL_OK) return st;
  if (!workspace || workspace_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(FKL_ERR_INVALID, "workspace must be >= %zu bytes and 256-byte aligned", need);
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  st = validate_batch(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  uint8_t* ws0 = static_cast<uint8_t*>(workspace);
  uint8_t* ws1 = ws0 + need / 2;  // need = 2 x unfused_slot_bytes
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = launch_unfused_image(p->spec, imgs[i], od.p, i, od.H, od.W, ws0, ws1, s);
    if (e != cudaSuccess) return cuda_fail(e, "unfused launch");
  }
  return FKL_OK;
}

fkl_status fkl_pipeline_get_shape(fkl_pipeline p, fkl_launch_shape* shape) {
  if (!p || !shape) return fail(FKL_ERR_INVALID, "null argument");
  *shape = p->shape;
  return FKL_OK;
}

fkl_status fkl_pipeline_set_shape(fkl_pipeline p, const fkl_launch_shape* shape) {
  if (!p || !shape) return fail(FKL_ERR_INVALID, "null argument");
  for (const auto& c : shapes_for(p->spec)) {
    if (c.vec == shape->vec && c.tx == shape->tx && c.ty == shape->ty && c.ry == shape->ry) {
      p->shape = *shape;
      return FKL_OK;
    }
  }
  return fail(FKL_ERR_INVALID, "no compiled launch shape vec=%d block=%dx%d ry=%d for this chain", shape->vec,
              shape->tx, shape->ty, shape->ry);
}

int32_t fkl_pipeline_shape_count(fkl_pipeline p) {
  return p ? static_cast<int32_t>(shapes_for(p->spec).size()) : 0;
}

fkl_status fkl_pipeline_shape_at(fkl_pipeline p, int32_t k, fkl_launch_shape* shape) {
  if (!p || !shape) return fail(FKL_ERR_INVALID, "null argument");
  const auto v = shapes_for(p->spec);
  if (k < 0 || k >= static_cast<int32_t>(v.size())) return fail(FKL_ERR_INVALID, "shape index %d out of range", k);
  *shape = v[k];
  return FKL_OK;
}

fkl_status fkl_pipeline_autotune_ex(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                    fkl_tensor* out, void* stream, int32_t reps, void (*before)(void*), void* user,
                                    fkl_launch_shape* best, float* best_us) {
  constexpr int kMaxReps = 32;
  constexpr int kFinalists = 4;      // re-timed: the shapes within 3% of the fastest
  constexpr float kFinalSlack = 1.03f;
  constexpr int kRounds = 3;         // interleaved, so that drift hits every finalist alike
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (reps < 1 || reps > kMaxReps) return fail(FKL_ERR_INVALID, "reps must be in 1..%d", kMaxReps);
  auto run = [&]() -> fkl_status { return fkl_execute_batch(p, n, ins, rois, out, stream); };
  const std::vector<fkl_launch_shape> shapes = shapes_for(p->spec);
  const fkl_launch_shape saved = p->shape;
  float best_t = -1.f;
  fkl_launch_shape best_s = saved;
  if (shapes.size() > 1) {
    // The timed launches of one shape are enqueued back to back, each
    // bracketed by its own pair of events (and preceded by the flush), the
    // way a caller's steady state runs; the median launch time ranks shapes.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[2 * kMaxReps] = {};
    cudaError_t ce = cudaSuccess;
    int made = 0;
    for (; made < 2 * reps && ce == cudaSuccess; ++made) ce = cudaEventCreate(&ev[made]);
    fkl_status st = FKL_OK;
    // median microseconds of `reps` launches with shape k (after one warm-up)
    auto time_shape = [&](const fkl_launch_shape& shape, float& us) -> bool {
      p->shape = shape;
      st = run();
      for (int r = 0; r < reps && st == FKL_OK && ce == cudaSuccess; ++r) {
        if (before) before(user);
        if ((ce = cudaEventRecord(ev[2 * r], s)) != cudaSuccess) break;
        st = run();
        if (st == FKL_OK) ce = cudaEventRecord(ev[2 * r + 1], s);
      }
      if (st != FKL_OK || ce != cudaSuccess) return false;
      if ((ce = cudaEventSynchronize(ev[2 * reps - 1])) != cudaSuccess) return false;
      float t[kMaxReps];
      for (int r = 0; r < reps && ce == cudaSuccess; ++r) ce = cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
      if (ce != cudaSuccess) return false;
      std::sort(t, t + reps);
      us = 1000.f * t[reps / 2];
      return true;
    };
    std::vector<std::pair<float, size_t>> first;  // (median, shape index)
    bool ok = ce == cudaSuccess;
    for (size_t k = 0; k < shapes.size() && ok; ++k) {
      float us = 0.f;
      ok = time_shape(shapes[k], us);
      if (ok) first.emplace_back(us, k);
    }
    if (ok && !first.empty()) {
      std::sort(first.begin(), first.end());
      std::vector<size_t> fin;
      for (const auto& f : first)
        if (fin.size() < kFinalists && f.first <= first[0].first * kFinalSlack) fin.push_back(f.second);
      best_t = first[0].first;
      best_s = shapes[first[0].second];
      if (fin.size() > 1) {
        std::vector<std::vector<float>> rounds(fin.size());
        for (int r = 0; r < kRounds && ok; ++r)
          for (size_t i = 0; i < fin.size() && ok; ++i) {
            float us = 0.f;
            ok = time_shape(shapes[fin[i]], us);
            if (ok) rounds[i].push_back(us);
          }
        if (ok) {
          for (size_t i = 0; i < fin.size(); ++i) {
            std::sort(rounds[i].begin(), rounds[i].end());
            const float us = rounds[i][rounds[i].size() / 2];
            if (i == 0 || us < best_t) {
              best_t = us;
              best_s = shapes[fin[i]];
            }
          }
        }
      }
    }
    for (int i = 0; i < made; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    if (st != FKL_OK || ce != cudaSuccess) {
      p->shape = saved;
      return st != FKL_OK ? st : cuda_fail(ce, "autotune timing");
    }
  }
  p->shape = best_s;
  if (best) *best = best_s;
  if (best_us) *best_us = best_t;
  return FKL_OK;
}

fkl_status fkl_pipeline_autotune(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                 fkl_tensor* out, void* stream, int32_t reps, fkl_launch_shape* best,
                                 float* best_us) {
  return fkl_pipeline_autotune_ex(p, n, ins, rois, out, stream, reps, nullptr, nullptr, best, best_us);
}

namespace {
// Per-image slots of the per-op form, rounded up to 768 bytes (16-byte
// vectors and 3-channel pixels in phase): an output-size float32 image, and
// the larger slot that also holds a decoded NV12 source window.
int64_t per_op_round(int64_t px) { return (px * 12 + 767) / 768 * 768; }
int64_t per_op_slot_bytes(const OutDesc& od) { return per_op_round(unfused_min_px(od)); }
int64_t per_op_slot_in_bytes(const Spec& s, const OutDesc& od, const std::vector<fkl::ResampleParams>& imgs) {
  int64_t px = unfused_min_px(od);
  for (const auto& r : imgs) px = std::max(px, unfused_image_px(s, od, r));
  return per_op_round(px);
}
int per_op_chunk(int32_t chunk, int32_t n) {
  const int c = chunk <= 0 ? n : std::min<int32_t>(chunk, n);
  return std::max(1, std::min(c, kBatchCap));
}
fkl_status per_op_validate(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                           const fkl_tensor* out, OutDesc& od, std::vector<fkl::ResampleParams>& imgs) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  if (p->spec.family != FAM_PACKED && p->spec.family != FAM_NV12)
    return fail(FKL_ERR_UNSUPPORTED, "the per-op form runs float image chains (READ_U8C3 / READ_NV12)");
  return validate_batch(p, n, ins, rois, out, od, imgs);
}
}  // namespace

fkl_status fkl_per_op_workspace_bytes(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                      const fkl_tensor* out, int32_t chunk, size_t* bytes) {
  if (!bytes) return fail(FKL_ERR_INVALID, "bytes is NULL");
  *bytes = 0;
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  const fkl_status st = per_op_validate(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  if (n == 0) return FKL_OK;
  *bytes = static_cast<size_t>(per_op_chunk(chunk, n) * (per_op_slot_in_bytes(p->spec, od, imgs) +
                                                          per_op_slot_bytes(od)));
  return FKL_OK;
}

fkl_status fkl_execute_batch_per_op(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                    fkl_tensor* out, int32_t chunk, void* workspace, size_t workspace_bytes,
                                    void* stream, fkl_kernel_time* times, int32_t max_times, int32_t* n_times) {
  if (n_times) *n_times = 0;
  if (times && (!n_times || max_times < 1)) return fail(FKL_ERR_INVALID, "times needs n_times and max_times >= 1");
  OutDesc od;
  std::vector<fkl::ResampleParams> imgs;
  fkl_status st = per_op_validate(p, n, ins, rois, out, od, imgs);
  if (st != FKL_OK) return st;
  if (n == 0) return FKL_OK;
  const int c = per_op_chunk(chunk, n);
  const int64_t slot_in = per_op_slot_in_bytes(p->spec, od, imgs), slot = per_op_slot_bytes(od);
  const size_t need = static_cast<size_t>(c * (slot_in + slot));
  if (!workspace || workspace_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
    return fail(FKL_ERR_INVALID, "workspace must be >= %zu bytes and 256-byte aligned", need);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws0 = static_cast<uint8_t*>(workspace);
  uint8_t* ws1 = ws0 + c * slot_in;
  PerOpLog log;
  log.on = times != nullptr;
  cudaError_t e = cudaSuccess;
  for (int start = 0; start < n && e == cudaSuccess; start += c) {
    fkl::OutParams o = od.p;
    o.base += start * od.p.img;
    e = launch_per_op_chunk(p->spec, imgs.data() + start, std::min(c, n - start), o, od.H, od.W, ws0, ws1, slot_in,
                            slot, log, s);
  }
  if (e == cudaSuccess && log.failed) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess && log.on) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && log.on) {  // one entry per operation, in chain order
    int k = 0;
    for (const auto& en : log.entries) {
      int j = 0;
      while (j < k && std::strncmp(times[j].name, en.name, sizeof(times[j].name)) != 0) ++j;
      if (j == k) {
        if (k == max_times) continue;
        std::memset(&times[k], 0, sizeof(times[k]));
        std::snprintf(times[k].name, sizeof(times[k].name), "%s", en.name);
        ++k;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, en.start, en.stop) != cudaSuccess) ms = 0.f;
      times[j].launches += 1;
      times[j].bytes += en.bytes;
      times[j].ms += ms;
    }
    *n_times = k;
  }
  for (const auto& en : log.entries) {
    if (en.start) cudaEventDestroy(en.start);
    if (en.stop) cudaEventDestroy(en.stop);
  }
  return e == cudaSuccess ? FKL_OK : cuda_fail(e, "per-op launch");
}

fkl_status fkl_execute_batch_unfused_static(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                            fkl_tensor* out, void* stream) {
  if (!p) return fail(FKL_ERR_INVALID, "null pipeline");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (is_tensor_chain(p->spec)) {  // the float32 copy of one tensor, if any, lives in the static scratch
    int64_t len = 0;
    const fkl_status st = check_linear(p->spec, n, ins, rois, out, len);
    if (st != FKL_OK) return st;
    const size_t need = linear_workspace_bytes(p->spec, len);
    if (need > kStaticScratchBytes)
      return fail(FKL_ERR_INVALID,
                  "tensors of %lld elements need %zu bytes of scratch; the static scratch holds %zu bytes "
                  "(use fkl_execute_batch_unfused with a caller workspace)",
                  static_cast<long long>(len), need, kStaticScratchBytes);
    void* scratch = nullptr;
    if (need > 0 && n > 0) {
      const cudaError_t e = static_scratch(&scratch);
      if (e != cudaSuccess) return cuda_fail(e, "static scratch lookup");
    }
    return run_linear(p, n, ins, out, len, true, stream, scratch, kStaticScratchBytes);
  }
  if (n < 0) return fail(FKL_ERR_INVALID, "negative batch size");
  if (n > 0 && !ins) return fail(FKL_ERR_INVALID, "inputs missing");
  OutDesc od;
  fkl_status st = check_out(p->spec, out, n, od);
  if (st != FKL_OK) return st;
  // First pass: validate every image and size the two intermediates (no
  // host or device allocation: one image's parameters at a time).
  int64_t px = unfused_min_px(od);
  for (int i = 0; i < n; ++i) {
    fkl::ResampleParams r;
    st = image_params(p->spec, &ins[i], rois, i, od, r);
    if (st != FKL_OK) return st;
    px = std::max(px, unfused_image_px(p->spec, od, r));
  }
  const int64_t each = unfused_slot_bytes(p->spec, px);
  if (2 * each > static_cast<int64_t>(kStaticScratchBytes))
    return fail(FKL_ERR_INVALID,
                "these images need %lld bytes of scratch; the static scratch holds %zu bytes "
                "(use fkl_execute_batch_unfused with a caller workspace)",
                static_cast<long long>(2 * each), kStaticScratchBytes);
  if (n == 0) return FKL_OK;
  void* base = nullptr;
  const cudaError_t ce = static_scratch(&base);
  if (ce != cudaSuccess) return cuda_fail(ce, "static scratch address");
  uint8_t* ws0 = static_cast<uint8_t*>(base);
  uint8_t* ws1 = ws0 + each;
  for (int i = 0; i < n; ++i) {
    fkl::ResampleParams r;
    st = image_params(p->spec, &ins[i], rois, i, od, r);
    if (st != FKL_OK) return st;
    const cudaError_t e = launch_unfused_image(p->spec, r, od.p, i, od.H, od.W, ws0, ws1, s);
    if (e != cudaSuccess) return cuda_fail(e, "unfused launch");
  }
  return FKL_OK;
}

}  // extern "C"
