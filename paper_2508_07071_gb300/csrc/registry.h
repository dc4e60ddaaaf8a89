// Internal interface between the C ABI (api.cu) and the translation units
// that hold the compiled chain instantiations (k_*.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fkl.h"
#include "fkl/dpp.cuh"

namespace fkl {
struct ReduceAcc;    // fkl/reduce.cuh
struct ReduceFinal;  // fkl/reduce.cuh
}  // namespace fkl

namespace fkl_impl {

enum Family { FAM_PACKED = 1, FAM_NV12 = 2, FAM_INT = 3, FAM_VCHAIN = 4, FAM_CAST = 5 };
enum Geom { GEOM_NONE = 0, GEOM_RESIZE = 1, GEOM_LETTERBOX = 2 };

// A parsed chain: which compiled family runs it and the runtime parameters
// of every op (absent arithmetic ops hold their identity constants).
struct Spec {
  Family family;
  bool has_crop = false;
  int32_t crop[4] = {0, 0, 0, 0};
  Geom geom = GEOM_NONE;
  int32_t out_w = 0, out_h = 0;
  float pad = 0.f;
  bool swap = false;
  bool has_mul = false, has_sub = false, has_div = false, has_addsat = false;
  float mul[3] = {1.f, 1.f, 1.f};
  float sub[3] = {0.f, 0.f, 0.f};  // ADD c is stored as SUB -c (same bits)
  float div[3] = {1.f, 1.f, 1.f};
  int32_t addsat[3] = {0, 0, 0};
  bool split = true;
  int32_t out_dtype = FKL_F32;
  float fp8_scale = 1.f;
  bool vinput_u8 = false;       // vertical chain over a u8 tensor
  int32_t in_dtype = FKL_U8;    // typed chains: element type of the inputs
  std::vector<int32_t> vkinds;  // vertical chain: 0 = Mul, 1 = Add
  std::vector<float> vconsts;
};

// One launch of an image family: up to kBatchCap images.
using fkl::kBatchCap;

struct LaunchCtx {
  const Spec* spec;
  fkl_launch_shape shape;
  const fkl::ResampleParams* imgs;  // host array of n entries
  int n;
  fkl::OutParams out;
  int H, W;
  cudaStream_t stream;
  bool all_exact2x;  // every image of the launch is an exact 2x downscale
  int* device_error = nullptr;  // flag a bounded device wait sets when it gives up
  unsigned long long wait_ns = 0;  // limit of one bounded device wait
};

// Limit of one bounded device wait of the fused kernels (fkl_set_device_wait_limit).
unsigned long long device_wait_limit_ns();

// Device address of this library's wait-timeout flag on the current device.
cudaError_t device_error_flag(int** out);

// Fused launches of the float image families, one translation unit per
// (source, output type): k_<src>_<type>.cu.
cudaError_t launch_packed_f32(const LaunchCtx& c);
cudaError_t launch_packed_f16(const LaunchCtx& c);
cudaError_t launch_packed_bf16(const LaunchCtx& c);
cudaError_t launch_packed_e4m3(const LaunchCtx& c);
cudaError_t launch_nv12_f32(const LaunchCtx& c);
cudaError_t launch_nv12_f16(const LaunchCtx& c);
cudaError_t launch_nv12_bf16(const LaunchCtx& c);
cudaError_t launch_nv12_e4m3(const LaunchCtx& c);
// Integer chains (k_int.cu).
cudaError_t launch_int(const LaunchCtx& c);
// ReduceDPP over a float image chain (k_reduce.cu). plan_reduce sizes the
// reduction launch of one chunk of at most kBatchCap images (grid 0: no
// window pixels, no launch); launch_reduce reduces the ROp's values over
// each image's placed window into `acc` (zeroed by the caller), and the
// block that completes `fin.blocks`, the blocks of all the call's launches,
// writes the statistics of include/fkl.h; finish_reduce writes them for a
// call that launched nothing. reduce_final describes the call: `count`
// output pixels per channel, `fill_count` of them fill pixels.
struct ReducePlan {
  int32_t col_tiles = 0, row_tiles = 0;
  int64_t jobs = 0;
  int grid = 0;
};
cudaError_t plan_reduce(const LaunchCtx& c, ReducePlan& pl);
cudaError_t launch_reduce(const LaunchCtx& c, const ReducePlan& pl, fkl::ReduceAcc* acc, const fkl::ReduceFinal& fin);
fkl::ReduceFinal reduce_final(const Spec& s, float* stats, double count, double fill_count, int64_t jobs, int grid,
                              int64_t blocks);
cudaError_t finish_reduce(const fkl::ReduceAcc* acc, const fkl::ReduceFinal& fin, cudaStream_t st);
// Vertical chain (k_vchain.cu): one fused launch per chunk of ops.
constexpr int kVChainCap = 4096;
cudaError_t launch_vchain(const Spec& s, const fkl_launch_shape& shape, const void* in, float* out,
                          int64_t n, cudaStream_t stream);

// Typed chains (k_cast.cu): n linear tensors of `len` elements each into
// out[n * len]; fused (one launch per 256 tensors) and unfused (one kernel
// per op and tensor, in place on a float32/float64 output, else on `ws`:
// len float32 values).
cudaError_t launch_cast(const Spec& s, const fkl_launch_shape& shape, int n, const void* const* ins, void* out,
                        int64_t len, cudaStream_t stream);
cudaError_t launch_unfused_cast(const Spec& s, int n, const void* const* ins, void* out, int64_t len, void* ws,
                                cudaStream_t stream);

// Unfused reference form (k_unfused.cu): one kernel per op for one image;
// ws0 and ws1 each hold one intermediate image.
cudaError_t launch_unfused_image(const Spec& s, const fkl::ResampleParams& img,
                                 const fkl::OutParams& out, int z, int H, int W,
                                 void* ws0, void* ws1, cudaStream_t stream);
cudaError_t launch_unfused_vchain(const Spec& s, const void* in, float* out, int64_t n,
                                  cudaStream_t stream);

// Optional per-kernel timing of the per-op form: events around each launch
// (only when `on`), with the kernel's name and algorithmic bytes.
struct PerOpLog {
  struct Entry {
    const char* name;
    double bytes;
    cudaEvent_t start = nullptr, stop = nullptr;
  };
  bool on = false;
  bool failed = false;
  std::vector<Entry> entries;
  void begin(const char* name, double bytes, cudaStream_t st);
  void end(cudaStream_t st);
};

// The per-op form over a chunk of n <= kBatchCap images (k_unfused.cu): one
// kernel per operation over all n images. ws0 holds n slots of `slot_in`
// bytes (the NV12 decode at source size, later reused at output size), ws1 n
// slots of `slot` bytes (one output-size image each); slot_in >= slot, both
// multiples of 768, so the output-size images of a chunk are contiguous in
// either buffer.
cudaError_t launch_per_op_chunk(const Spec& s, const fkl::ResampleParams* imgs, int n, const fkl::OutParams& out,
                                int H, int W, uint8_t* ws0, uint8_t* ws1, int64_t slot_in, int64_t slot,
                                PerOpLog& log, cudaStream_t stream);

// Launch shapes compiled for a family/dtype (the autotuner's search space).
std::vector<fkl_launch_shape> shapes_for(const Spec& s);
fkl_launch_shape default_shape(const Spec& s);

int sm_count();

// Sets the thread-local message returned by fkl_last_error().
void set_last_error(const char* msg);

// Resize / letterbox placement of a source window (r.rx..r.rh set) in an
// out_w x out_h output: fills dw, dh, ox, oy, pad, inv_area, kExact2x.
void place(const Spec& s, int out_w, int out_h, fkl::ResampleParams& r);

}  // namespace fkl_impl

// A bound chain (the handle behind fkl_pipeline).
struct fkl_pipeline_s {
  fkl_impl::Spec spec;
  fkl_launch_shape shape;
  std::string name;
};
