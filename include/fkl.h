/*
 * fkl.h -- C ABI of the fused image-preprocessing library for GB300 (sm_103a).
 *
 * The library follows the Fused Kernel method (paper §IV): a user chain is one
 * Read Operation (ROp), any number of Compute Operations (COps) and one Write
 * Operation (WOp), run as ONE CUDA kernel whose intermediates stay in
 * registers (vertical fusion, paper §II and Fig. 3), over one image or a batch
 * of independent images in one launch (horizontal fusion, paper §II Fig. 5 and
 * §IV-B BatchRead/BatchWrite). Functions return descriptions of work and
 * launch nothing until an execute call (the lazy final interface of §IV-D).
 *
 * Memory: every tensor is caller-owned device memory (borrowed for the length
 * of the call and of the work it enqueues). The library allocates no
 * intermediate images (paper §VI-L). Streams are the caller's; all execute
 * calls are asynchronous on the given stream (NULL = legacy default stream).
 * No call synchronises the device except where stated.
 *
 * Errors: every call returns an fkl_status; on failure a thread-local message
 * is available from fkl_last_error(). Invalid arguments are rejected before
 * anything is enqueued. There is no CPU fallback: a chain that no compiled
 * kernel implements is FKL_ERR_UNSUPPORTED.
 *
 * Thread safety: distinct pipelines may be used from distinct threads; one
 * pipeline may be executed concurrently (it holds no per-call state), but
 * fkl_pipeline_set_shape and fkl_pipeline_autotune change its launch shape
 * and must not overlap other calls on the same pipeline.
 * fkl_set_device_wait_limit is process-wide.
 */
#ifndef FKL_H_
#define FKL_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FKL_API __attribute__((visibility("default")))
#else
#define FKL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                             */
/* ------------------------------------------------------------------------ */
typedef enum {
  FKL_OK = 0,
  FKL_ERR_INVALID = 1,     /* bad argument: grammar, dims, dtype, pitch, ROI */
  FKL_ERR_UNSUPPORTED = 2, /* valid chain with no compiled kernel           */
  FKL_ERR_OOM = 3,         /* host allocation failed                        */
  FKL_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has it)   */
  FKL_ERR_TIMEOUT = 5      /* a bounded device wait gave up                 */
} fkl_status;

/* ------------------------------------------------------------------------ */
/* Tensors                                                                  */
/* ------------------------------------------------------------------------ */
enum {                 /* element types                                     */
  FKL_U8 = 0,
  FKL_F32 = 1,
  FKL_F16 = 2,         /* IEEE binary16                                     */
  FKL_BF16 = 3,
  FKL_E4M3 = 4,        /* OCP FP8 E4M3 (finite-only, max 448)               */
  FKL_U16 = 5,         /* typed chains (inputs)                             */
  FKL_F64 = 6          /* typed chains (inputs and outputs)                 */
};

enum {                 /* layouts and the meaning of dims[]                 */
  FKL_LAYOUT_LINEAR = 0, /* dims = {N}: N contiguous elements               */
  FKL_LAYOUT_HWC = 1,    /* dims = {H, W, C}: packed pixels, rows pitch_bytes apart */
  FKL_LAYOUT_NV12 = 2,   /* dims = {H, W}: u8 luma rows, then H/2 rows of
                            interleaved (U, V) pairs starting at
                            data + H * pitch_bytes, same pitch; H, W even   */
  FKL_LAYOUT_NCHW = 3,   /* dims = {N, C, H, W}: planar; rows pitch_bytes
                            apart, planes H * pitch_bytes apart              */
  FKL_LAYOUT_NHWC = 4    /* dims = {N, H, W, C}: packed; rows pitch_bytes
                            apart, images H * pitch_bytes apart              */
};

typedef struct {
  void* data;            /* device pointer, caller-owned                      */
  int64_t dims[4];       /* see the layout; unused entries 0                  */
  int64_t pitch_bytes;   /* bytes between rows; 0 = tightly packed rows       */
  int32_t dtype;         /* FKL_U8 ...                                        */
  int32_t layout;        /* FKL_LAYOUT_...                                    */
} fkl_tensor;

/* ------------------------------------------------------------------------ */
/* Operation descriptors (the IOps of paper §IV-A/§IV-B)                     */
/* ------------------------------------------------------------------------ */
enum {
  /* Read Operations (paper Table I "ReadType"): the first descriptor.      */
  FKL_OP_READ_U8C3 = 1,  /* packed 3-channel u8 image (HWC)                 */
  FKL_OP_READ_NV12 = 2,  /* NV12 frame, decoded BT.601 limited range to RGB */
  FKL_OP_READ_F32 = 3,   /* linear float32 tensor                           */
  FKL_OP_READ_U8 = 4,    /* linear u8 tensor, converted to float exactly
                            (vertical and typed chains)                    */
  FKL_OP_READ_U16 = 5,   /* linear u16 tensor (typed chains)                */
  FKL_OP_READ_F64 = 6,   /* linear float64 tensor (typed chains)            */

  /* Read modifiers: together with the source they form the one ROp.       */
  FKL_OP_CROP = 10,      /* i[0..3] = x, y, w, h of the window read        */
  FKL_OP_RESIZE = 11,    /* i[0], i[1] = output width, height; bilinear,
                            half-pixel centres, border clamp               */
  FKL_OP_LETTERBOX = 12, /* i[0], i[1] = output width, height; f[0] = pad
                            value in source units; aspect-preserving fit,
                            size floor(s*r + 0.5), centred, odd pad pixel
                            at the bottom/right                            */

  /* Compute Operations (paper Table I "UnaryType"/"BinaryType").          */
  FKL_OP_SWAP_RB = 20,   /* BGR <-> RGB: reverse the 3 channels             */
  FKL_OP_MUL = 21,       /* x * f[c]   (3-channel chains: f[0..2]; F32: f[0]) */
  FKL_OP_ADD = 22,       /* x + f[c]                                        */
  FKL_OP_SUB = 23,       /* x - f[c]                                        */
  FKL_OP_DIV = 24,       /* x / f[c], IEEE division                         */
  FKL_OP_ADD_SAT_U8 = 25,/* u8 chains: clamp(x + i[c], 0, 255)              */

  /* Write Operations (paper Table I "WriteType"): the last descriptor.    */
  FKL_OP_WRITE_PACKED = 40, /* i[0] = output dtype; packed (HWC / linear)   */
  FKL_OP_WRITE_SPLIT = 41   /* i[0] = output dtype; planar (paper Fig. 9
                               Split); for FKL_E4M3, f[0] = per-tensor
                               scale s > 0 and the stored code is
                               satfinite_rne(x / s)                         */
};

typedef struct {
  int32_t op;            /* FKL_OP_...                                      */
  float f[8];            /* float parameters                                */
  int32_t i[8];          /* integer parameters                              */
} fkl_op_desc;

typedef struct fkl_pipeline_s* fkl_pipeline;  /* library-owned handle        */

/* ------------------------------------------------------------------------ */
/* Pipelines                                                                */
/* ------------------------------------------------------------------------ */

/*
 * Bind a chain (paper §IV-C TransformDPP: ROp -> COp* -> WOp, §IV-D executor)
 * to one compiled kernel.
 *
 * ops[0] is a READ_*; then optional read modifiers (CROP, then RESIZE or
 * LETTERBOX); then COps; ops[n_ops-1] is a WRITE_*. Anything else is
 * FKL_ERR_INVALID. The kernel is chosen from a fixed set compiled ahead of
 * time from C++17 templates (one instantiation per chain shape):
 *   READ_U8C3 [CROP] RESIZE [SWAP_RB] [MUL] [ADD|SUB] [DIV] WRITE_{SPLIT,PACKED}
 *        (float math; output F32/F16/BF16/E4M3)
 *   READ_NV12 (RESIZE|LETTERBOX) [SWAP_RB] [MUL] [ADD|SUB] [DIV] WRITE_{SPLIT,PACKED}
 *   READ_U8C3 [CROP] [SWAP_RB] [ADD_SAT_U8] WRITE_{SPLIT,PACKED} (U8 output)
 *   READ_F32|READ_U8 (MUL|ADD){0..65536} WRITE_PACKED(F32)   (vertical chain)
 *   READ_U8|READ_U16|READ_F32|READ_F64 [MUL] [ADD|SUB] [DIV]
 *        WRITE_PACKED(F32|F64|F16|BF16|E4M3)
 *        (typed chain, paper §VI-I Read -> Cast -> Multiply -> Subtract ->
 *        Divide -> Write: the input is cast to the compute type -- F64 for an
 *        F64 output, else F32 -- then every op runs and rounds once in it,
 *        constants f[0] taken exactly into it; the write rounds to the output
 *        type to nearest even (E4M3: sat_RNE(v / s), saturating at +-448;
 *        the kernel forms v / s as the F32 product with fl32(1/s), so next to
 *        an E4M3 tie the stored code may be the neighbour of the rounded
 *        exact quotient, within one E4M3 ulp). A READ_F32|READ_U8 chain of
 *        MUL/ADD only writing F32 is a vertical chain)
 * An absent MUL/ADD/SUB/DIV is bound as its identity (x*1, x-0, x/1 are
 * exact, so the result equals the shorter chain bit for bit). A chain of the
 * right grammar outside this set returns FKL_ERR_UNSUPPORTED.
 *
 * On success *out owns host memory only; free it with fkl_pipeline_destroy.
 */
FKL_API fkl_status fkl_pipeline_create(const fkl_op_desc* ops, int32_t n_ops,
                               fkl_pipeline* out);

/*
 * Run the chain once: one image `in` to one output `out` (batch of one) --
 * the TransformDPP of paper §IV-C over one image: every output pixel reads
 * its value through the ROp, passes it through the COps in order and stores
 * it with the WOp, in one kernel (vertical fusion, paper §II Fig. 3B and
 * Algorithm 1 "KernelFunctionB").
 * Image chains: `in` is HWC u8 (READ_U8C3) or NV12 (READ_NV12); the ROI is the
 * CROP descriptor's, else the whole image. `out` is NCHW (WRITE_SPLIT) or
 * NHWC (WRITE_PACKED) with N = 1 and the dtype the WOp names; its H, W must
 * equal the RESIZE/LETTERBOX size (the ROI size when there is no resize).
 * Vertical chains: `in` (LINEAR F32, or U8 for READ_U8) and `out` (LINEAR
 * F32) have the same length (F32 input may alias the output). Typed chains:
 * `in` LINEAR of the read's type, `out` LINEAR of the write's type, same
 * length (a batch of one). stream is a cudaStream_t. One kernel launch per call (vertical
 * chains longer than 4096 ops use one launch per 4096 ops).
 */
FKL_API fkl_status fkl_execute(fkl_pipeline p, const fkl_tensor* in, fkl_tensor* out,
                       void* stream);

/*
 * Horizontal fusion (paper §IV-B BatchRead/BatchWrite): n independent images
 * ins[0..n-1] (each its own size and pointer; the same pointer may repeat,
 * e.g. many crops of one frame) into out[n, C, H, W] (or [n, H, W, C]).
 * rois: n x 4 int32 (x, y, w, h) on the host, or NULL to use the CROP
 * descriptor (or the whole image) for every image. Every ROI must lie inside
 * its image. One launch covers up to 256 images; larger n uses ceil(n/256)
 * launches.
 * Tensor chains (vertical and typed): n LINEAR tensors of the read's type and
 * one common length L (each its own pointer) into one LINEAR output of n * L
 * elements of the write's type, tensor i at elements [i * L, (i + 1) * L);
 * rois must be NULL; an empty batch may pass NULL data. Typed chains run in
 * one launch per 256 tensors, vertical chains in one launch per tensor.
 */
FKL_API fkl_status fkl_execute_batch(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                             const int32_t* rois, fkl_tensor* out,
                             void* stream);

/*
 * Release a pipeline: the host-side counterpart of fkl_pipeline_create (the
 * IOp description the executor of paper §IV-D holds). It frees host memory
 * only; the pipeline owns no device memory and no stream, so work already
 * enqueued with it is unaffected. NULL is ignored. Do not destroy a pipeline
 * while another thread is calling into the library with it.
 */
FKL_API void fkl_pipeline_destroy(fkl_pipeline p);

/*
 * Message of the last failed call on this thread ("" if none). The paper
 * defines no error reporting (its C++ API fails at compile time, §IV-D); a C
 * ABI binds chains at run time, so every call returns an fkl_status and this
 * thread-local text says which argument or CUDA call failed. The pointer is
 * valid until the next library call on the same thread.
 */
FKL_API const char* fkl_last_error(void);

/* ------------------------------------------------------------------------ */
/* Unfused reference form (same GPU): one kernel per operation               */
/* ------------------------------------------------------------------------ */

/*
 * The chain as a conventional library runs it (paper §II Fig. 3A, Algorithm
 * 1 "MainFunctionA"): one kernel per operation, every intermediate written to
 * and read back from device memory. It uses the same Operation code as the
 * fused kernel, so results are identical to fkl_execute_batch.
 *
 * fkl_unfused_workspace_bytes: bytes of device workspace (for the
 * intermediates of one image, reused image after image) that
 * fkl_execute_batch_unfused needs for these arguments. This is also the
 * device memory that fusion saves (paper §VI-L).
 * fkl_execute_batch_unfused: `workspace` is caller-owned device memory of at
 * least that size, 256-byte aligned. Launch count = n * (ops in the chain).
 * Tensor chains (vertical and typed): one kernel per tensor and op, in place
 * on the output (0 bytes of workspace); for typed chains the first kernel
 * reads and casts, and F16/BF16/E4M3 outputs keep the F32 values of one
 * tensor in the workspace (its length x 4 bytes, rounded up to 256) and
 * write the output in a last kernel per tensor.
 */
FKL_API fkl_status fkl_unfused_workspace_bytes(fkl_pipeline p, int32_t n,
                                       const fkl_tensor* ins,
                                       const int32_t* rois,
                                       const fkl_tensor* out, size_t* bytes);
FKL_API fkl_status fkl_execute_batch_unfused(fkl_pipeline p, int32_t n,
                                     const fkl_tensor* ins, const int32_t* rois,
                                     fkl_tensor* out, void* workspace,
                                     size_t workspace_bytes, void* stream);

/*
 * The per-op form over the whole batch: the unfused chain as the paper
 * states it (paper §II Fig. 3A, Algorithm 1 "MainFunctionA"; the vertical-
 * fusion comparison of §VI-B): each operation is ONE kernel over every image
 * of a chunk, every intermediate written to and read back from device
 * memory. fkl_execute_batch_unfused above is the per-image form (one kernel
 * per operation and image, the horizontal-fusion comparison of §VI-C).
 * Float image chains (READ_U8C3 / READ_NV12 families) only; others are
 * FKL_ERR_UNSUPPORTED. The kernels run the same Operation code as the fused
 * kernel, so the results equal fkl_execute_batch's bit for bit.
 *
 * Kernels, each over the chunk: NV12 chains decode the source windows to
 * float32 RGB at full resolution (one launch per run of images with equal
 * windows), then resize / letterbox them; packed chains crop + resize the u8
 * source to float32 RGB; then one kernel per COp (SWAP_RB, MUL, ADD/SUB,
 * DIV) over the chunk's pixels; then the write (split and cast).
 * Intermediates are packed float32 images (12 bytes per pixel) in two sets
 * of slots: an output-size slot = H x W x 12 bytes, and an input slot = (the
 * largest of H x W and, for NV12, the source windows' w x h) x 12 bytes, both
 * rounded up to a multiple of 768; the COp kernels ping-pong between the two
 * sets over the chunk's output-size images only.
 *
 * chunk: images per launch, 1..256 (<= 0: min(n, 256)); n images run as
 * ceil(n / chunk) rounds of every kernel.
 * fkl_per_op_workspace_bytes: min(chunk, n) x (input slot + output slot)
 * bytes of device workspace.
 * fkl_execute_batch_per_op: `workspace` is caller-owned device memory of at
 * least that size, 256-byte aligned. times (optional, NULL = none): when
 * given, every launch is bracketed by CUDA events, the call synchronizes
 * `stream` before it returns, and times[0 .. *n_times - 1] receive one entry
 * per operation in chain order (at most max_times): its name, launches,
 * algorithmic bytes read and written (the distinct tap bytes of a resize,
 * the whole images otherwise), and device time. Without `times` the call is
 * asynchronous and may be captured in a CUDA graph.
 */
typedef struct {
  char name[32];      /* the operation, e.g. "decode NV12 -> RGB f32"          */
  int32_t launches;   /* kernel launches of this operation in the call         */
  double bytes;       /* algorithmic bytes its launches read and write         */
  double ms;          /* their device time (CUDA events on the stream)         */
} fkl_kernel_time;

FKL_API fkl_status fkl_per_op_workspace_bytes(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                              const int32_t* rois, const fkl_tensor* out, int32_t chunk,
                                              size_t* bytes);
FKL_API fkl_status fkl_execute_batch_per_op(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                            fkl_tensor* out, int32_t chunk, void* workspace,
                                            size_t workspace_bytes, void* stream, fkl_kernel_time* times,
                                            int32_t max_times, int32_t* n_times);

/*
 * fkl_execute_batch_unfused_static: the unfused form above, for callers that
 * cannot allocate device memory -- for example a host framework that owns
 * every device allocation under a fixed memory budget, or a latency-critical
 * loop where cudaMalloc's implicit device synchronisation is not acceptable.
 * This call allocates nothing (no cudaMalloc/cudaFree, no host heap): the two
 * intermediate images live in one 32 MiB array (32 * 2^20 bytes) that the
 * library declares statically in device memory; every GPU that loads the
 * library holds it until the process exits. The paper has no counterpart: it
 * is a service of this library, not part of the fused method.
 *
 * Arguments and results are those of fkl_execute_batch_unfused without the
 * workspace. A batch whose intermediates need more than 32 MiB (the value
 * fkl_unfused_workspace_bytes reports) is rejected with FKL_ERR_INVALID
 * before anything is enqueued; vertical chains need no scratch.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. Every call shares the one array and leaves its last contents in
 * it: nothing needs to start at zero, because each intermediate is written in
 * full before it is read, but calls whose work overlaps on the GPU (other
 * streams, other threads) race on it -- order them on one stream or with
 * events.
 */
FKL_API fkl_status fkl_execute_batch_unfused_static(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                                    const int32_t* rois, fkl_tensor* out,
                                                    void* stream);

/* ------------------------------------------------------------------------ */
/* ReduceDPP: several reductions from one read; dynamic FP8 scaling         */
/* ------------------------------------------------------------------------ */

/*
 * The reduction pattern of paper §IV-C: the statistics of the values the
 * pipeline's chain gives every output pixel of an fkl_execute_batch call with
 * these arguments, from one read of the inputs and with no output written.
 * `out` fixes the output size and is not written. `stats` is device memory
 * of FKL_REDUCE_STATS_BYTES bytes, 16-byte aligned; when the work is done
 * (stream order) it holds floats:
 *   [0..2] minimum per channel   [3..5] maximum per channel
 *   [6..8] mean per channel      [9]    maximum absolute value, amax
 *   [10]   s = amax / 448, the per-tensor scale that maps the values onto
 *          the FP8-E4M3 range (1 when amax is 0)   [11] 1 / s
 * and two int32 words describing the work split: [12] reduction jobs (tiles
 * of window pixels), [13] blocks of the largest reduction launch (a
 * persistent grid: each block walks every grid-th job).
 * Bytes 64..127 are the accumulator (overwritten). Float image families
 * only (READ_U8C3 / READ_NV12 with a resize or letterbox).
 * How: the ROp is evaluated once per pixel of each image's placed window and
 * its per-channel extremes and sum are reduced; the COps of these chains
 * (SWAP_RB, MUL, ADD/SUB, DIV by per-channel constants, each rounded) are
 * monotone and affine on every channel, so the block that finishes last
 * maps the read values' extremes through them (the result equals the
 * extremes of the values fkl_execute_batch writes with an F32 output, bit
 * for bit) and the mean through the affine map in float64; fill pixels (the
 * letterbox pad) join on the host's count. Min/max are exact; sums are
 * accumulated in 64-bit fixed point (2^-10 read units), independent of the
 * grid and of the order in which blocks finish. Launches: one memset of the
 * accumulator and one reduction launch per 256 images (a call without any
 * window pixel launches one small kernel that writes the statistics
 * instead). Calls that share a `stats` buffer must not overlap on the GPU.
 * An empty batch (n = 0) leaves NaN extremes, mean 0, amax 0 and s = 1.
 */
#define FKL_REDUCE_STATS_BYTES 128
FKL_API fkl_status fkl_reduce_batch(fkl_pipeline p, int32_t n, const fkl_tensor* ins, const int32_t* rois,
                                    const fkl_tensor* out, float* stats, void* stream);

/*
 * fkl_execute_batch with the FP8-E4M3 scale read from device memory:
 * `scale_inv_dev` points at 1/s (e.g. stats + 11 of fkl_reduce_batch), so a
 * reduce pass and a write pass give dynamic per-tensor scaling with no
 * host round trip. The pipeline's WOp must write E4M3.
 */
FKL_API fkl_status fkl_execute_batch_scaled(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                            const int32_t* rois, fkl_tensor* out, const float* scale_inv_dev,
                                            void* stream);

/*
 * fkl_execute_batch on buffers in pinned host memory (cudaHostAlloc, or
 * cudaHostRegister'ed), read and written by the fused kernel itself over the
 * host link (no staging copies: on a Grace host the NVLink-C2C link is
 * coherent, and the one kernel streams the inputs in and the outputs out).
 * Every input and the output may each be pinned host memory or device memory;
 * each pointer is checked with cudaPointerGetAttributes and replaced by its
 * device address. Pageable (unregistered) host memory is FKL_ERR_INVALID and
 * nothing is launched. Arguments and results are otherwise those of
 * fkl_execute_batch; the host buffers must stay valid until `stream` has
 * passed the launch.
 */
FKL_API fkl_status fkl_execute_batch_mapped(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                            const int32_t* rois, fkl_tensor* out, void* stream);

/* ------------------------------------------------------------------------ */
/* Host-buffer executor: overlapped copy-in, fused launch, copy-out          */
/* ------------------------------------------------------------------------ */

/*
 * For callers whose images live in host memory. The executor owns `depth`
 * device slots, each holding the inputs and outputs of up to `chunk` images
 * (`in_bytes` and `out_bytes` per image at most), and three non-blocking
 * streams (copy-in, compute, copy-out). fkl_execute_batch_host splits a
 * batch into chunks and pipelines them: while chunk c is computed, chunk c+1
 * is copied in and chunk c-1 copied out, so the host link in both directions
 * and the fused kernel overlap. The paper measures device-resident data
 * only; this is the library's data path from and to the host.
 *
 * create: allocates the slots (cudaMalloc) and streams on the current
 * device; FKL_ERR_CUDA if that fails. destroy synchronises the executor's
 * streams and frees everything.
 * execute: `ins` are host tensors (HWC u8 or NV12, pinned memory for
 * asynchronous copies; pageable memory works but serialises), `out` a host
 * tensor laid out as for fkl_execute_batch. The call enqueues everything and
 * returns; the work is ordered after earlier work on `stream`, and `stream`
 * waits for its completion (synchronise `stream`, then read `out`). The host
 * buffers must stay valid and unmodified until then. Images are copied into
 * a slot at a 16-byte-aligned pitch, so vector loads apply to any host pitch.
 * An image larger than `in_bytes` (or an output image larger than
 * `out_bytes`) is FKL_ERR_INVALID. One fused launch per chunk.
 */
typedef struct fkl_host_executor_s* fkl_host_executor;
FKL_API fkl_status fkl_host_executor_create(fkl_pipeline p, int32_t chunk, int32_t depth, size_t in_bytes,
                                            size_t out_bytes, fkl_host_executor* out);
FKL_API fkl_status fkl_execute_batch_host(fkl_host_executor e, int32_t n, const fkl_tensor* ins,
                                          const int32_t* rois, fkl_tensor* out, void* stream);
FKL_API void fkl_host_executor_destroy(fkl_host_executor e);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of preprocessing requests                    */
/* ------------------------------------------------------------------------ */

/*
 * A server runs one image chain (a READ_U8C3 [CROP] RESIZE ... WRITE_SPLIT
 * pipeline) for a stream of requests, each a list of host images of mixed
 * sizes. It is the horizontal fusion of paper §IV-B applied over time:
 * requests that arrive while others run are admitted as soon as a request
 * slot and enough device memory are free, and their images are processed
 * alongside the ones already on the GPU. The paper has no serving loop; this
 * is the library's.
 *
 * Modes:
 *   FKL_SERVE_PERSISTENT  a persistent kernel (up to ctas_per_sm CTAs per SM)
 *                         pulls tasks from a queue in mapped host memory;
 *                         a task is a band of 16 output rows of one image.
 *                         The CTA reads the source rows its band's taps
 *                         reference straight from the request's pinned host
 *                         image (16-byte loads over the host link; for a
 *                         downscale by more than 2, only the two tap rows of
 *                         each output row -- e.g. at most 448 rows of a
 *                         2160-row image for 224 output rows -- instead of
 *                         the whole image) into device memory, then runs the
 *                         chain on the band. No copy engine and no host
 *                         round trip sit between admission and the kernel;
 *                         request completion is counted on the device. Images
 *                         must be pinned host memory (cudaHostAlloc or
 *                         cudaHostRegister; anything else is
 *                         FKL_ERR_INVALID at submit) and stay valid until
 *                         the request is done; a request holds at most
 *                         8192 / ceil(H / 16) images.
 *   FKL_SERVE_BATCH       one fused fkl_execute_batch launch per request.
 *   FKL_SERVE_UNFUSED     per request, the unfused one-kernel-per-op form
 *                         (the conventional-library baseline).
 * Admission: requests are admitted in arrival order (FIFO) when one of
 * `max_inflight` slots is free and the first-fit allocator of a device arena
 * of `arena_bytes` finds room for the request's device copies of its images
 * (persistent mode: the staged tap rows; other modes: the whole images,
 * copied with tight rows, one contiguous copy per image when the host rows
 * are tight) and outputs. A request that could never fit is refused at
 * submit (FKL_ERR_INVALID).
 * Waits: the persistent kernel's CTAs stop after `idle_us` microseconds
 * without work (or at destroy); the server relaunches them when work
 * arrives. No device wait is unbounded.
 * Threading: one internal host thread drives admission, copies, launches and
 * completion; submit/poll/wait/release may be called from any thread.
 * Times are CLOCK_MONOTONIC seconds.
 */
enum { FKL_SERVE_PERSISTENT = 0, FKL_SERVE_BATCH = 1, FKL_SERVE_UNFUSED = 2 };

typedef struct {
  int32_t mode;            /* FKL_SERVE_*                                      */
  int32_t max_inflight;    /* request slots, 1..1024                           */
  size_t arena_bytes;      /* device memory for admitted requests              */
  int32_t ctas_per_sm;     /* persistent mode: CTAs per SM (1..8); 1 is the
                              fastest measured (more bands in flight read
                              more scattered host pages at once: a burst of
                              1,201 mixed images ran at 47K, 25K and 13K
                              images/s with 1, 2 and 4)                      */
  int32_t idle_us;         /* persistent mode: CTA idle timeout                */
} fkl_server_config;

typedef struct {
  double t_submit;         /* submit() called                                  */
  double t_admit;          /* slot and memory granted, copies enqueued         */
  double t_ready;          /* work published to the kernel (persistent mode:
                              at once; other modes: copies complete)          */
  double t_done;           /* every output image written                       */
  int32_t n_images;
  int32_t state;           /* 0 queued, 1 copying, 2 running, 3 done           */
} fkl_request_info;

typedef struct {
  uint64_t submitted, admitted, completed, images_completed;
  uint64_t kernel_launches;     /* persistent kernels, or per-request launches */
  uint64_t arena_peak_bytes;    /* high-water mark of the arena                */
  int32_t queued, inflight;     /* right now                                   */
} fkl_server_stats;

typedef struct fkl_server_s* fkl_server;

/* Create: allocates the arena and control blocks, starts the host thread.
 * The pipeline must outlive the server. */
FKL_API fkl_status fkl_server_create(fkl_pipeline p, const fkl_server_config* cfg, fkl_server* out);
/* Submit n host images (HWC u8). Persistent mode: pinned host memory, valid
 * until the request is done (the kernel reads it). Other modes: pinned memory
 * for asynchronous copies, valid until the request's t_ready. Returns at
 * once. */
FKL_API fkl_status fkl_server_submit(fkl_server s, int32_t n, const fkl_tensor* images,
                                     uint64_t* request_id);
/* Non-blocking: *done = 1 once every output of the request is written;
 * `out` (may be NULL) then describes the request's device output
 * [n, 3, H, W] (valid until release). */
FKL_API fkl_status fkl_server_poll(fkl_server s, uint64_t request_id, int32_t* done, fkl_tensor* out);
/* Blocking poll with a timeout; FKL_ERR_TIMEOUT if not done in time. */
FKL_API fkl_status fkl_server_wait(fkl_server s, uint64_t request_id, int32_t timeout_ms, fkl_tensor* out);
/* Times and state of a request (before release). */
FKL_API fkl_status fkl_server_request_info(fkl_server s, uint64_t request_id, fkl_request_info* info);
/* Frees the request's slot and device memory (after it is done). */
FKL_API fkl_status fkl_server_release(fkl_server s, uint64_t request_id);
FKL_API fkl_status fkl_server_get_stats(fkl_server s, fkl_server_stats* st);
/* Stops the host thread and the kernels, waits for in-flight work, frees
 * everything. */
FKL_API void fkl_server_destroy(fkl_server s);

/* ------------------------------------------------------------------------ */
/* Introspection and tuning                                                 */
/* ------------------------------------------------------------------------ */

/* Name of the compiled kernel the pipeline is bound to; the string is owned
 * by the pipeline and valid until fkl_pipeline_destroy. */
FKL_API const char* fkl_pipeline_kernel_name(fkl_pipeline p);

/* Launch shape used by the fused kernel.
 * Image chains: V output pixels per thread along x, a TX x TY thread block
 * (TX * TY <= 256), RY output rows per thread.
 * Float32 tensor chains: `vec` elements per thread and iteration (2, 4, 8,
 * 16 or 32), TX threads per block (TY = 1); RY = 1 runs a persistent grid of
 * (2048 / TX) blocks per SM striding over the tensor, RY = 0 one block per
 * TX * vec elements.
 * NV12 chains with a split output, RY <= 0: the row-staged kernel (paper
 * §IV-C DPP on the bulk-copy engine). Jobs of TY output rows; a persistent
 * grid of TX-thread CTAs copies each job's source rows (two luma rows and one
 * chroma row per output row) into a shared-memory ring of -RY stages (RY = 0:
 * as many as fill about 64 KB) with asynchronous bulk copies and computes
 * from there. It runs when every image of a launch is an
 * exact 2x downscale of a 16-byte aligned window (x offset a multiple of 16,
 * even y offset, pitch a multiple of 16, 16-byte aligned base) that fills the
 * output width, and the output width is a multiple of `vec`; any other launch
 * of the pipeline runs the register kernel with a 32 x 8 block and RY = 1.
 * Packed-image chains, RY = -1 (V <= 4): the tile-staged reader; each block
 * stages the source bytes its tile's taps reference in shared memory before
 * blending (when every image's span fits 48 KB, else the register kernel
 * with a 32 x 8 block and RY = 1).
 * All forms give the same bytes. */
typedef struct {
  int32_t vec;      /* pixels (elements) per thread along x               */
  int32_t tx, ty;   /* threads per block along x and y                    */
  int32_t ry;       /* output rows per thread (image chains)              */
} fkl_launch_shape;

/* Current / set the launch shape. fkl_pipeline_set_shape validates it
 * (FKL_ERR_INVALID if the kernel has no instantiation for it). */
FKL_API fkl_status fkl_pipeline_get_shape(fkl_pipeline p, fkl_launch_shape* shape);
FKL_API fkl_status fkl_pipeline_set_shape(fkl_pipeline p, const fkl_launch_shape* shape);

/* Number of launch shapes the autotuner may try for this pipeline, and the
 * k-th of them (k in [0, count)). */
FKL_API int32_t fkl_pipeline_shape_count(fkl_pipeline p);
FKL_API fkl_status fkl_pipeline_shape_at(fkl_pipeline p, int32_t k,
                                 fkl_launch_shape* shape);

/*
 * Autotuner (tile, coarsening and block shape): runs every launch shape
 * fkl_pipeline_shape_at lists on these arguments -- one warm-up launch, then
 * `reps` (1..32) launches enqueued back to back, each timed with its own pair
 * of CUDA events on `stream` -- then times the shapes within 3% of the
 * fastest median again (at most four, three rounds that visit each in turn,
 * so that a drift in the GPU's speed hits them alike) and keeps the one with
 * the lowest median of its round medians as the pipeline's shape. `best` and
 * `best_us` (median microseconds per launch, may be NULL) report it. Every trial writes `out`. Synchronises `stream`;
 * not capturable in a CUDA graph. A pipeline with a single shape returns it
 * without timing.
 * fkl_pipeline_autotune_ex: the same, but calls `before(user)` on the host
 * before every timed launch, outside its timed interval, so the caller can
 * enqueue the work that precedes a launch in its own steady state (for
 * example an L2 flush, for inputs smaller than L2). `before` may be NULL.
 */
FKL_API fkl_status fkl_pipeline_autotune(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                         const int32_t* rois, fkl_tensor* out, void* stream,
                                         int32_t reps, fkl_launch_shape* best, float* best_us);
FKL_API fkl_status fkl_pipeline_autotune_ex(fkl_pipeline p, int32_t n, const fkl_tensor* ins,
                                            const int32_t* rois, fkl_tensor* out, void* stream,
                                            int32_t reps, void (*before)(void* user), void* user,
                                            fkl_launch_shape* best, float* best_us);

/* Reads and clears the flag the fused kernels' bounded device waits set when
 * one gives up (the row-staged NV12 kernel waits on its own copies; a wait
 * longer than the limit, 1 s by default, stops that CTA, whose outputs are
 * then incomplete).
 * Synchronises the current device first. Returns FKL_ERR_TIMEOUT if the flag
 * was set since the last call on this device, FKL_OK if not, FKL_ERR_CUDA if a
 * CUDA call failed (the message has it). */
FKL_API fkl_status fkl_device_check(void);

/* Limit of one bounded device wait of the fused kernels, for launches made
 * after the call (process-wide). 0 restores the default of 1 s; at most
 * 10 s (FKL_ERR_INVALID above); below 1 us (the device timer's resolution) a
 * wait gives up unless its phase is complete at the first poll. A wait that runs out sets the flag
 * fkl_device_check reads; the kernel still lets its own copies in flight land
 * (a separate, fixed 1 s bound) before it leaves, so a short limit ends work
 * early but leaves the device usable. */
FKL_API fkl_status fkl_set_device_wait_limit(uint64_t ns);

/* Library version string. */
FKL_API const char* fkl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FKL_H_ */
