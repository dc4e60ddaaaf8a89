#pragma once

#include "ops.cuh"

namespace fkl {

// ---------------------------------------------------------------------------
// ReduceDPP (paper §IV-C, the reduction pattern): several reductions of a
// chain's values from one read -- per-channel minimum, maximum and sum; the
// maximum absolute value follows from the extremes.
//
// The COps of the float chains (channel swap, Mul, Sub/Add, Div by per-
// channel constants) act on each channel as one monotone map f, rounded at
// every op: f(x) = fl(fl(fl(x * m) - s) / d). Rounding is monotone, so the
// extremes of f over a set of read values are f of the read values'
// extremes, exactly (f non-decreasing for m d > 0, non-increasing otherwise);
// and f is affine, so the mean of f is f of the mean, up to the rounding of
// the per-pixel values. The kernel therefore reduces the ROp's values only,
// over the placed window of every image (the fill around it is one known
// value, counted on the host), and the finishing block maps the statistics
// through the COps once. The extremes are the same floats the TransformDPP
// writes.
//
// A persistent grid of blocks, each walking a contiguous range of jobs of
// blockDim.y window rows x blockDim.x * V window columns of one image. On the NV12 exact-2x span each
// pixel pair's tap sums (fl(fl(u00 + u10) + fl(u01 + u11)) per channel, the
// read's value before its exact-scale multiply by 63.75) are folded at once:
// three-input min/max and a packed f32x2 partial sum per job; the read value
// of an extreme is fl(S * 63.75), monotone in S. Other spans fold read values
// pixel by pixel. Every job's partial sums become 64-bit fixed point (2^-10
// read units), min/max travel as order-preserving unsigned keys, so the
// result does not depend on the grid or on the order in which blocks finish.
// The last block of a call to finish (a counter over every launch of the
// call) maps the accumulator into the statistics, so a call is one memset
// of the accumulator and one launch per 256 images.
// ---------------------------------------------------------------------------
struct ReduceAcc {
  unsigned int min_inv[3];       // per channel, ~(order key) of the ROp's minimum: the maximum
                                 // of the inverted keys, so that zero is the identity
  unsigned int max_key[3];       // order key of the maximum
  unsigned long long sum_fx[3];  // fixed point, 2^-10 read units
  unsigned int done;             // blocks finished, over every launch of one call
};
// Sums: every job's float32 partial sum (of at most 16 values below 256,
// or 16 tap sums below 4) is scaled to 2^-10 read units -- below 2^22 --
// and rounded to an integer by the float32 magic-number addition
// (x + 1.5 * 2^23 puts round(x) in the mantissa: an FP32 add and an integer
// subtract, where a float -> int64 conversion would take the slow FP64 pipe).
constexpr float kSumScale = 1024.f;               // 2^10
constexpr float kSum2xScale = 63.75f * 1024.f;    // tap sums to fixed-point read units (exact)
constexpr float kRoundMagic = 12582912.f;         // 1.5 * 2^23

// round(x) for 0 <= x < 2^22, exactly (round to nearest even).
FKL_D int round_small(float x) { return __float_as_int(__fadd_rn(x, kRoundMagic)) - 0x4B400000; }

FKL_D unsigned int order_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
FKL_D float key_value(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

FKL_D float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
FKL_D float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// The chain's statistics from the ROp's (paper §IV-C: the COps applied to
// the reduced values). Per output channel c the read channel is c, or 2 - c
// after a BGR <-> RGB swap; the fill (letterbox) value joins the extremes
// and the sum when the output has fill pixels.
struct ReduceChain {
  int32_t swap;
  int32_t has_div;
  float mul[3], sub[3], div[3];
  float pad;
};

FKL_D float apply_reduce_chain(const ReduceChain& ch, int c, float x) {
  x = __fmul_rn(x, ch.mul[c]);
  x = __fsub_rn(x, ch.sub[c]);
  return ch.has_div ? __fdiv_rn(x, ch.div[c]) : x;
}

// What the block that completes a call needs to write the statistics.
struct ReduceFinal {
  float* stats;
  double count;       // output pixels per channel
  double fill_count;  // of them, fill pixels (the pad value)
  ReduceChain chain;
  int32_t jobs, grid;  // the work split reported in the statistics
  uint32_t blocks;     // blocks of all the call's reduction launches
};

// The statistics of include/fkl.h from the accumulator (one thread). Reads
// go through volatile loads: the other blocks' atomics are in L2.
FKL_D void reduce_finish(const ReduceAcc* acc_in, const ReduceFinal& f) {
  const volatile ReduceAcc* acc = acc_in;
  float* stats = f.stats;
  const ReduceChain& ch = f.chain;
  float amax = 0.f;
  for (int c = 0; c < 3; ++c) {
    const int rc = ch.swap ? 2 - c : c;  // the read channel output channel c comes from
    float lo = key_value(~acc->min_inv[rc]);
    float hi = key_value(acc->max_key[rc]);
    if (f.fill_count > 0) {
      lo = fminf(lo, ch.pad);
      hi = fmaxf(hi, ch.pad);
    }
    const float a = apply_reduce_chain(ch, c, lo), b = apply_reduce_chain(ch, c, hi);
    stats[c] = f.count > 0 ? fminf(a, b) : __int_as_float(0x7fc00000);
    stats[3 + c] = f.count > 0 ? fmaxf(a, b) : __int_as_float(0x7fc00000);
    // the mean: the chain's affine map of the read values' mean, in float64
    const double sum = static_cast<double>(static_cast<long long>(acc->sum_fx[rc])) / kSumScale +
                       f.fill_count * static_cast<double>(ch.pad);
    double m = f.count > 0 ? sum / f.count : 0.0;
    m = (m * ch.mul[c] - ch.sub[c]) / (ch.has_div ? static_cast<double>(ch.div[c]) : 1.0);
    stats[6 + c] = f.count > 0 ? static_cast<float>(m) : 0.f;
    // the largest magnitude is that of a channel's minimum or maximum
    if (f.count > 0) amax = fmaxf(amax, fmaxf(fabsf(stats[c]), fabsf(stats[3 + c])));
  }
  stats[9] = amax;
  const float s = amax > 0.f ? __fdiv_rn(amax, 448.f) : 1.f;  // E4M3 per-tensor scale
  stats[10] = s;
  stats[11] = __fdiv_rn(1.f, s);
  reinterpret_cast<int32_t*>(stats)[12] = f.jobs;
  reinterpret_cast<int32_t*>(stats)[13] = f.grid;
}

template <class RB>
struct ReduceArgs {
  typename RB::ParamsType rp;
  int32_t col_tiles;  // jobs per window row band: ceil(ceil(max dw / V) / blockDim.x)
  int32_t row_tiles;  // row bands per image: ceil(max dh / blockDim.y)
  ReduceAcc* acc;
  ReduceFinal fin;
};

// A thread's running statistics on the exact-2x span: extremes of the tap
// sums S and the fixed-point sum in read units. (Other spans fold into the
// block's shared-memory accumulator, see ReduceShared.)
struct ReduceThread {
  float s_min[3], s_max[3];
  long long fx[3];
};

// The block's accumulator for spans off the 2x path: read values folded
// with shared-memory atomics (order keys; fixed-point sums).
struct ReduceShared {
  unsigned int min_key[3], max_key[3];
  unsigned long long sum_fx[3];
};

template <class ROp>
struct HasPairSums2x : std::integral_constant<bool, std::is_same_v<ROp, ResizeNV12> ||
                                                        std::is_same_v<ROp, ResizeNV12x2>> {};

// Where a job puts a thread: window column lx, window row ly of image z;
// `in`: inside the image's window; `fast`: the whole span takes the 2x path.
struct ReduceSpan {
  int lx, ly, z;
  bool in, fast;
};

// A job's position as (image, row band, column tile), column tile fastest;
// advanced one job at a time with carries (no division in the job loop).
struct JobPos {
  int z, band, tile;
  FKL_D void next(int col_tiles, int row_tiles) {
    if (++tile == col_tiles) {
      tile = 0;
      if (++band == row_tiles) {
        band = 0;
        ++z;
      }
    }
  }
};

template <int V, class RB>
FKL_D ReduceSpan reduce_locate(const ReduceArgs<RB>& a, const JobPos& j) {
  ReduceSpan sp;
  sp.z = j.z;
  sp.lx = (j.tile * blockDim.x + threadIdx.x) * V;
  sp.ly = j.band * blockDim.y + threadIdx.y;
  const ResampleParams& q = a.rp.p[sp.z];
  sp.in = sp.lx < q.dw && sp.ly < q.dh;
  sp.fast = false;
  if constexpr (HasPairSums2x<typename RB::Op>::value && V % 8 == 0)
    sp.fast = sp.in && sp.lx + V <= q.dw && ResizeNV12::fast2x<V>(q, sp.lx, sp.ly);
  return sp;
}

// Folds the tap sums of one 2x span (its 16-byte words) into the thread's statistics.
template <int V>
FKL_D void reduce_fold2x(const uint4 (&wa)[V / 8], const uint4 (&wb)[V / 8], const uint4 (&wc)[V / 8],
                         ReduceThread& t) {
  F2 ps[3] = {f2s(0.f), f2s(0.f), f2s(0.f)};
#pragma unroll
  for (int k = 0; k < V; k += 2) {
    const int vi = k / 8, wi = (k % 8) / 2;
    F2 sum[3];
    ResizeNV12::pair_sums2x(reinterpret_cast<const uint32_t*>(&wa[vi])[wi],
                            reinterpret_cast<const uint32_t*>(&wb[vi])[wi],
                            reinterpret_cast<const uint32_t*>(&wc[vi])[wi], sum);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s0, s1;
      f2split(sum[c], s0, s1);
      t.s_min[c] = min3f(t.s_min[c], s0, s1);
      t.s_max[c] = max3f(t.s_max[c], s0, s1);
      ps[c] = f2add(ps[c], sum[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float p0, p1;
    f2split(ps[c], p0, p1);
    t.fx[c] += round_small(__fmul_rn(__fadd_rn(p0, p1), kSum2xScale));
  }
}

// A span off the 2x path, pixel by pixel (the read's own value), into the
// block's shared accumulator.
template <int V, class RB>
FKL_D void reduce_slow(const ReduceArgs<RB>& a, const ReduceSpan& sp, ReduceShared& sh) {
  const ResampleParams& q = a.rp.p[sp.z];
  const int n = min(V, q.dw - sp.lx);
  float lo[3], hi[3], ps[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    lo[c] = __int_as_float(0x7f800000);
    hi[c] = -__int_as_float(0x7f800000);
    ps[c] = 0.f;
  }
  for (int k = 0; k < n; ++k) {
    const F3 v = RB::Op::exec(Point{q.ox + sp.lx + k, q.oy + sp.ly, sp.z}, q);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], v.v[c]);
      hi[c] = fmaxf(hi[c], v.v[c]);
      ps[c] = __fadd_rn(ps[c], v.v[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    atomicMin(&sh.min_key[c], order_key(lo[c]));
    atomicMax(&sh.max_key[c], order_key(hi[c]));
    atomicAdd(&sh.sum_fx[c], static_cast<unsigned long long>(round_small(__fmul_rn(ps[c], kSumScale))));
  }
}

template <int V, class RB>
FKL_D void reduce2d_body(const ReduceArgs<RB>& a) {
  __shared__ ReduceShared sh;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < 3) {
    sh.min_key[tid] = 0xFFFFFFFFu;
    sh.max_key[tid] = 0u;
    sh.sum_fx[tid] = 0ull;
  }
  __syncthreads();
  ReduceThread t;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    t.s_min[c] = __int_as_float(0x7f800000);
    t.s_max[c] = -__int_as_float(0x7f800000);
    t.fx[c] = 0;
  }
  // jobs in (image, row band, column tile) order over the window; block b
  // takes the contiguous range [b J / G, (b + 1) J / G) of the J jobs. The
  // words of the block's next job are loaded before the current job is
  // folded, so every thread keeps one job's loads in flight while it computes.
  const int per_image = a.col_tiles * a.row_tiles;
  const long long jobs = static_cast<long long>(per_image) * a.rp.count;
  const int first = static_cast<int>(jobs * blockIdx.x / gridDim.x);
  const int last = static_cast<int>(jobs * (blockIdx.x + 1) / gridDim.x);
  JobPos pos;
  pos.z = first / per_image;
  pos.band = (first - pos.z * per_image) / a.col_tiles;
  pos.tile = first - pos.z * per_image - pos.band * a.col_tiles;
  ReduceSpan cur{0, 0, 0, false, false};
  uint4 wa[V / 8], wb[V / 8], wc[V / 8];
  if (first < last) {
    cur = reduce_locate<V>(a, pos);
    if constexpr (HasPairSums2x<typename RB::Op>::value && V % 8 == 0)
      if (cur.fast) ResizeNV12::load2x<V>(a.rp.p[cur.z], cur.lx, cur.ly, wa, wb, wc);
  }
  for (int job = first; job < last; ++job) {
    ReduceSpan nxt{0, 0, 0, false, false};
    uint4 na[V / 8], nb[V / 8], nc[V / 8];
    if (job + 1 < last) {
      pos.next(a.col_tiles, a.row_tiles);
      nxt = reduce_locate<V>(a, pos);
      if constexpr (HasPairSums2x<typename RB::Op>::value && V % 8 == 0)
        if (nxt.fast) ResizeNV12::load2x<V>(a.rp.p[nxt.z], nxt.lx, nxt.ly, na, nb, nc);
    }
    if (cur.fast) {
      if constexpr (HasPairSums2x<typename RB::Op>::value && V % 8 == 0) reduce_fold2x<V>(wa, wb, wc, t);
    } else if (cur.in) {
      reduce_slow<V>(a, cur, sh);
    }
    cur = nxt;
#pragma unroll
    for (int i = 0; i < V / 8; ++i) {
      wa[i] = na[i];
      wb[i] = nb[i];
      wc[i] = nc[i];
    }
  }
  // the extremes in read units: fl(S * 63.75) is monotone in S
  unsigned int kmin[3], kmax[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    kmin[c] = order_key(__fmul_rn(t.s_min[c], 63.75f));
    kmax[c] = order_key(__fmul_rn(t.s_max[c], 63.75f));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      kmin[c] = min(kmin[c], __shfl_xor_sync(0xffffffffu, kmin[c], off));
      kmax[c] = max(kmax[c], __shfl_xor_sync(0xffffffffu, kmax[c], off));
      t.fx[c] += __shfl_xor_sync(0xffffffffu, t.fx[c], off);
    }
  }
  const int lane = tid & 31;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(&sh.min_key[c], kmin[c]);
      atomicMax(&sh.max_key[c], kmax[c]);
      atomicAdd(&sh.sum_fx[c], static_cast<unsigned long long>(t.fx[c]));
    }
  }
  __syncthreads();
  if (tid < 3) {
    atomicMax(&a.acc->min_inv[tid], ~sh.min_key[tid]);
    atomicMax(&a.acc->max_key[tid], sh.max_key[tid]);
    atomicAdd(&a.acc->sum_fx[tid], sh.sum_fx[tid]);
    __threadfence();  // this block's totals before its count below
  }
  __syncthreads();
  // the block that completes the call's count writes the statistics
  if (tid == 0 && atomicAdd(&a.acc->done, 1u) + 1u == a.fin.blocks) {
    __threadfence();
    reduce_finish(a.acc, a.fin);
  }
}

// kMinBlocks > 0 caps the registers so that that many 256-thread blocks are
// resident per SM; 0 keeps the compiler's choice.
template <int V, int kMinBlocks, class RB>
__global__ void __launch_bounds__(256, kMinBlocks > 0 ? kMinBlocks : 1)
    reduce2d_kernel(const __grid_constant__ ReduceArgs<RB> a) {
  reduce2d_body<V>(a);
}

}  // namespace fkl
