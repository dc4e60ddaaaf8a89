// Tile-staged resize of packed 3-channel u8 images (the Crop -> Resize ROp
// of the chains of paper §VI-F and §VI-J) under the TransformDPP of §IV-C.
//
// A block owns a tile of (blockDim.x * V) x blockDim.y output pixels of one
// image (blockIdx.z: horizontal fusion, §IV-B). It first stages in shared
// memory exactly the source bytes its bilinear taps reference -- the two tap
// rows of each output row, over the tile's span of tap columns -- with
// 16-byte loads (single bytes at the two ends of a span, so nothing outside
// it is read), then every thread blends its V pixels from shared memory with
// the integer arithmetic of ResizeU8C3T::blend_bytes, so the result is the
// register reader's, bit for bit. The register reader issues twelve byte
// loads per output pixel, scattered over the row; here a warp's loads are
// contiguous 16-byte vectors and the taps come from shared memory.
#pragma once

#include "dpp.cuh"

namespace fkl {

constexpr int kTileMaxRows = 32;  // blockDim.y limit (two staged rows per output row)

template <class RB, class W, class Cops>
struct TileArgs {
  typename RB::ParamsType rp;
  typename W::ParamsType wp;
  Cops cops;
  int32_t H, W_;       // output rows and columns per image
  int32_t row_stride;  // shared bytes per staged tap row: 16 ((span + 30) / 16 + 1) or more
};

template <int V, class RB, class W, class Cops>
__global__ void __launch_bounds__(256) tile_resize_kernel(const __grid_constant__ TileArgs<RB, W, Cops> a) {
  using ROp = typename RB::Op;
  using WT = typename ChainResult<F3, Cops>::type;
  extern __shared__ __align__(16) uint8_t staged[];
  __shared__ int s_row[2 * kTileMaxRows];  // source row of staged row r, -1: not staged
  __shared__ int s_off[2 * kTileMaxRows];  // staged row r holds span byte b at r * stride + s_off[r] + b
  __shared__ int s_wy[kTileMaxRows];       // vertical weight of output row j (units of 1 / (2 dh))
  __shared__ int s_cx0, s_nb;              // first tap column of the tile, bytes per span

  const int z = blockIdx.z;
  if (z >= a.rp.count) return;  // uniform for the block
  const ResampleParams& q = a.rp.p[z];
  const int tile_w = blockDim.x * V;
  const int x0 = blockIdx.x * tile_w, y0 = blockIdx.y * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthreads = blockDim.x * blockDim.y;
  // the tile's columns inside the placed window, in window coordinates
  const int lx_lo = max(x0 - q.ox, 0);
  const int lx_hi = min(min(x0 + tile_w, a.W_) - 1 - q.ox, q.dw - 1);
  const bool any_col = lx_lo <= lx_hi;

  // 1. the tap rows of the tile's output rows and the span of tap columns
  if (tid == 0) {
    if (any_col) {
      s_cx0 = AxisWalker(lx_lo, q.rw, q.dw).tap().i0;
      s_nb = 3 * (AxisWalker(lx_hi, q.rw, q.dw).tap().i1 - s_cx0 + 1);
    } else {
      s_cx0 = 0;
      s_nb = 0;
    }
  }
  __syncthreads();
  if (tid < static_cast<int>(blockDim.y)) {
    const int ly = y0 + tid - q.oy;
    if (any_col && y0 + tid < a.H && ly >= 0 && ly < q.dh) {
      const AxisTap t = AxisWalker(ly, q.rh, q.dh).tap();
      s_row[2 * tid] = q.ry + t.i0;
      s_row[2 * tid + 1] = q.ry + t.i1;
      s_wy[tid] = t.w1;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint8_t* g = q.src + static_cast<int64_t>(s_row[2 * tid + k]) * q.pitch + 3 * (q.rx + s_cx0);
        s_off[2 * tid + k] = static_cast<int>(reinterpret_cast<uintptr_t>(g) & 15);
      }
    } else {
      s_row[2 * tid] = s_row[2 * tid + 1] = -1;
    }
  }
  __syncthreads();

  // 2. stage the spans: chunk c of staged row r is the aligned 16 bytes at
  //    span offset 16 c - off; chunks wholly inside the span are one vector
  //    load, the (at most two) partial ones are read byte by byte
  const int nb = s_nb;
  const int rows = 2 * blockDim.y;
  const int chunks = (nb + 30) / 16 + 1;  // per row, whatever its offset
  for (int i = tid; i < rows * chunks; i += nthreads) {
    const int r = i / chunks, c = i - r * chunks;
    if (s_row[r] < 0) continue;
    const int off = s_off[r];
    const int lo = 16 * c - off;  // span byte of the chunk's first byte
    if (lo >= nb) continue;
    const uint8_t* g = q.src + static_cast<int64_t>(s_row[r]) * q.pitch + 3 * (q.rx + s_cx0) + lo;
    uint8_t* d = staged + r * a.row_stride + 16 * c;
    if (lo >= 0 && lo + 16 <= nb) {
      *reinterpret_cast<uint4*>(d) = __ldg(reinterpret_cast<const uint4*>(g));
    } else {
#pragma unroll
      for (int b = 0; b < 16; ++b)
        if (lo + b >= 0 && lo + b < nb) d[b] = __ldg(g + b);
    }
  }
  __syncthreads();

  // 3. V outputs of this thread's row, from the staged bytes
  const int j = threadIdx.y, y = y0 + j;
  const int xs = x0 + threadIdx.x * V;
  if (y >= a.H || xs >= a.W_) return;
  const int n = min(V, a.W_ - xs);
  const typename W::ParamsType wp = [&] {
    if constexpr (HasPrepare<W>::value) {
      return W::prepare(a.wp);
    } else {
      return a.wp;
    }
  }();
  const bool row_in = s_row[2 * j] >= 0;
  // staged index of source column 0 in the two tap rows (tap columns below
  // the span's first are never read)
  const int b0 = row_in ? (2 * j) * a.row_stride + s_off[2 * j] - 3 * s_cx0 : 0;
  const int b1 = row_in ? (2 * j + 1) * a.row_stride + s_off[2 * j + 1] - 3 * s_cx0 : 0;
  AxisTap ty;
  ty.w1 = row_in ? s_wy[j] : 0;
  const int lx0 = xs - q.ox;
  AxisWalker wx(max(lx0, 0), q.rw, q.dw);
  WT out[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (k < n) {
      const int lx = lx0 + k;
      F3 v;
      if (!row_in || lx < 0 || lx >= q.dw) {
        v = F3{{q.pad, q.pad, q.pad}};
      } else {
        const AxisTap tx = wx.tap();
        uint32_t s[4][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s[0][c] = staged[b0 + 3 * tx.i0 + c];
          s[1][c] = staged[b0 + 3 * tx.i1 + c];
          s[2][c] = staged[b1 + 3 * tx.i0 + c];
          s[3][c] = staged[b1 + 3 * tx.i1 + c];
        }
        v = ROp::blend_bytes(s, tx, 2 * q.dw, ty, 2 * q.dh, q.inv_area);
        wx.next();
      }
      out[k] = apply_chain(v, a.cops);
    }
  }
  W::template exec_span<V>(Point{xs, y, z}, n, out, wp);
}

}  // namespace fkl
