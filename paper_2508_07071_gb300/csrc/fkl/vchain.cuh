#pragma once

#include "core.cuh"

namespace fkl {

// ---------------------------------------------------------------------------
// Linear TransformDPP for 1-D float tensors (the vertical Mul/Add chain of
// paper §VI-B/§VI-G). The chain is a table of constants plus a bitmask of op
// kinds held in the kernel parameters; each thread keeps E elements (2 or a
// multiple of 4, loaded as one float2 or as float4 vectors) in registers
// and applies every op to all of them before the next op, so the dependent
// chain of one element is interleaved with E - 1 independent ones.
// ---------------------------------------------------------------------------
template <int CAP>
struct VChainParams {
  const void* in;  // float32, or u8 converted exactly
  float* out;
  int64_t n;          // elements
  int32_t len;        // ops in this launch (<= CAP)
  int32_t alternating;  // 1: kinds are Mul, Add, Mul, Add, ... from op 0
  uint32_t add_mask[(CAP + 31) / 32];  // bit i set: op i is an Add
  alignas(16) float c[CAP];            // two Mul/Add pairs are read as one 16-byte vector
};

// E consecutive input elements as floats (vector loads when `vec`).
template <class InT, int E>
FKL_D void vchain_load(const void* in, int64_t base, int64_t n, bool vec, float (&x)[E]) {
  if constexpr (std::is_same_v<InT, float>) {
    const float* f = static_cast<const float*>(in);
    if constexpr (E == 2) {
      if (vec) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(f + base));
        x[0] = v.x;
        x[1] = v.y;
        return;
      }
    }
    if (vec && E % 4 == 0) {
#pragma unroll
      for (int u = 0; u < E / 4; ++u) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(f + base) + u);
        x[4 * u] = v.x;
        x[4 * u + 1] = v.y;
        x[4 * u + 2] = v.z;
        x[4 * u + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = base + e < n ? f[base + e] : 0.f;
    }
  } else {
    static_assert(std::is_same_v<InT, uint8_t> && (E == 2 || E == 4 || E % 8 == 0),
                  "u8 chains load 2, 4 or 8-byte multiples");
    const uint8_t* b = static_cast<const uint8_t*>(in);
    if (vec) {
      uint32_t w[(E + 3) / 4];
      if constexpr (E == 2) {
        w[0] = __ldcs(reinterpret_cast<const unsigned short*>(b + base));
      } else if constexpr (E == 4) {
        w[0] = __ldcs(reinterpret_cast<const unsigned int*>(b + base));
      } else if constexpr (E == 8) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(b + base));
        w[0] = v.x;
        w[1] = v.y;
      } else {
#pragma unroll
        for (int u = 0; u < E / 16; ++u) {
          const uint4 v = __ldcs(reinterpret_cast<const uint4*>(b + base) + u);
          w[4 * u] = v.x;
          w[4 * u + 1] = v.y;
          w[4 * u + 2] = v.z;
          w[4 * u + 3] = v.w;
        }
      }
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = static_cast<float>((w[e / 4] >> (8 * (e % 4))) & 0xFFu);
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = base + e < n ? static_cast<float>(b[base + e]) : 0.f;
    }
  }
}

// One Mul, Add pair on the thread's E elements: fl(fl(x * cm) + ca).
template <int E>
FKL_D void vchain_pair(float (&x)[E], float cm, float ca) {
  const F2 m = f2s(cm);
#pragma unroll
  for (int e = 0; e < E; e += 2) {
    float lo, hi;
    f2split(f2mul(f2(x[e], x[e + 1]), m), lo, hi);
    x[e] = __fadd_rn(lo, ca);
    x[e + 1] = __fadd_rn(hi, ca);
  }
}

template <int E, int CAP, bool kAlt, class InT = float>
__global__ void __launch_bounds__(512) vchain_kernel(const __grid_constant__ VChainParams<CAP> p) {
  static_assert(E == 2 || E % 4 == 0, "2 or a multiple of 4 elements per thread");
  constexpr int kInBytes = static_cast<int>(sizeof(InT));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * E;
  for (int64_t base = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * E; base < p.n;
       base += stride) {
    float x[E];
    const bool full = base + E <= p.n && (reinterpret_cast<uintptr_t>(p.in) % (kInBytes * E < 16 ? kInBytes * E : 16)) == 0 &&
                      (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
    vchain_load<InT, E>(p.in, base, p.n, full, x);
    if constexpr (kAlt) {
      // Mul, Add pairs: no per-op branch; two pairs' four constants come in
      // one 16-byte load (one 8-byte load per pair ran 8% slower on a
      // 360,000-element batch), and sixteen pairs per loop trip amortise
      // the loop (eight: 2% slower). The Mul runs on two elements
      // per packed f32x2 multiply and the Add on scalar adds: three FP32
      // issue slots per two elements and pair instead of four, for the same
      // FP32 lane work, so the constant loads and the loop fit beside the
      // FP32 pipe. (A packed multiply feeding a packed add is contracted into
      // a multiply-add by the assembler, which rounds once where the chain
      // rounds twice; with either side scalar it is not.)
      int i = 0;
#pragma unroll 8
      for (; i + 3 < p.len; i += 4) {
        const float4 cc = *reinterpret_cast<const float4*>(&p.c[i]);  // i % 4 == 0: 16-byte aligned
        vchain_pair<E>(x, cc.x, cc.y);
        vchain_pair<E>(x, cc.z, cc.w);
      }
      for (; i + 1 < p.len; i += 2) {
        const float2 cc = *reinterpret_cast<const float2*>(&p.c[i]);  // i is even: 8-byte aligned
        vchain_pair<E>(x, cc.x, cc.y);
      }
      if (i < p.len) {
        const float cm = p.c[i];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], cm);
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < p.len; ++i) {
        const float c = p.c[i];
        if ((p.add_mask[i >> 5] >> (i & 31)) & 1u) {
#pragma unroll
          for (int e = 0; e < E; ++e) x[e] = __fadd_rn(x[e], c);
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) x[e] = __fmul_rn(x[e], c);
        }
      }
    }
    if (full) {
      if constexpr (E == 2) {
        __stcs(reinterpret_cast<float2*>(p.out + base), make_float2(x[0], x[1]));
      } else {
#pragma unroll
        for (int u = 0; u < E / 4; ++u)
          __stcs(reinterpret_cast<float4*>(p.out + base) + u,
                 make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]));
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (base + e < p.n) p.out[base + e] = x[e];
    }
  }
}

}  // namespace fkl
