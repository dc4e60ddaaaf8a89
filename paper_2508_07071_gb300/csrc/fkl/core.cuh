// Core vocabulary of the Fused Kernel template library.
//
// An Operation (Op) is a stateless struct with one static __device__ exec
// function whose signature depends on its InstanceType (paper §IV-A/§IV-B,
// Table I):
//   ReadType   : OutputType exec(const Point&, const ParamsType&)
//   UnaryType  : OutputType exec(const InputType&)
//   BinaryType : OutputType exec(const InputType&, const ParamsType&)
//   WriteType  : void       exec(const Point&, const InputType&, const ParamsType&)
// An instantiable Op (IOp, paper §IV-A Fig. 7) pairs an Op type with the
// runtime parameters it needs; the chain of IOps is expanded at compile time
// into straight-line code (paper §IV-A Fig. 8, §IV-C), so intermediates never
// leave registers.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#define FKL_HD __host__ __device__ __forceinline__
#define FKL_D __device__ __forceinline__

namespace fkl {

// Images per launch of the batched image kernels: the capacity of their
// per-image parameter table (horizontal fusion, paper §IV-B BatchRead).
constexpr int kBatchCap = 256;

// ---------------------------------------------------------------------------
// Instance types (static reflection tags, paper §IV-C)
// ---------------------------------------------------------------------------
struct ReadType {};
struct UnaryType {};
struct BinaryType {};
struct WriteType {};

// Thread coordinates given to Memory Operations: x = output column,
// y = output row, z = batch index (blockIdx.z under horizontal fusion).
struct Point {
  int x;
  int y;
  int z;
};

// A pixel of C channels held in registers, channels in memory order.
template <typename T, int C>
struct Pix {
  T v[C];
};
using F3 = Pix<float, 3>;
using U3 = Pix<uint8_t, 3>;

// ---------------------------------------------------------------------------
// Instantiable Operations (paper §IV-A Fig. 7: UIOp / BIOp; §IV-B RIOp/WIOp)
// ---------------------------------------------------------------------------
template <class Op, class Kind = typename Op::InstanceType>
struct IOp {
  using Operation = Op;
  typename Op::ParamsType params;
};
template <class Op>
struct IOp<Op, UnaryType> {
  using Operation = Op;
};

// ---------------------------------------------------------------------------
// A minimal device tuple to carry the COp instances by value.
// ---------------------------------------------------------------------------
template <class... Ts>
struct Tuple;
template <>
struct Tuple<> {};
template <class H, class... Ts>
struct Tuple<H, Ts...> {
  H head;
  Tuple<Ts...> tail;
};

FKL_HD Tuple<> make_tuple() { return {}; }
template <class H, class... Ts>
FKL_HD Tuple<H, Ts...> make_tuple(const H& h, const Ts&... xs) {
  return Tuple<H, Ts...>{h, make_tuple(xs...)};
}

// (h, t...) from h and the tuple (t...).
template <class H, class... Ts>
FKL_HD Tuple<H, Ts...> prepend(const H& h, const Tuple<Ts...>& t) {
  return Tuple<H, Ts...>{h, t};
}

// Apply one compute IOp, choosing the exec form from its InstanceType at
// compile time (paper §IV-C, "if constexpr" on InstanceType).
template <class I, class T>
FKL_D auto apply_one(const I& iop, const T& v) {
  using Op = typename I::Operation;
  if constexpr (std::is_same_v<typename Op::InstanceType, UnaryType>) {
    return Op::exec(v);
  } else {
    static_assert(std::is_same_v<typename Op::InstanceType, BinaryType>,
                  "only Unary and Binary ops may sit between the ROp and the WOp");
    return Op::exec(v, iop.params);
  }
}

// Left-to-right application of every COp (the variadic recursion of paper
// §IV-A Fig. 8); the compiler sees one straight-line scope.
template <class T>
FKL_D T apply_chain(const T& v, const Tuple<>&) {
  return v;
}
template <class T, class H, class... Ts>
FKL_D auto apply_chain(const T& v, const Tuple<H, Ts...>& t) {
  return apply_chain(apply_one(t.head, v), t.tail);
}

// Pair form of a chain (see F3x2 in ops.cuh): available when every COp has
// an exec_pair; the DPP then runs the chain on two pixels per instruction.
template <class I, class = void>
struct HasPair : std::false_type {};
template <class I>
struct HasPair<I, std::void_t<decltype(&I::Operation::exec_pair)>> : std::true_type {};

template <class Tup>
struct ChainHasPair;
template <>
struct ChainHasPair<Tuple<>> : std::true_type {};
template <class H, class... Ts>
struct ChainHasPair<Tuple<H, Ts...>> {
  static constexpr bool value = HasPair<H>::value && ChainHasPair<Tuple<Ts...>>::value;
};

template <class P>
FKL_D P apply_chain_pair(const P& v, const Tuple<>&) {
  return v;
}
template <class P, class H, class... Ts>
FKL_D P apply_chain_pair(const P& v, const Tuple<H, Ts...>& t) {
  using Op = typename H::Operation;
  if constexpr (std::is_same_v<typename Op::InstanceType, UnaryType>) {
    return apply_chain_pair(Op::exec_pair(v), t.tail);
  } else {
    return apply_chain_pair(Op::exec_pair(v, t.head.params), t.tail);
  }
}

// Result type of a chain of COps applied to T.
template <class T, class Tup>
struct ChainResult;
template <class T>
struct ChainResult<T, Tuple<>> {
  using type = T;
};
template <class T, class H, class... Ts>
struct ChainResult<T, Tuple<H, Ts...>> {
  using type = typename ChainResult<typename H::Operation::OutputType, Tuple<Ts...>>::type;
};

// ---------------------------------------------------------------------------
// Output number formats. Conversions use the hardware cvt instructions
// (round to nearest even; FP8 saturates to the largest finite value).
// ---------------------------------------------------------------------------
struct bf16_t {
  uint16_t bits;
};
struct f16_t {
  uint16_t bits;
};
struct e4m3_t {
  uint8_t bits;
};

// Two floats -> packed pair; `lo` lands in the low half.
FKL_D uint32_t pack2_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
FKL_D uint32_t pack2_f16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
FKL_D uint32_t pack2_e4m3(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return static_cast<uint32_t>(r);
}

// ---------------------------------------------------------------------------
// Packed float pairs: two independent IEEE binary32 lanes per instruction
// (add/mul/fma .rn .f32x2, sm_100 and later). Each lane rounds exactly like
// the scalar __fadd_rn/__fmul_rn/__fmaf_rn, so packed and scalar code give
// the same bits.
// ---------------------------------------------------------------------------
struct F2 {
  unsigned long long v;
};
FKL_D F2 f2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
FKL_D F2 f2s(float x) { return f2(x, x); }
FKL_D void f2split(F2 a, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v)); }
FKL_D F2 f2add(F2 a, F2 b) {
  F2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
FKL_D F2 f2sub(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
FKL_D F2 f2mul(F2 a, F2 b) {
  F2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
FKL_D F2 f2fma(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}

template <class OutT>
struct Format;
template <>
struct Format<float> {
  static constexpr int bytes = 4;
};
template <>
struct Format<bf16_t> {
  static constexpr int bytes = 2;
};
template <>
struct Format<f16_t> {
  static constexpr int bytes = 2;
};
template <>
struct Format<e4m3_t> {
  static constexpr int bytes = 1;
};
template <>
struct Format<uint8_t> {
  static constexpr int bytes = 1;
};

// Store V consecutive values of one plane (V * bytes must be 4, 8, 16, 32
// or 64); `p` must be aligned to min(16, V * bytes). Floats are already
// scaled (FP8) by the caller.
template <class OutT, int V>
FKL_D void store_run(void* p, const float (&x)[V]);

template <int V>
FKL_D void store_words(void* p, const uint32_t (&w)[V]) {
  static_assert(V == 1 || V == 2 || V % 4 == 0, "unsupported run length");
  if constexpr (V == 1) {
    *reinterpret_cast<uint32_t*>(p) = w[0];
  } else if constexpr (V == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      __stcs(reinterpret_cast<uint4*>(p) + i / 4, make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]));
    }
  }
}

template <class OutT, int V>
FKL_D void store_run(void* p, const float (&x)[V]) {
  if constexpr (std::is_same_v<OutT, float>) {
    uint32_t w[V];
#pragma unroll
    for (int i = 0; i < V; ++i) w[i] = __float_as_uint(x[i]);
    store_words<V>(p, w);
  } else if constexpr (std::is_same_v<OutT, bf16_t> || std::is_same_v<OutT, f16_t>) {
    static_assert(V % 2 == 0, "16-bit runs need an even length");
    uint32_t w[V / 2];
#pragma unroll
    for (int i = 0; i < V / 2; ++i) {
      w[i] = std::is_same_v<OutT, bf16_t> ? pack2_bf16(x[2 * i], x[2 * i + 1])
                                          : pack2_f16(x[2 * i], x[2 * i + 1]);
    }
    store_words<V / 2>(p, w);
  } else if constexpr (std::is_same_v<OutT, e4m3_t>) {
    static_assert(V % 4 == 0, "FP8 runs need a multiple of 4");
    uint32_t w[V / 4];
#pragma unroll
    for (int i = 0; i < V / 4; ++i) {
      w[i] = pack2_e4m3(x[4 * i], x[4 * i + 1]) | (pack2_e4m3(x[4 * i + 2], x[4 * i + 3]) << 16);
    }
    store_words<V / 4>(p, w);
  } else {
    static_assert(sizeof(OutT) == 0, "unsupported output type");
  }
}

// Scalar store of one value (ragged tails, unaligned outputs).
template <class OutT>
FKL_D void store_one(void* p, float x) {
  if constexpr (std::is_same_v<OutT, float>) {
    *reinterpret_cast<float*>(p) = x;
  } else if constexpr (std::is_same_v<OutT, bf16_t>) {
    *reinterpret_cast<uint16_t*>(p) = static_cast<uint16_t>(pack2_bf16(x, 0.f) & 0xFFFFu);
  } else if constexpr (std::is_same_v<OutT, f16_t>) {
    *reinterpret_cast<uint16_t*>(p) = static_cast<uint16_t>(pack2_f16(x, 0.f) & 0xFFFFu);
  } else if constexpr (std::is_same_v<OutT, e4m3_t>) {
    *reinterpret_cast<uint8_t*>(p) = static_cast<uint8_t>(pack2_e4m3(x, 0.f) & 0xFFu);
  } else {
    static_assert(sizeof(OutT) == 0, "unsupported output type");
  }
}

}  // namespace fkl
