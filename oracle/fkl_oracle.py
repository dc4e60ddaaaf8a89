"""CPU oracle for the fused preprocessing path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module. The library itself never calls it and has
no CPU fallback.

What it computes
----------------
The Fused Kernel method (paper §II, §IV) promises the *same* result as running
each library function as its own kernel, only without the DRAM round trips:
vertical fusion keeps intermediates in registers (§II, Fig. 3) and horizontal
fusion runs independent images in one launch (§II, Fig. 5, §IV-B BatchRead).
So the oracle is that plain definition: every operation is one numpy step over
a whole image, every intermediate is materialised as float64, and the ops run
in the user's order, ROp -> COp* -> WOp (§IV-C, TransformDPP).

The paper prints no numerics for its ops; where it is silent the readings used
here are:
  * bilinear resize with half-pixel centres, sample clamped to the source
    (the OpenCV INTER_LINEAR convention the cvGS wrapper imitates, §V);
    resize works on the crop as if it had been materialised, and on the u8
    values promoted to float without rounding in between (the NPP chain of
    §VI-J/§VI-L converts the crop to 32F before resizing);
  * NV12 -> RGB is BT.601 limited range, U then V byte order, nearest
    (co-sited) chroma, each component clamped to [0, 255];
  * letterbox: uniform scale r = min(W_out/W, H_out/H), resized size
    floor(W*r + 0.5) x floor(H*r + 0.5), centred with the odd pixel of padding
    at the bottom/right, pad value given in u8 units before any scaling;
  * output casts round to nearest even; FP8-E4M3 divides by a per-tensor scale
    and saturates to +-448;
  * saturating u8 arithmetic clamps the exact integer result; float -> u8
    rounds half to even then clamps;
  * the vertical Mul/Add chain (§VI-B) is evaluated in float32 in chain order,
    every op rounded on its own (no multiply-add contraction);
  * the typed chains of the data-type experiment (§VI-I: Read -> Cast ->
    Multiply -> Subtract -> Divide -> Write) cast the input to the output
    type and run every op in that type, each rounded on its own.

Functions that no test pins against something other than themselves say
"parity unpinned" in their docstring; at present there are none.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# Read Operations (§IV-B, Table I "ReadType", Fig. 9)
# ----------------------------------------------------------------------------


def crop(img: np.ndarray, x: int, y: int, w: int, h: int) -> np.ndarray:
    """Crop ROp (§IV-B, Fig. 9; used in the chains of §VI-F and §VI-J).

    Returns the w x h window whose top-left source pixel is (x, y). The
    window must lie inside the image.
    """
    H, W = img.shape[:2]
    if not (0 <= x and 0 <= y and w > 0 and h > 0 and x + w <= W and y + h <= H):
        raise ValueError(f"crop ({x},{y},{w},{h}) outside {W}x{H}")
    return img[y:y + h, x:x + w]


def to_float(img: np.ndarray) -> np.ndarray:
    """Promote u8 (or any) samples to float64 without rounding."""
    return img.astype(np.float64)


def _bilinear_axis(n_src: int, n_dst: int):
    """Half-pixel sample positions along one axis.

    u = (d + 0.5) * n_src / n_dst - 0.5, clamped to [0, n_src - 1];
    i0 = floor(u), i1 = min(i0 + 1, n_src - 1), weight of i1 = u - i0.
    """
    d = np.arange(n_dst, dtype=np.float64)
    u = (d + 0.5) * (n_src / n_dst) - 0.5
    u = np.clip(u, 0.0, n_src - 1)
    i0 = np.floor(u).astype(np.int64)
    i1 = np.minimum(i0 + 1, n_src - 1)
    return i0, i1, u - i0


def resize_bilinear(img: np.ndarray, out_w: int, out_h: int) -> np.ndarray:
    """Resize ROp, bilinear (§VI-F and §VI-J chains: Crop -> Resize -> ...).

    img is H x W x C (float64). Each output sample is
    (1-b)[(1-a) S(x0,y0) + a S(x1,y0)] + b[(1-a) S(x0,y1) + a S(x1,y1)].
    """
    src = np.asarray(img, dtype=np.float64)
    Hs, Ws = src.shape[:2]
    x0, x1, a = _bilinear_axis(Ws, out_w)
    y0, y1, b = _bilinear_axis(Hs, out_h)
    a = a[None, :, None]
    b = b[:, None, None]
    top = (1.0 - a) * src[y0][:, x0] + a * src[y0][:, x1]
    bot = (1.0 - a) * src[y1][:, x0] + a * src[y1][:, x1]
    return (1.0 - b) * top + b * bot


# BT.601 luma weights; the rest of the decode matrix is derived from them.
BT601_KR = 0.299
BT601_KB = 0.114


def bt601_limited_coefficients():
    """Decode coefficients (cY, cRV, cGU, cGV, cBU) of BT.601 limited range.

    R = cY*Y' + cRV*V';  G = cY*Y' - cGU*U' - cGV*V';  B = cY*Y' + cBU*U',
    with Y' = Y - 16, U' = U - 128, V' = V - 128 (8-bit studio swing:
    219 luma steps, 224 chroma steps).
    """
    kr, kb = BT601_KR, BT601_KB
    kg = 1.0 - kr - kb
    c_y = 255.0 / 219.0
    c_rv = 255.0 / 112.0 * (1.0 - kr)
    c_bu = 255.0 / 112.0 * (1.0 - kb)
    c_gu = c_bu * kb / kg
    c_gv = c_rv * kr / kg
    return c_y, c_rv, c_gu, c_gv, c_bu


def nv12_to_rgb(nv12: np.ndarray) -> np.ndarray:
    """NV12 read + BT.601 YUV -> RGB ColorConvert (NV12 frames: §VI-L).

    nv12 is uint8 [H*3/2, W]: luma rows then interleaved (U, V) rows.
    Returns float64 H x W x 3 in RGB order, each channel clamped to [0, 255].
    """
    H = nv12.shape[0] * 2 // 3
    W = nv12.shape[1]
    luma = nv12[:H].astype(np.float64)
    chroma = nv12[H:].astype(np.float64)            # [H/2, W] = (U,V) pairs
    xs = np.arange(W) // 2
    ys = np.arange(H) // 2
    u = chroma[ys][:, 2 * xs]                        # nearest chroma sample
    v = chroma[ys][:, 2 * xs + 1]
    c_y, c_rv, c_gu, c_gv, c_bu = bt601_limited_coefficients()
    yp, up, vp = luma - 16.0, u - 128.0, v - 128.0
    r = c_y * yp + c_rv * vp
    g = c_y * yp - c_gu * up - c_gv * vp
    b = c_y * yp + c_bu * up
    return np.clip(np.stack([r, g, b], axis=-1), 0.0, 255.0)


def letterbox_geometry(src_w: int, src_h: int, out_w: int, out_h: int):
    """(new_w, new_h, left, top) of an aspect-preserving fit into out_w x out_h."""
    r = min(out_w / src_w, out_h / src_h)
    new_w = min(out_w, int(np.floor(src_w * r + 0.5)))
    new_h = min(out_h, int(np.floor(src_h * r + 0.5)))
    return new_w, new_h, (out_w - new_w) // 2, (out_h - new_h) // 2


def letterbox(img: np.ndarray, out_w: int, out_h: int, pad: float) -> np.ndarray:
    """Letterbox ROp: bilinear resize to the fitted size, then pad around it."""
    Hs, Ws = img.shape[:2]
    new_w, new_h, left, top = letterbox_geometry(Ws, Hs, out_w, out_h)
    out = np.full((out_h, out_w, img.shape[2]), float(pad), dtype=np.float64)
    out[top:top + new_h, left:left + new_w] = resize_bilinear(img, new_w, new_h)
    return out


# ----------------------------------------------------------------------------
# Compute Operations (§IV-A, Table I "UnaryType" / "BinaryType")
# ----------------------------------------------------------------------------


def swap_rb(img: np.ndarray) -> np.ndarray:
    """ColorConvert BGR <-> RGB (§VI-F, §VI-J chains): reverse channel order."""
    return img[..., ::-1]


def multiply(img: np.ndarray, c) -> np.ndarray:
    """Multiply BOp (§VI-B, §VI-C): per-channel constant c (scalar or [C])."""
    return img * np.asarray(c, dtype=np.float64)


def add(img: np.ndarray, c) -> np.ndarray:
    """Add BOp (§VI-B): per-channel constant."""
    return img + np.asarray(c, dtype=np.float64)


def subtract(img: np.ndarray, c) -> np.ndarray:
    """Subtract BOp (§VI-C, §VI-J): per-channel constant, indexed by the
    channel of the value it receives (after any ColorConvert)."""
    return img - np.asarray(c, dtype=np.float64)


def divide(img: np.ndarray, c) -> np.ndarray:
    """Divide BOp (§VI-C, §VI-J): true division by a per-channel constant."""
    return img / np.asarray(c, dtype=np.float64)


def add_saturate_u8(img: np.ndarray, k) -> np.ndarray:
    """Saturating u8 add of an integer per-channel constant k (may be < 0):
    clamp(x + k, 0, 255) on the exact integer sum."""
    s = img.astype(np.int64) + np.asarray(k, dtype=np.int64)
    return np.clip(s, 0, 255).astype(np.uint8)


def saturate_cast_u8(x: np.ndarray) -> np.ndarray:
    """float -> u8: round half to even, then clamp to [0, 255]."""
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


# ----------------------------------------------------------------------------
# Write Operations (§IV-B, Table I "WriteType", Fig. 9 Split)
# ----------------------------------------------------------------------------


def split(img: np.ndarray) -> np.ndarray:
    """Split WOp (§IV-B, Fig. 9): packed H x W x C -> C planes [C, H, W]."""
    return np.moveaxis(img, -1, 0)


# ----------------------------------------------------------------------------
# Output number formats (round to nearest even from the float64 value)
# ----------------------------------------------------------------------------


def _round_to_grid(x: np.ndarray, mant_bits: int, min_exp: int) -> np.ndarray:
    """Round to the nearest value with `mant_bits` fraction bits, ties to even.

    Values below 2**min_exp use the fixed spacing 2**(min_exp - mant_bits)
    (gradual underflow). No overflow handling: callers clamp or check range.
    """
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                      # |x| = m * 2**e, 0.5 <= m < 1
    exp = np.maximum(e - 1, min_exp)        # floor(log2|x|), floored at min_exp
    ulp = np.ldexp(1.0, exp - mant_bits)
    return np.rint(x / ulp) * ulp           # x/ulp and the product are exact


def round_bf16(x: np.ndarray) -> np.ndarray:
    """IEEE-style bfloat16 (8 exponent bits, 7 fraction bits), RNE."""
    return _round_to_grid(x, 7, -126)


F16_OVERFLOW = 65520.0  # halfway between 65504 (the largest finite) and 2**16


def round_f16(x: np.ndarray) -> np.ndarray:
    """IEEE binary16 (5 exponent bits, 10 fraction bits), RNE, subnormals;
    |x| >= 65520 overflows to +-inf (the tie at 65520 goes to the even
    neighbour 2**16, which is out of range)."""
    x = np.asarray(x, dtype=np.float64)
    r = _round_to_grid(x, 10, -14)
    return np.where(np.abs(x) >= F16_OVERFLOW, np.copysign(np.inf, x), r)


E4M3_MAX = 448.0


def round_e4m3(q: np.ndarray) -> np.ndarray:
    """OCP FP8 E4M3 (bias 7, 3 fraction bits, no infinities), RNE,
    saturating to +-448 (the largest finite value). NaN stays NaN."""
    r = _round_to_grid(q, 3, -6)
    return np.clip(r, -E4M3_MAX, E4M3_MAX)


def quantize_e4m3(v: np.ndarray, scale: float) -> np.ndarray:
    """Per-tensor scaled FP8: q = sat_RNE(v / scale); dequantised value q*scale."""
    return round_e4m3(np.asarray(v, dtype=np.float64) / float(scale))


def format_ulp(x: np.ndarray, fmt: str) -> np.ndarray:
    """Spacing of format `fmt` at |x| (the ulp used in the 1-ulp tolerance)."""
    mant, min_exp = {"bf16": (7, -126), "f16": (10, -14), "e4m3": (3, -6)}[fmt]
    _, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(1.0, np.maximum(e - 1, min_exp) - mant)


def decode_e4m3(codes: np.ndarray) -> np.ndarray:
    """Value of each E4M3 byte (sign, 4-bit biased exponent, 3-bit fraction)."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    normal = np.ldexp(1.0 + m / 8.0, e - 7)
    sub = np.ldexp(m / 8.0, -6)
    val = np.where(e == 0, sub, normal)
    val = np.where((e == 0xF) & (m == 0x7), np.nan, val)
    return sign * val


def decode_bf16(bits: np.ndarray) -> np.ndarray:
    """Value of each bfloat16 bit pattern (upper half of a binary32)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------
# Vertical Mul/Add chain (§VI-B, §VI-D, §VI-G): float32, chain order
# ----------------------------------------------------------------------------

KIND_MUL = 0
KIND_ADD = 1


def vertical_chain_f32(x: np.ndarray, kinds, consts) -> np.ndarray:
    """Apply x <- x*c_i (Mul) or x <- x + c_i (Add) for i = 0..L-1 in float32.

    Each op is a separate numpy float32 operation, so every result is rounded
    to binary32 before the next op reads it (no multiply-add contraction).
    """
    y = np.array(x, dtype=np.float32, copy=True)
    for kind, c in zip(kinds, consts):
        c32 = np.float32(c)
        if kind == KIND_MUL:
            y = np.multiply(y, c32, dtype=np.float32)
        elif kind == KIND_ADD:
            y = np.add(y, c32, dtype=np.float32)
        else:
            raise ValueError(f"unknown op kind {kind}")
    return y


_TYPES = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32, "f64": np.float64}


def typed_chain(x: np.ndarray, out_dtype: str, mul=None, sub=None, div=None, scale=None) -> np.ndarray:
    """Read -> Cast -> Multiply -> Subtract -> Divide -> Write (§VI-I).

    The input is cast to the compute type -- float64 for an f64 output,
    float32 otherwise -- (numpy's cast: exact for u8, u16 and f32; round to
    nearest even for f64 into f32); then each present op is one numpy
    operation in that type, rounded to it before the next op reads it. The
    constants are float32 values (what a descriptor carries) taken exactly
    into the compute type. An absent op is skipped. The write rounds to the
    output type: f16 and bf16 round to nearest even (returned as float64
    values); e4m3 stores sat_RNE(v / s): the compute value v divided by the
    per-tensor scale s (the float32 value of `scale`) in float64, then
    rounded to nearest even with saturation at +-448. The quotient of a
    float32 v by a float32 s can round in float64 only far from an E4M3 tie
    (an E4M3 tie has at most 5 significant bits, and a float64 rounding error
    of v/s is 2^-53 relative), so this is the rounding of the exact quotient.
    """
    if out_dtype not in ("f32", "f64", "f16", "bf16", "e4m3"):
        raise ValueError("typed chains write f32, f64, f16, bf16 or e4m3")
    ct = np.float64 if out_dtype == "f64" else np.float32
    y = np.asarray(x).astype(ct)
    if mul is not None:
        y = np.multiply(y, ct(np.float32(mul)), dtype=ct)
    if sub is not None:
        y = np.subtract(y, ct(np.float32(sub)), dtype=ct)
    if div is not None:
        y = np.divide(y, ct(np.float32(div)), dtype=ct)
    if out_dtype == "bf16":
        return round_bf16(y)
    if out_dtype == "f16":
        return round_f16(y)
    if out_dtype == "e4m3":
        return round_e4m3(y.astype(np.float64) / float(np.float32(scale)))
    return y


# ----------------------------------------------------------------------------
# Whole chains: the unfused definition, one op after another
# ----------------------------------------------------------------------------


def preprocess_packed(src: np.ndarray, roi, out_w: int, out_h: int,
                      swap: bool = True, mul=1.0, sub=0.0, div=1.0) -> np.ndarray:
    """Crop -> Resize -> (BGR->RGB) -> Multiply -> Subtract -> Divide -> Split.

    The chain of §VI-F / §VI-J (there with a 64x128 output). src is uint8
    H x W x 3, roi = (x, y, w, h). Returns float64 [3, out_h, out_w].
    """
    x, y, w, h = (int(v) for v in roi)
    t = to_float(crop(src, x, y, w, h))
    t = resize_bilinear(t, out_w, out_h)
    if swap:
        t = swap_rb(t)
    t = multiply(t, mul)
    t = subtract(t, sub)
    t = divide(t, div)
    return split(t)


def preprocess_packed_batch(src_list, rois, out_w, out_h, **kw) -> np.ndarray:
    """Horizontal fusion (§IV-B BatchRead): the chain applied per image."""
    return np.stack([preprocess_packed(s, r, out_w, out_h, **kw)
                     for s, r in zip(src_list, rois)])


def preprocess_nv12(nv12: np.ndarray, out_w: int, out_h: int, pad: float = 114.0,
                    mul=1.0 / 255.0, sub=0.0, div=1.0,
                    letterboxed: bool = True) -> np.ndarray:
    """NV12 -> RGB -> (letterbox) resize -> Multiply [-> Subtract -> Divide]
    -> Split. Returns float64 [3, out_h, out_w]."""
    t = nv12_to_rgb(nv12)
    if letterboxed:
        t = letterbox(t, out_w, out_h, pad)
    else:
        t = resize_bilinear(t, out_w, out_h)
    t = multiply(t, mul)
    t = subtract(t, sub)
    t = divide(t, div)
    return split(t)


def integer_chain_packed(src: np.ndarray, roi, swap: bool, add_k) -> np.ndarray:
    """Crop -> (BGR->RGB) -> saturating add, all on u8, packed H x W x 3 out."""
    x, y, w, h = (int(v) for v in roi)
    t = crop(src, x, y, w, h)
    if swap:
        t = swap_rb(t)
    return add_saturate_u8(t, add_k)


# ----------------------------------------------------------------------------
# Reductions of a chain's values (the reduction pattern of §IV-C)
# ----------------------------------------------------------------------------


def reduce_stats(values: np.ndarray) -> dict:
    """Per-channel min, max and mean of planar values [N, C, H, W] (or
    [C, H, W]), the maximum absolute value over everything, and the E4M3
    per-tensor scale amax / 448 (1 when amax is 0)."""
    v = np.asarray(values, dtype=np.float64)
    if v.ndim == 3:
        v = v[None]
    per_c = np.moveaxis(v, 1, 0).reshape(v.shape[1], -1)
    amax = float(np.max(np.abs(v)))
    return {"min": per_c.min(axis=1), "max": per_c.max(axis=1), "mean": per_c.mean(axis=1),
            "amax": amax, "scale": amax / E4M3_MAX if amax > 0 else 1.0}
