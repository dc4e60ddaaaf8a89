"""Chains and shapes of the preprocessing workloads (op descriptor lists).

Each function returns the descriptor list of one chain in the order the paper
writes it (ROp -> COps -> WOp). The constants (ImageNet mean/std, 1/255,
letterbox pad 114) are chain parameters, passed to the kernels unchanged.
"""
from __future__ import annotations

from . import fkl as F

IMAGENET_MEAN = (0.485, 0.456, 0.406)
IMAGENET_STD = (0.229, 0.224, 0.225)
INV255 = 1.0 / 255.0
E4M3_SCALE = 1.0 / 448.0  # inputs in [0, 1] map onto the whole E4M3 range

# Single image: 1920x1080 BGR, crop 640x480 at (320, 200), resize to 224x224.
SINGLE = dict(src_h=1080, src_w=1920, roi=(320, 200, 640, 480), out_w=224, out_h=224)
# Horizontal fusion: 50 crops of one 3840x2160 frame, each resized to 128x64.
HF = dict(src_h=2160, src_w=3840, n=50, w_range=(32, 640), h_range=(32, 480), out_w=128, out_h=64)
# Vertical Mul/Add chains over 64M float32 values.
VCHAIN = dict(n=64 * 1024 * 1024, lengths=(1, 10, 100, 1000))
# NV12 batch: 256 frames of 1280x720, letterboxed to 640x640 with pad 114.
NV12 = dict(n=256, h=720, w=1280, out=640, pad=114.0)
# Serving: full-frame resize to 224x224, FP16 planar.
SERVE = dict(out_w=224, out_h=224)
# Data types (paper §VI-I): 50 matrices of 60x120, Read -> Cast -> Multiply ->
# Subtract -> Divide -> Write, for every input type in {u8, u16, f32, f64}
# and output (compute) type in {f32, f64}: the 8 combinations.
DTYPES = dict(n=50, rows=60, cols=120, ins=("u8", "u16", "f32", "f64"), outs=("f32", "f64"),
              mul=INV255, sub=0.485, div=0.229)


def normalize_chain(out_w, out_h, out_dtype=F.FKL_F32, roi=None, scale=None, swap=True):
    """Crop -> Resize -> BGR->RGB -> x1/255 -> -mean -> /std -> Split."""
    ops = [F.read_u8c3()]
    if roi is not None:
        ops.append(F.crop(*roi))
    ops.append(F.resize(out_w, out_h))
    if swap:
        ops.append(F.swap_rb())
    ops += [F.mul(INV255), F.sub(IMAGENET_MEAN), F.div(IMAGENET_STD),
            F.write_split(out_dtype, scale)]
    return ops


def nv12_letterbox_chain(out_dtype, out=640, pad=114.0, scale=None):
    """NV12 -> BT.601 RGB -> letterbox (pad) -> x1/255 -> Split."""
    if out_dtype == F.FKL_E4M3 and scale is None:
        scale = E4M3_SCALE
    return [F.read_nv12(), F.letterbox(out, out, pad), F.mul(INV255),
            F.write_split(out_dtype, scale)]


def vertical_chain(kinds, consts, u8_input=False):
    """READ_F32 (or READ_U8) -> (MUL|ADD)* -> WRITE_PACKED(F32)."""
    ops = [F.read_u8() if u8_input else F.read_f32()]
    for k, c in zip(kinds, consts):
        ops.append(F.scalar_op(F.FKL_OP_ADD if k == 1 else F.FKL_OP_MUL, float(c)))
    ops.append(F.write_packed(F.FKL_F32))
    return ops


def integer_chain(roi=None, swap=True, add_k=(0, 0, 0), split=False):
    ops = [F.read_u8c3()]
    if roi is not None:
        ops.append(F.crop(*roi))
    if swap:
        ops.append(F.swap_rb())
    ops.append(F.add_sat_u8(add_k))
    ops.append(F.write_split(F.FKL_U8) if split else F.write_packed(F.FKL_U8))
    return ops


def typed_chain(in_dtype, out_dtype, mul=None, sub=None, div=None, scale=None):
    """READ_<in> [MUL] [SUB] [DIV] WRITE_PACKED(<out>) (paper §VI-I); `scale`
    is the per-tensor scale of an E4M3 output."""
    ops = [F.read_linear(in_dtype)]
    if mul is not None:
        ops.append(F.mul(mul))
    if sub is not None:
        ops.append(F.sub(sub))
    if div is not None:
        ops.append(F.div(div))
    ops.append(F.write_packed(out_dtype, scale))
    return ops
