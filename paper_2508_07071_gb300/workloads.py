"""Chains of the preprocessing workloads (op descriptor lists).

Each function returns the descriptor list of one chain in the order the paper
writes it (ROp -> COps -> WOp). The constants (ImageNet mean/std, 1/255,
letterbox pad 114) are chain parameters, passed to the kernels unchanged;
they and the workload shapes are defined in `configs.py` and re-exported
here.
"""
from __future__ import annotations

from . import fkl as F
from .configs import (DTYPES, E4M3_SCALE, HF, IMAGENET_MEAN, IMAGENET_STD, INV255, NV12, SERVE, SINGLE,  # noqa: F401
                      VCHAIN)


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
