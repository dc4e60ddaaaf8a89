"""Shapes and parameters of the preprocessing workloads.

Plain constants with no dependency on the CUDA library, so that CPU-only
code (the oracle timings) can size a workload without loading it; the chains
themselves are built in `workloads.py`.
"""
from __future__ import annotations

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
