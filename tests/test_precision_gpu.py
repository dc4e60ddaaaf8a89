"""Maximum and mean |error| of every output format against the float64
oracle, on sampled frames of the workloads the benchmark times: the NV12
letterbox batch (256 x 1280x720 -> 640x640) written as bf16, f16, FP8-E4M3
with the static scale 1/448 and FP8-E4M3 with the dynamic per-tensor scale
from ReduceDPP, and the float32 single-image and 50-crop chains.

Each case asserts the parity bound of its format (tests/parity.py) and
records the errors; with FKL_PRECISION_OUT set, the table is written there as
JSON (the command in the measurement notes that make the precision table).
Errors are in output units: for FP8 the dequantised value code * s against
the oracle value.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2508_07071_gb300 import synth
from parity import check_f32, check_lowp, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RESULTS = {}
SAMPLE = (0, 85, 170, 255)  # frames of the 256-frame batch compared element by element


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2508_07071_gb300 import build
    build.build()
    from paper_2508_07071_gb300 import fkl
    return fkl


@pytest.fixture(scope="module")
def W():
    from paper_2508_07071_gb300 import workloads
    return workloads


@pytest.fixture(scope="module")
def nv12(W):
    cfg = W.NV12
    frames = synth.nv12_frames(3, cfg["n"], cfg["h"], cfg["w"])
    want = {i: O.preprocess_nv12(frames[i], cfg["out"], cfg["out"], pad=cfg["pad"], mul=1 / 255) for i in SAMPLE}
    return frames, torch.from_numpy(frames).cuda(), want


@pytest.fixture(scope="module", autouse=True)
def write_table():
    yield
    path = os.environ.get("FKL_PRECISION_OUT")
    if path and RESULTS:
        with open(path, "w") as fh:
            json.dump(RESULTS, fh, indent=1, sort_keys=True)


def _record(key, errs):
    g = np.concatenate([e[0].ravel() for e in errs])
    o = np.concatenate([e[1].ravel() for e in errs])
    d = np.abs(g - o)
    RESULTS[key] = {"max_abs_err": float(d.max()), "mean_abs_err": float(d.mean()),
                    "max_rel_err_where_|o|>1e-3": float(np.max(d[np.abs(o) > 1e-3] / np.abs(o[np.abs(o) > 1e-3]))),
                    "values": int(g.size)}
    return RESULTS[key]


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
def test_nv12_batch_format_error(F, W, nv12, fmt):
    frames, dev, want = nv12
    cfg = W.NV12
    n = cfg["n"]
    code = {"bf16": F.FKL_BF16, "f16": F.FKL_F16, "e4m3": F.FKL_E4M3}[fmt]
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "e4m3": torch.float8_e4m3fn}[fmt]
    p = F.Pipeline(W.nv12_letterbox_chain(code))
    out = torch.zeros((n, 3, cfg["out"], cfg["out"]), dtype=tdt, device="cuda")
    F.fkl_execute_batch(p.handle, [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(n)], None,
                        F.as_fkl(out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    s = W.E4M3_SCALE if fmt == "e4m3" else 1.0
    errs = []
    for i in SAMPLE:
        got = to_numpy(out[i]).astype(np.float64)
        check_lowp(got, want[i], fmt, s, f"{fmt} frame {i}")
        errs.append((got * s, want[i]))
    r = _record(f"nv12_letterbox_{fmt}" + ("_static_scale" if fmt == "e4m3" else ""), errs)
    # the format's spacing at the top of the range (values in [0, 1]; FP8 codes
    # in [256, 448] are 32 apart), in output units
    ulp_top = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11, "e4m3": 32.0 * s}[fmt]
    assert r["max_abs_err"] <= ulp_top


def test_nv12_batch_dynamic_fp8_error(F, W, nv12):
    frames, dev, want = nv12
    cfg = W.NV12
    n = cfg["n"]
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, scale=1.0))
    out = torch.zeros((n, 3, cfg["out"], cfg["out"]), dtype=torch.float8_e4m3fn, device="cuda")
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(n)]
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, ins, None, o, stats.data_ptr())
    F.fkl_execute_batch_scaled(p.handle, ins, None, o, stats.data_ptr() + 11 * 4)
    torch.cuda.synchronize()
    s = float(stats[10].item())
    errs = []
    for i in SAMPLE:
        got = to_numpy(out[i]).astype(np.float64)
        check_lowp(got, want[i] / np.float32(s), "e4m3", 1.0, f"dynamic fp8 frame {i}")
        errs.append((got * s, want[i]))
    r = _record("nv12_letterbox_e4m3_dynamic_scale", errs)
    RESULTS["nv12_letterbox_e4m3_dynamic_scale"]["scale"] = s
    assert r["max_abs_err"] <= 32.0 * s  # one E4M3 step at the top of the range (codes 256..448), in output units


@pytest.mark.parametrize("which", ["single", "hf"])
def test_packed_f32_error(F, W, which):
    if which == "single":
        cfg = W.SINGLE
        src = synth.packed_image(0, cfg["src_h"], cfg["src_w"])
        rois = np.array([cfg["roi"]], np.int32)
    else:
        cfg = W.HF
        src = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
        rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
    n = len(rois)
    d = torch.from_numpy(src).cuda()
    p = F.Pipeline(W.normalize_chain(cfg["out_w"], cfg["out_h"]))
    out = torch.zeros((n, 3, cfg["out_h"], cfg["out_w"]), device="cuda")
    F.fkl_execute_batch(p.handle, [F.as_fkl(d)] * n, rois, F.as_fkl(out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    want = O.preprocess_packed_batch([src] * n, rois, cfg["out_w"], cfg["out_h"], swap=True, mul=1 / 255,
                                     sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    got = out.cpu().numpy().astype(np.float64)
    check_f32(got, want, which)
    r = _record(f"{'single_image_224' if which == 'single' else 'hf_50_crops'}_f32", [(got, want)])
    assert r["max_abs_err"] <= 1e-5 * np.abs(want).max() + 1e-6
