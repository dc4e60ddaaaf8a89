"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small cases are compared element by element; the full-size workloads run in
the launch configuration the benchmark times and are compared on sampled
images (or sampled elements for the elementwise vertical chain).
"""
import numpy as np
import pytest

import oracle as O
from paper_2508_07071_gb300 import synth
from parity import check_f32, check_output, check_lowp, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def code(F, fmt):
    return {"f32": F.FKL_F32, "f16": F.FKL_F16, "bf16": F.FKL_BF16, "e4m3": F.FKL_E4M3, "u8": F.FKL_U8}[fmt]


def tdtype(fmt):
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16,
            "e4m3": torch.float8_e4m3fn, "u8": torch.uint8}[fmt]


def run_batch(F, ops, srcs, rois, out_shape, fmt, layout_in=None, unfused=False, shape=None):
    p = F.Pipeline(ops)
    if shape is not None:
        F.fkl_pipeline_set_shape(p.handle, shape)
    out = torch.full(out_shape, float("nan") if fmt != "u8" and fmt != "e4m3" else 0,
                     dtype=tdtype(fmt), device="cuda")
    layout = F.FKL_LAYOUT_NCHW if out_shape[1] == 3 else F.FKL_LAYOUT_NHWC
    ins = [F.as_fkl(s, layout_in) for s in srcs]
    o = F.as_fkl(out, layout)
    if unfused:
        nbytes = F.fkl_unfused_workspace_bytes(p.handle, ins, rois, o)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        F.fkl_execute_batch_unfused(p.handle, ins, rois, o, ws.data_ptr(), nbytes)
    else:
        F.fkl_execute_batch(p.handle, ins, rois, o)
    torch.cuda.synchronize()
    return out


# ------------------------------------------------------------------ single image (crop -> resize -> normalise)


def test_single_image_full_size(F, W):
    cfg = W.SINGLE
    src = synth.packed_image(0, cfg["src_h"], cfg["src_w"])
    ops = W.normalize_chain(cfg["out_w"], cfg["out_h"], roi=cfg["roi"])
    out = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 3, cfg["out_h"], cfg["out_w"]), "f32")
    want = O.preprocess_packed(src, cfg["roi"], cfg["out_w"], cfg["out_h"], swap=True, mul=1 / 255,
                               sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(out)[0], want, "single image")


def test_hf_batch_full_size(F, W):
    cfg = W.HF
    frame = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
    rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
    dframe = torch.from_numpy(frame).cuda()
    ops = W.normalize_chain(cfg["out_w"], cfg["out_h"])
    out = run_batch(F, ops, [dframe] * cfg["n"], rois, (cfg["n"], 3, cfg["out_h"], cfg["out_w"]), "f32")
    want = O.preprocess_packed_batch([frame] * cfg["n"], rois, cfg["out_w"], cfg["out_h"], swap=True,
                                     mul=1 / 255, sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(out), want, "HF batch")


@pytest.mark.parametrize("fmt", ["f32", "f16", "bf16", "e4m3"])
@pytest.mark.parametrize("swap", [True, False])
def test_packed_formats(F, W, fmt, swap):
    src = synth.packed_image(2, 90, 131)
    rois = np.array([[0, 0, 131, 90], [5, 7, 60, 41], [100, 50, 31, 40]], np.int32)
    scale = W.E4M3_SCALE if fmt == "e4m3" else None
    mean, std = W.IMAGENET_MEAN, W.IMAGENET_STD
    ops = [F.read_u8c3(), F.resize(37, 23)] + ([F.swap_rb()] if swap else []) + [
        F.mul(W.INV255), F.sub(mean), F.div(std), F.write_split(code(F, fmt), scale)]
    d = torch.from_numpy(src).cuda()
    out = run_batch(F, ops, [d] * 3, rois, (3, 3, 23, 37), fmt)
    want = O.preprocess_packed_batch([src] * 3, rois, 37, 23, swap=swap, mul=1 / 255, sub=mean, div=std)
    if fmt == "e4m3":
        # normalised values exceed [0, 1]; |v| / scale stays finite and saturates at 448
        check_output(out, want, fmt, scale, "packed e4m3")
    else:
        check_output(out, want, fmt, 1.0, f"packed {fmt}")


@pytest.mark.parametrize("src_hw,roi,out_wh", [
    ((7, 5), (0, 0, 5, 7), (19, 13)),          # upscale with border clamp
    ((1, 1), (0, 0, 1, 1), (9, 4)),            # 1x1 source
    ((50, 60), (59, 49, 1, 1), (3, 3)),        # corner pixel
    ((33, 47), (3, 2, 40, 30), (40, 30)),      # identity resize = exact copy
    ((480, 640), (1, 1, 637, 477), (224, 224)),
    ((64, 33), (0, 0, 33, 64), (128, 64)),     # ragged width
])
def test_packed_geometry_edges(F, W, src_hw, roi, out_wh):
    src = synth.packed_image(3, *src_hw)
    ops = [F.read_u8c3(), F.crop(*roi), F.resize(*out_wh), F.write_split(F.FKL_F32)]
    out = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 3, out_wh[1], out_wh[0]), "f32")
    want = O.preprocess_packed(src, roi, out_wh[0], out_wh[1], swap=False)
    check_f32(to_numpy(out)[0], want, f"geometry {src_hw} {roi} {out_wh}")
    if roi[2:] == out_wh:  # identity resize reproduces the crop exactly
        assert np.array_equal(to_numpy(out)[0], O.split(O.crop(src, *roi).astype(np.float64)))


def test_crop_only_float_chain(F):
    src = synth.packed_image(4, 20, 30)
    ops = [F.read_u8c3(), F.crop(2, 3, 17, 11), F.mul(0.5), F.write_split(F.FKL_F32)]
    out = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 3, 11, 17), "f32")
    want = O.split(O.multiply(O.to_float(O.crop(src, 2, 3, 17, 11)), 0.5))
    assert np.array_equal(to_numpy(out)[0], want)


def test_packed_output_layout(F, W):
    src = synth.packed_image(5, 40, 60)
    ops = [F.read_u8c3(), F.resize(21, 13), F.swap_rb(), F.mul(W.INV255), F.write_packed(F.FKL_F32)]
    out = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 13, 21, 3), "f32")
    want = O.preprocess_packed(src, (0, 0, 60, 40), 21, 13, swap=True, mul=1 / 255)
    check_f32(to_numpy(out)[0], np.moveaxis(want, 0, -1), "packed output")


def test_large_batch_multi_launch(F, W):
    src = synth.packed_image(6, 64, 64)
    rois = synth.crop_rois(6, 300, 64, 64, (4, 40), (4, 40))
    ops = W.normalize_chain(16, 8)
    d = torch.from_numpy(src).cuda()
    out = run_batch(F, ops, [d] * 300, rois, (300, 3, 8, 16), "f32")
    want = O.preprocess_packed_batch([src] * 300, rois, 16, 8, swap=True, mul=1 / 255,
                                     sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(out), want, "300 images")


def test_empty_batch_is_a_no_op(F, W):
    p = F.Pipeline(W.normalize_chain(16, 8))
    out = torch.zeros((1, 3, 8, 16), device="cuda")
    F.fkl_execute_batch(p.handle, [], None, F.as_fkl(out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0


def test_unaligned_pitches_take_scalar_paths(F, W):
    src = synth.packed_image(7, 40, 50)
    big = torch.zeros((40, 51, 3), dtype=torch.uint8)
    big[:, :50] = torch.from_numpy(src)
    d = big.cuda()[:, :50]                      # row pitch 153 bytes
    outbuf = torch.full((1, 3, 20, 27), float("nan"), device="cuda")
    out = outbuf[..., :25]                      # output pitch 108 bytes
    p = F.Pipeline(W.normalize_chain(25, 20))
    F.fkl_execute(p.handle, F.as_fkl(d), F.as_fkl(out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    want = O.preprocess_packed(src, (0, 0, 50, 40), 25, 20, swap=True, mul=1 / 255,
                               sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(out)[0], want, "unaligned")
    assert torch.isnan(outbuf[..., 25:]).all()  # nothing written past the row


# ------------------------------------------------------------------ NV12 -> letterbox


def nv12_case(F, W, fmt, frames, out=640, shape=None, unfused=False, rois=None):
    dev = torch.from_numpy(frames).cuda()
    ops = W.nv12_letterbox_chain(code(F, fmt), out=out)
    scale = W.E4M3_SCALE if fmt == "e4m3" else 1.0
    res = run_batch(F, ops, [dev[i] for i in range(len(frames))], rois, (len(frames), 3, out, out), fmt,
                    layout_in=F.FKL_LAYOUT_NV12, unfused=unfused, shape=shape)
    return res, scale


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3", "f32"])
def test_nv12_letterbox_small_batch(F, W, fmt):
    frames = synth.nv12_frames(3, 3, 720, 1280)
    out, scale = nv12_case(F, W, fmt, frames)
    for i in range(len(frames)):
        want = O.preprocess_nv12(frames[i], 640, 640, pad=114.0, mul=1 / 255)
        stats = check_output(out[i], want, fmt, scale, f"nv12 {fmt} frame {i}")
        if fmt != "f32":
            # one ulp of the format at the top of the [0, 1] range
            assert stats["max_abs_err_vs_fp64"] <= {"bf16": 2 ** -8, "f16": 2 ** -11, "e4m3": 32 * scale}[fmt]


def test_nv12_full_batch_sampled(F, W):
    cfg = W.NV12
    frames = synth.nv12_frames(3, cfg["n"], cfg["h"], cfg["w"])
    out, _ = nv12_case(F, W, "bf16", frames)
    for i in [0, 1, 77, 128, 200, cfg["n"] - 1]:
        want = O.preprocess_nv12(frames[i], 640, 640, pad=114.0, mul=1 / 255)
        check_output(out[i], want, "bf16", 1.0, f"full batch frame {i}")


@pytest.mark.parametrize("hw,out,roi", [
    ((720, 1280), 512, None),                  # 2.5x: general bilinear path
    ((480, 640), 640, None),                   # upscale
    ((96, 130), 64, [(3, 5, 101, 77)]),        # odd crop offsets and sizes
    ((64, 48), 32, [(16, 8, 32, 40)]),         # 2x with 16-aligned crop: vector path
    ((2, 2), 1, None),                         # smallest frame, 1x1 output (exact 2x)
    ((2, 6), 3, None),                         # 3x1 window, fill rows above and below
])
def test_nv12_general_geometry(F, W, hw, out, roi):
    frames = synth.nv12_frames(4, 1, *hw)
    dev = torch.from_numpy(frames).cuda()
    ops = [F.read_nv12(), F.letterbox(out, out, 114.0), F.mul(W.INV255), F.write_split(F.FKL_F32)]
    res = run_batch(F, ops, [dev[0]], roi, (1, 3, out, out), "f32", layout_in=F.FKL_LAYOUT_NV12)
    rgb = O.nv12_to_rgb(frames[0])
    if roi is not None:
        x, y, w, h = roi[0]
        rgb = rgb[y:y + h, x:x + w]
    want = O.split(O.multiply(O.letterbox(rgb, out, out, 114.0), 1 / 255))
    check_f32(to_numpy(res)[0], want, f"nv12 geometry {hw} {out} {roi}")


def test_nv12_resize_with_normalise(F, W):
    frames = synth.nv12_frames(5, 2, 360, 640)
    dev = torch.from_numpy(frames).cuda()
    ops = [F.read_nv12(), F.resize(320, 180), F.swap_rb(), F.mul(W.INV255), F.sub(W.IMAGENET_MEAN),
           F.div(W.IMAGENET_STD), F.write_split(F.FKL_F16)]
    res = run_batch(F, ops, [dev[0], dev[1]], None, (2, 3, 180, 320), "f16", layout_in=F.FKL_LAYOUT_NV12)
    for i in range(2):
        rgb = O.nv12_to_rgb(frames[i])
        t = O.swap_rb(O.resize_bilinear(rgb, 320, 180))
        want = O.split(O.divide(O.subtract(O.multiply(t, 1 / 255), W.IMAGENET_MEAN), W.IMAGENET_STD))
        check_output(res[i], want, "f16", 1.0, "nv12 normalise")


# ------------------------------------------------------------------ vertical chain


@pytest.mark.parametrize("L", [0, 1, 2, 7, 10, 13, 100, 1000, 4099])
def test_vertical_chain_bit_exact(F, W, L):
    """Alternating Mul/Add chains against the same-order float32 oracle, bit
    for bit. The kernel reads the constants of two pairs at a time, then of
    one pair, then a lone Mul: lengths 7 and 13 take all three steps in one
    launch, 4099 two launches."""
    n = 100_003
    x = synth.f32_uniform(2, n)
    kinds, consts = synth.chain_constants(2, L)
    p = F.Pipeline(W.vertical_chain(kinds, consts))
    xin = torch.from_numpy(x).cuda()
    out = torch.empty_like(xin)
    F.fkl_execute(p.handle, F.as_fkl(xin), F.as_fkl(out))
    torch.cuda.synchronize()
    want = O.vertical_chain_f32(x, kinds, consts)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_vertical_chain_irregular_kinds_in_place(F, W):
    rng = np.random.default_rng(9)
    kinds = rng.integers(0, 2, 333)
    consts = rng.uniform(0.5, 1.5, 333).astype(np.float32)
    x = synth.f32_uniform(3, 4097)
    buf = torch.from_numpy(x).cuda()
    p = F.Pipeline(W.vertical_chain(kinds, consts))
    F.fkl_execute(p.handle, F.as_fkl(buf), F.as_fkl(buf))
    torch.cuda.synchronize()
    want = O.vertical_chain_f32(x, kinds, consts)
    assert np.array_equal(buf.cpu().numpy().view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("L", [1, 10, 1000])
def test_vertical_chain_full_size_sampled(F, W, L):
    n = W.VCHAIN["n"]
    x = synth.f32_uniform(2, n)
    kinds, consts = synth.chain_constants(2, L)
    p = F.Pipeline(W.vertical_chain(kinds, consts))
    xin = torch.from_numpy(x).cuda()
    out = torch.empty_like(xin)
    F.fkl_execute(p.handle, F.as_fkl(xin), F.as_fkl(out))
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([np.random.default_rng(L).integers(0, n, 20000), [0, n - 1]]))
    want = O.vertical_chain_f32(x[idx], kinds, consts)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ------------------------------------------------------------------ integer chains


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("swap", [False, True])
def test_integer_chain_bit_exact(F, W, split, swap):
    src = synth.packed_image(8, 37, 45)
    roi = (3, 4, 33, 29)
    k = (40, -70, 200)
    ops = W.integer_chain(roi=roi, swap=swap, add_k=k, split=split)
    shape = (1, 3, 29, 33) if split else (1, 29, 33, 3)
    out = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, shape, "u8")
    want = O.integer_chain_packed(src, roi, swap=swap, add_k=k)
    got = out.cpu().numpy()[0]
    assert np.array_equal(np.moveaxis(got, 0, -1) if split else got, want)


# ------------------------------------------------------------------ unfused form, launch shapes, graphs


def test_unfused_equals_fused_bitwise(F, W):
    cfg = W.HF
    frame = synth.packed_image(1, 720, 1280)
    rois = synth.crop_rois(1, 7, 1280, 720, cfg["w_range"], cfg["h_range"])
    d = torch.from_numpy(frame).cuda()
    ops = W.normalize_chain(128, 64)
    a = run_batch(F, ops, [d] * 7, rois, (7, 3, 64, 128), "f32")
    b = run_batch(F, ops, [d] * 7, rois, (7, 3, 64, 128), "f32", unfused=True)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))

    frames = synth.nv12_frames(3, 2, 720, 1280)
    for fmt in ["f32", "f16", "bf16", "e4m3"]:
        a, _ = nv12_case(F, W, fmt, frames)
        b, _ = nv12_case(F, W, fmt, frames, unfused=True)
        assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), fmt

    src = synth.packed_image(8, 37, 45)
    ops = W.integer_chain(roi=(3, 4, 33, 29), swap=True, add_k=(1, -2, 3), split=True)
    a = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 3, 29, 33), "u8")
    b = run_batch(F, ops, [torch.from_numpy(src).cuda()], None, (1, 3, 29, 33), "u8", unfused=True)
    assert torch.equal(a, b)

    kinds, consts = synth.chain_constants(2, 37)
    x = torch.from_numpy(synth.f32_uniform(2, 5000)).cuda()
    p = F.Pipeline(W.vertical_chain(kinds, consts))
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    F.fkl_execute(p.handle, F.as_fkl(x), F.as_fkl(y1))
    F.fkl_execute_batch_unfused(p.handle, [F.as_fkl(x)], None, F.as_fkl(y2), 0, 0)
    torch.cuda.synchronize()
    assert torch.equal(y1.view(torch.int32), y2.view(torch.int32))


@pytest.mark.parametrize("src", ["packed", "nv12"])
def test_mul_sub_pair_chain_equals_unfused_bitwise(F, W, src):
    """A chain without Div runs its compute ops on packed pixel pairs; each op
    still rounds on its own, as in the one-kernel-per-op form."""
    if src == "packed":
        img = torch.from_numpy(synth.packed_image(21, 90, 131)).cuda()
        ops = [F.read_u8c3(), F.resize(64, 45), F.swap_rb(), F.mul(W.INV255), F.sub(W.IMAGENET_MEAN),
               F.write_split(F.FKL_F32)]
        srcs, layout = [img, img], None
        rois = np.array([[0, 0, 131, 90], [3, 5, 101, 77]], np.int32)
    else:
        fr = torch.from_numpy(synth.nv12_frames(21, 2, 90, 128)).cuda()
        ops = [F.read_nv12(), F.resize(64, 45), F.mul(W.INV255), F.sub(W.IMAGENET_MEAN), F.write_split(F.FKL_F32)]
        srcs, layout, rois = [fr[0], fr[1]], F.FKL_LAYOUT_NV12, None
    a = run_batch(F, ops, srcs, rois, (2, 3, 45, 64), "f32", layout_in=layout)
    b = run_batch(F, ops, srcs, rois, (2, 3, 45, 64), "f32", layout_in=layout, unfused=True)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_every_launch_shape_gives_the_same_bytes(F, W):
    frames = synth.nv12_frames(3, 2, 720, 1280)
    base, _ = nv12_case(F, W, "bf16", frames)
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    for shape in F.fkl_pipeline_shapes(p.handle):
        got, _ = nv12_case(F, W, "bf16", frames, shape=shape)
        assert torch.equal(got.view(torch.uint8), base.view(torch.uint8)), shape

    src = synth.packed_image(2, 90, 131)
    rois = np.array([[0, 0, 131, 90], [5, 7, 60, 41]], np.int32)
    ops = W.normalize_chain(37, 23)
    d = torch.from_numpy(src).cuda()
    base = run_batch(F, ops, [d, d], rois, (2, 3, 23, 37), "f32")
    p = F.Pipeline(ops)
    for shape in F.fkl_pipeline_shapes(p.handle):
        got = run_batch(F, ops, [d, d], rois, (2, 3, 23, 37), "f32", shape=shape)
        assert torch.equal(got.view(torch.int32), base.view(torch.int32)), shape


def test_cuda_graph_capture_replays(F, W):
    frames = synth.nv12_frames(3, 4, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    out = torch.zeros((4, 3, 640, 640), dtype=torch.bfloat16, device="cuda")
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(4)]
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        F.fkl_execute_batch(p.handle, ins, None, o, stream=s)  # warm up outside the capture
    torch.cuda.synchronize()
    ref = out.clone()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        F.fkl_execute_batch(p.handle, ins, None, o, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.uint8), ref.view(torch.uint8))


def test_vertical_chain_every_shape_bit_exact(F, W):
    x = synth.f32_uniform(2, 300_001)
    kinds, consts = synth.chain_constants(2, 21)
    want = O.vertical_chain_f32(x, kinds, consts).view(np.uint32)
    p = F.Pipeline(W.vertical_chain(kinds, consts))
    xin = torch.from_numpy(x).cuda()
    for shape in F.fkl_pipeline_shapes(p.handle):
        F.fkl_pipeline_set_shape(p.handle, shape)
        out = torch.full_like(xin, float("nan"))
        F.fkl_execute(p.handle, F.as_fkl(xin), F.as_fkl(out))
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want), shape


def test_autotune_keeps_results(F, W):
    frames = synth.nv12_frames(3, 8, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    out = torch.zeros((8, 3, 640, 640), dtype=torch.bfloat16, device="cuda")
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(8)]
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    best, us = F.fkl_pipeline_autotune(p.handle, ins, None, o, reps=2)
    assert best in F.fkl_pipeline_shapes(p.handle) and us > 0
    assert F.fkl_pipeline_get_shape(p.handle) == best
    ref, _ = nv12_case(F, W, "bf16", frames)
    out.zero_()
    F.fkl_execute_batch(p.handle, ins, None, o)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.uint8), ref.view(torch.uint8))

    kinds, consts = synth.chain_constants(2, 10)
    pv = F.Pipeline(W.vertical_chain(kinds, consts))
    x = torch.from_numpy(synth.f32_uniform(2, 1 << 20)).cuda()
    y = torch.empty_like(x)
    best, us = F.fkl_pipeline_autotune(pv.handle, [F.as_fkl(x)], None, F.as_fkl(y), reps=2)
    assert best in F.fkl_pipeline_shapes(pv.handle)


def test_host_executor_matches_device_path(F, W):
    n = 37                                            # 5 chunks of 8, ragged last chunk
    frames = synth.nv12_frames(13, n, 720, 1280)
    host_in = torch.from_numpy(frames).pin_memory()
    host_out = torch.zeros((n, 3, 640, 640), dtype=torch.bfloat16).pin_memory()
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    e = F.fkl_host_executor_create(p.handle, 8, 3, 1080 * 1280, 3 * 640 * 640 * 2)
    try:
        ins = [F.as_fkl(host_in[i], F.FKL_LAYOUT_NV12) for i in range(n)]
        for _ in range(2):                            # slots are reused across calls
            host_out.zero_()
            F.fkl_execute_batch_host(e, ins, None, F.as_fkl(host_out, F.FKL_LAYOUT_NCHW))
            torch.cuda.synchronize()
            ref, _ = nv12_case(F, W, "bf16", frames)
            assert torch.equal(host_out.view(torch.uint8), ref.cpu().view(torch.uint8))
        # pitched host images (copied with 2-D copies) and an image too big for a slot
        big = torch.zeros((n, 1080, 1296), dtype=torch.uint8).pin_memory()
        big[:, :, :1280] = host_in
        ins2 = [F.as_fkl(big[i, :, :1280], F.FKL_LAYOUT_NV12) for i in range(4)]
        out2 = torch.zeros((4, 3, 640, 640), dtype=torch.bfloat16).pin_memory()
        F.fkl_execute_batch_host(e, ins2, None, F.as_fkl(out2, F.FKL_LAYOUT_NCHW))
        torch.cuda.synchronize()
        assert torch.equal(out2.view(torch.uint8), host_out[:4].view(torch.uint8))
        huge = torch.zeros((2160 * 3 // 2, 3840), dtype=torch.uint8)
        with pytest.raises(F.FklError):
            F.fkl_execute_batch_host(e, [F.as_fkl(huge, F.FKL_LAYOUT_NV12)], None,
                                     F.as_fkl(out2, F.FKL_LAYOUT_NCHW))
    finally:
        F.fkl_host_executor_destroy(e)


@pytest.mark.parametrize("L", [0, 3, 200, 4101])
def test_vertical_chain_u8_input_bit_exact(F, W, L):
    n = 50 * 60 * 120 + 5                               # ragged tail
    x = synth.packed_image(15, 1, n, 1).reshape(-1)
    kinds, consts = synth.chain_constants(5, L)
    p = F.Pipeline(W.vertical_chain(kinds, consts, u8_input=True))
    assert "ReadU8" in p.kernel_name
    xin = torch.from_numpy(x).cuda()
    want = O.vertical_chain_f32(x.astype(np.float32), kinds, consts).view(np.uint32)
    for shape in F.fkl_pipeline_shapes(p.handle)[:: 3 if L > 1000 else 1]:
        F.fkl_pipeline_set_shape(p.handle, shape)
        out = torch.full((n,), float("nan"), device="cuda")
        F.fkl_execute(p.handle, F.as_fkl(xin), F.as_fkl(out))
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want), shape
    if L <= 200:
        out2 = torch.full((n,), float("nan"), device="cuda")
        F.fkl_execute_batch_unfused(p.handle, [F.as_fkl(xin)], None, F.as_fkl(out2), 0, 0)
        torch.cuda.synchronize()
        assert np.array_equal(out2.cpu().numpy().view(np.uint32), want)
    with pytest.raises(F.FklError):                     # a u8 chain refuses float input
        F.fkl_execute(p.handle, F.as_fkl(torch.zeros(n, device="cuda")), F.as_fkl(out))


def test_reduce_stats_and_dynamic_fp8(F, W):
    frames = synth.nv12_frames(17, 3, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(3)]
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, scale=1.0))
    out = torch.zeros((3, 3, 640, 640), dtype=torch.float8_e4m3fn, device="cuda")
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, ins, None, o, stats.data_ptr())
    F.fkl_execute_batch_scaled(p.handle, ins, None, o, stats.data_ptr() + 11 * 4)
    torch.cuda.synchronize()
    st = stats.cpu().numpy().astype(np.float64)
    vals = np.stack([O.preprocess_nv12(f, 640, 640, pad=114.0, mul=1 / 255) for f in frames])
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-6)
    check_f32(st[9], want["amax"], "amax")
    check_f32(st[10], want["scale"], "scale")
    # the stored codes are the oracle values quantised with the kernel's scale
    check_lowp(to_numpy(out), vals / np.float32(st[10]), "e4m3", 1.0, "dynamic fp8")
    assert out.view(torch.uint8).max().item() == 0x7E  # amax maps onto 448


def test_reduce_stats_normalised_packed(F, W):
    src = synth.packed_image(18, 300, 500)
    rois = np.array([[0, 0, 500, 300], [10, 20, 200, 150]], np.int32)
    d = torch.from_numpy(src).cuda()
    p = F.Pipeline(W.normalize_chain(224, 224))
    out = torch.zeros((2, 3, 224, 224), device="cuda")
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, [F.as_fkl(d)] * 2, rois, F.as_fkl(out, F.FKL_LAYOUT_NCHW), stats.data_ptr())
    torch.cuda.synchronize()
    st = stats.cpu().numpy().astype(np.float64)
    vals = O.preprocess_packed_batch([src] * 2, rois, 224, 224, swap=True, mul=1 / 255,
                                     sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-5, atol=1e-6)
    check_f32(st[9], want["amax"], "amax")
    assert float(out.abs().sum()) == 0.0               # the reduction writes no output


def _reduce_split(stats):
    """(float statistics, jobs, blocks) of a stats buffer."""
    st = stats.cpu()
    return st[:12].numpy().astype(np.float64), int(st.view(torch.int32)[12]), int(st.view(torch.int32)[13])


def test_reduce_many_jobs_per_block_against_the_oracle_and_the_write(F, W):
    """The reduction's persistent grid with several jobs per block (the job
    count is checked against the grid): statistics against the oracle's, the
    extremes equal bit for bit to those of the fused chain's float32 output,
    and the dynamic FP8 codes of sampled frames within 1 ulp."""
    n = 48
    frames = synth.nv12_frames(19, n, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(n)]
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, scale=1.0))
    out = torch.zeros((n, 3, 640, 640), dtype=torch.float8_e4m3fn, device="cuda")
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, ins, None, o, stats.data_ptr())
    F.fkl_execute_batch_scaled(p.handle, ins, None, o, stats.data_ptr() + 11 * 4)
    f32 = run_batch(F, W.nv12_letterbox_chain(F.FKL_F32), [dev[i] for i in range(n)], None, (n, 3, 640, 640),
                    "f32", layout_in=F.FKL_LAYOUT_NV12)
    torch.cuda.synchronize()
    st, jobs, grid = _reduce_split(stats)
    assert jobs > 2 * grid > 0, (jobs, grid)
    per_c = f32.permute(1, 0, 2, 3).reshape(3, -1)
    assert np.array_equal(st[0:3].astype(np.float32), per_c.min(dim=1).values.cpu().numpy())
    assert np.array_equal(st[3:6].astype(np.float32), per_c.max(dim=1).values.cpu().numpy())
    vals = np.stack([O.preprocess_nv12(f, 640, 640, pad=114.0, mul=1 / 255) for f in frames])
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-6)
    check_f32(st[9], want["amax"], "amax")
    check_f32(st[10], want["scale"], "scale")
    for i in (0, n // 2, n - 1):
        check_lowp(to_numpy(out[i]), vals[i] / np.float32(st[10]), "e4m3", 1.0, f"dynamic fp8 frame {i}")
    assert out.view(torch.uint8).max().item() == 0x7E


@pytest.mark.parametrize("swap", [True, False])
def test_reduce_decreasing_chain(F, W, swap):
    """Negative Mul and Div make the chain decreasing on every channel: the
    minimum comes from the largest read value. Extremes equal the float32
    write's; mean and amax match the oracle."""
    src = synth.packed_image(29, 300, 500)
    rois = np.array([[0, 0, 500, 300], [17, 9, 333, 201], [100, 50, 64, 32]], np.int32)
    mul, sub, div = (-1 / 255, 2 / 255, -0.5), (0.25, -0.5, 1.0), (-0.229, 0.5, -2.0)
    ops = [F.read_u8c3(), F.resize(97, 61)] + ([F.swap_rb()] if swap else []) + \
        [F.mul(mul), F.sub(sub), F.div(div), F.write_split(F.FKL_F32)]
    d = torch.from_numpy(src).cuda()
    got = run_batch(F, ops, [d] * 3, rois, (3, 3, 61, 97), "f32")
    p = F.Pipeline(ops)
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, [F.as_fkl(d)] * 3, rois, F.as_fkl(got, F.FKL_LAYOUT_NCHW), stats.data_ptr())
    torch.cuda.synchronize()
    st, _, _ = _reduce_split(stats)
    per_c = got.permute(1, 0, 2, 3).reshape(3, -1)
    assert np.array_equal(st[0:3].astype(np.float32), per_c.min(dim=1).values.cpu().numpy())
    assert np.array_equal(st[3:6].astype(np.float32), per_c.max(dim=1).values.cpu().numpy())
    vals = O.preprocess_packed_batch([src] * 3, rois, 97, 61, swap=swap, mul=mul, sub=sub, div=div)
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-5, atol=1e-6)
    check_f32(st[9], want["amax"], "amax")


@pytest.mark.parametrize("fmt", ["e4m3", "f16"])
def test_nv12_full_batch_autotuned_sampled(F, W, fmt):
    """The bench's configuration: 256 frames, autotuned launch shape."""
    cfg = W.NV12
    frames = synth.nv12_frames(3, cfg["n"], cfg["h"], cfg["w"])
    dev = torch.from_numpy(frames).cuda()
    p = F.Pipeline(W.nv12_letterbox_chain(code(F, fmt)))
    out = torch.zeros((cfg["n"], 3, 640, 640), dtype=tdtype(fmt), device="cuda")
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(cfg["n"])]
    o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
    best, _ = F.fkl_pipeline_autotune(p.handle, ins, None, o, reps=3)
    out.zero_()
    F.fkl_execute_batch(p.handle, ins, None, o)
    torch.cuda.synchronize()
    scale = W.E4M3_SCALE if fmt == "e4m3" else 1.0
    for i in [0, 100, cfg["n"] - 1]:
        want = O.preprocess_nv12(frames[i], 640, 640, pad=114.0, mul=1 / 255)
        check_output(out[i], want, fmt, scale, f"{fmt} frame {i} shape {best}")


# ------------------------------------------------------------------ row-staged NV12 kernel (bulk copies into shared memory)

def _staged_shapes(F, p):
    return [s for s in F.fkl_pipeline_shapes(p.handle) if s[3] <= 0]


@pytest.mark.parametrize("fmt", ["bf16", "e4m3", "f16", "f32"])
@pytest.mark.parametrize("hw,out_wh", [
    ((720, 1280), (640, 640)),   # letterbox: band rows above and below
    ((720, 1280), (640, 600)),   # 600 rows: the last job of every image is ragged
    ((80, 80), (40, 40)),        # width 40: V = 16 does not divide it (register kernel)
])
def test_every_nv12_launch_shape_gives_the_same_bytes(F, W, fmt, hw, out_wh):
    """Scalar (V=4), vector and row-staged launches of one chain agree bit for bit."""
    frames = synth.nv12_frames(11, 3, *hw)
    dev = torch.from_numpy(frames).cuda()
    ow, oh = out_wh
    ops = [F.read_nv12(), F.letterbox(ow, oh, 114.0), F.mul(W.INV255),
           F.write_split(code(F, fmt), W.E4M3_SCALE if fmt == "e4m3" else None)]
    srcs = [dev[i] for i in range(3)]
    base = run_batch(F, ops, srcs, None, (3, 3, oh, ow), fmt, layout_in=F.FKL_LAYOUT_NV12)
    p = F.Pipeline(ops)
    assert _staged_shapes(F, p), "row-staged shapes are listed for NV12 split outputs"
    for shape in F.fkl_pipeline_shapes(p.handle):
        got = run_batch(F, ops, srcs, None, (3, 3, oh, ow), fmt, layout_in=F.FKL_LAYOUT_NV12, shape=shape)
        assert torch.equal(got.view(torch.uint8), base.view(torch.uint8)), shape
    F.fkl_device_check()
    scale = W.E4M3_SCALE if fmt == "e4m3" else 1.0
    rgb = O.nv12_to_rgb(frames[2])
    want = O.split(O.multiply(O.letterbox(rgb, ow, oh, 114.0), 1 / 255))
    check_output(got[2], want, fmt, scale, f"staged {fmt} {hw}->{out_wh}")


def test_row_staged_kernel_many_images_and_normalise(F, W):
    """300 images (two launches of the 256-entry parameter table), swap + normalise tail."""
    n = 300
    frames = synth.nv12_frames(12, n, 64, 128)
    dev = torch.from_numpy(frames).cuda()
    ops = [F.read_nv12(), F.resize(64, 32), F.swap_rb(), F.mul(W.INV255), F.sub(W.IMAGENET_MEAN),
           F.div(W.IMAGENET_STD), F.write_split(F.FKL_F16)]
    srcs = [dev[i] for i in range(n)]
    base = run_batch(F, ops, srcs, None, (n, 3, 32, 64), "f16", layout_in=F.FKL_LAYOUT_NV12)
    p = F.Pipeline(ops)
    for shape in _staged_shapes(F, p):
        got = run_batch(F, ops, srcs, None, (n, 3, 32, 64), "f16", layout_in=F.FKL_LAYOUT_NV12, shape=shape)
        assert torch.equal(got.view(torch.int16), base.view(torch.int16)), shape
    F.fkl_device_check()
    for i in [0, 255, 256, n - 1]:
        t = O.swap_rb(O.resize_bilinear(O.nv12_to_rgb(frames[i]), 64, 32))
        want = O.split(O.divide(O.subtract(O.multiply(t, 1 / 255), W.IMAGENET_MEAN), W.IMAGENET_STD))
        check_output(got[i], want, "f16", 1.0, f"staged normalise image {i}")


def test_row_staged_shape_falls_back_on_unaligned_crops(F, W):
    """A crop whose x offset is not a multiple of 16 makes the batch ineligible."""
    frames = synth.nv12_frames(13, 2, 96, 160)
    dev = torch.from_numpy(frames).cuda()
    ops = [F.read_nv12(), F.resize(64, 32), F.mul(W.INV255), F.write_split(F.FKL_BF16)]
    rois = np.array([[8, 4, 128, 64], [16, 2, 128, 64]], np.int32)
    srcs = [dev[0], dev[1]]
    base = run_batch(F, ops, srcs, rois, (2, 3, 32, 64), "bf16", layout_in=F.FKL_LAYOUT_NV12)
    p = F.Pipeline(ops)
    for shape in _staged_shapes(F, p):
        got = run_batch(F, ops, srcs, rois, (2, 3, 32, 64), "bf16", layout_in=F.FKL_LAYOUT_NV12, shape=shape)
        assert torch.equal(got.view(torch.int16), base.view(torch.int16)), shape
    F.fkl_device_check()
    for i in range(2):
        x, y, w, h = rois[i]
        t = O.resize_bilinear(O.nv12_to_rgb(frames[i])[y:y + h, x:x + w], 64, 32)
        check_output(got[i], O.split(O.multiply(t, 1 / 255)), "bf16", 1.0, f"fallback image {i}")


def test_row_staged_wait_limit_reports_timeout_and_device_stays_usable(F, W):
    """A consumer wait that runs out sets the device flag; the kernel drains
    its own copies and leaves, and the next launch is whole again."""
    frames = synth.nv12_frames(14, 64, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    ops = W.nv12_letterbox_chain(F.FKL_BF16)
    srcs = [dev[i] for i in range(64)]
    base = run_batch(F, ops, srcs, None, (64, 3, 640, 640), "bf16", layout_in=F.FKL_LAYOUT_NV12)
    F.fkl_device_check()
    shape = (8, 128, 4, -2)
    try:
        F.fkl_set_device_wait_limit(1)  # 1 ns: every wait that has to wait at all gives up
        run_batch(F, ops, srcs, None, (64, 3, 640, 640), "bf16", layout_in=F.FKL_LAYOUT_NV12, shape=shape)
        with pytest.raises(F.FklError) as e:
            F.fkl_device_check()
        assert e.value.status == F.FKL_ERR_TIMEOUT
    finally:
        F.fkl_set_device_wait_limit(0)
    F.fkl_device_check()  # cleared by the previous call
    got = run_batch(F, ops, srcs, None, (64, 3, 640, 640), "bf16", layout_in=F.FKL_LAYOUT_NV12, shape=shape)
    F.fkl_device_check()
    assert torch.equal(got.view(torch.int16), base.view(torch.int16))


# ------------------------------------------------------------------ typed chains (§VI-I data types)

_TD = {"u8": "FKL_U8", "u16": "FKL_U16", "f32": "FKL_F32", "f64": "FKL_F64"}


def _typed_run(F, ops, xs, dst, shape=None, unfused=False, offset=0):
    """Run a typed chain over device copies of xs (views starting `offset`
    elements in, to test unaligned pointers); returns the output on the host."""
    dev = [torch.from_numpy(x).cuda()[offset:] for x in xs]
    L = dev[0].numel() if dev else 0
    out = torch.full((len(xs) * L,), float("nan"), dtype=tdtype(dst) if dst == "f32" else torch.float64,
                     device="cuda")
    p = F.Pipeline(ops)
    if shape is not None:
        F.fkl_pipeline_set_shape(p.handle, shape)
    ins = [F.as_fkl(d) for d in dev]
    if unfused:
        F.fkl_execute_batch_unfused(p.handle, ins, None, F.as_fkl(out), 0, 0)
    else:
        F.fkl_execute_batch(p.handle, ins, None, F.as_fkl(out))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _bits_equal(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()


@pytest.mark.parametrize("src", ["u8", "u16", "f32", "f64"])
@pytest.mark.parametrize("dst", ["f32", "f64"])
def test_typed_chain_bit_exact_every_shape_and_unfused(F, W, src, dst):
    cfg = W.DTYPES
    L = cfg["rows"] * cfg["cols"]
    xs = [synth.linear_values(100 + i, L, src) for i in range(cfg["n"])]
    ops = W.typed_chain(getattr(F, _TD[src]), getattr(F, _TD[dst]), cfg["mul"], cfg["sub"], cfg["div"])
    want = np.concatenate([O.typed_chain(x, dst, cfg["mul"], cfg["sub"], cfg["div"]) for x in xs])
    p = F.Pipeline(ops)
    for shape in F.fkl_pipeline_shapes(p.handle):
        assert _bits_equal(_typed_run(F, ops, xs, dst, shape=shape), want), shape
    assert _bits_equal(_typed_run(F, ops, xs, dst, unfused=True), want)


@pytest.mark.parametrize("src,dst", [("u8", "f32"), ("u16", "f64"), ("f64", "f32"), ("f32", "f64")])
def test_typed_chain_edges(F, W, src, dst):
    si, di = getattr(F, _TD[src]), getattr(F, _TD[dst])
    # ragged length and unaligned views (scalar loads and stores)
    xs = [synth.linear_values(7 + i, 1003, src) for i in range(3)]
    ops = W.typed_chain(si, di, 3.0, -0.5, 7.0)
    for off in (0, 1):
        want = np.concatenate([O.typed_chain(x[off:], dst, 3.0, -0.5, 7.0) for x in xs])
        for shape in [(8, 128, 1, 1), (16, 256, 1, 1)]:
            assert _bits_equal(_typed_run(F, ops, xs, dst, shape=shape, offset=off), want), (off, shape)
    # more than 256 tensors (two launches), partial chains
    xs = [synth.linear_values(300 + i, 40, src) for i in range(300)]
    for kw in [dict(div=3.0), dict(mul=0.1), dict(sub=2.0), {}]:
        ops = W.typed_chain(si, di, **kw)
        want = np.concatenate([O.typed_chain(x, dst, **kw) for x in xs])
        assert _bits_equal(_typed_run(F, ops, xs, dst), want), kw
        assert _bits_equal(_typed_run(F, ops, xs, dst, unfused=True), want), kw
    # empty batch and empty tensors are no-ops
    p = F.Pipeline(W.typed_chain(si, di, 2.0))
    out = torch.zeros(4, dtype=torch.float64 if dst == "f64" else torch.float32, device="cuda")
    F.fkl_execute_batch(p.handle, [], None, F.as_fkl(out[:0]))
    e = torch.from_numpy(synth.linear_values(1, 4, src)).cuda()[:0]
    F.fkl_execute_batch(p.handle, [F.as_fkl(e)], None, F.as_fkl(out[:0]))
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0


def _decode(F, t, fmt):
    """Values of a device tensor of bf16 / f16 / e4m3 codes as float64 (host)."""
    if fmt == "bf16":
        b = t.view(torch.int16).cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
        return b.view(np.float32).astype(np.float64)
    if fmt == "f16":
        return t.view(torch.int16).cpu().numpy().view(np.float16).astype(np.float64)
    return O.decode_e4m3(t.view(torch.uint8).cpu().numpy())


_NARROW = {"bf16": (torch.bfloat16, "FKL_BF16"), "f16": (torch.float16, "FKL_F16"),
           "e4m3": (getattr(torch, "float8_e4m3fn", None), "FKL_E4M3")}


def _narrow_cases():
    for src in ("u8", "u16", "f64"):
        for dst in ("bf16", "f16"):
            yield src, dst, None
        for scale in (0.75, 1 / 448):
            yield src, "e4m3", scale


@pytest.mark.parametrize("src,dst,scale", list(_narrow_cases()))
def test_typed_chain_narrow_outputs(F, W, src, dst, scale):
    """bf16 / f16 writes are bit-exact against the oracle (round to nearest
    even of the float32 chain value). The FP8 write stores sat_RNE(v / s);
    the kernel forms v / s as the float32 product v * fl32(1/s), which can
    sit on the other side of an E4M3 tie than the exact quotient, so E4M3 is
    held to the 1-ulp rule of the other narrow formats (at s = 0.75 and
    s = 1/448, neither reciprocal exact in float32), on every launch shape
    and in both unfused forms."""
    tdt, code_name = _NARROW[dst]
    ops = W.typed_chain(getattr(F, _TD[src]), getattr(F, code_name), 1 / 255, 100.0, 0.229, scale=scale)
    xs = [synth.linear_values(60 + i, 2001, src) for i in range(5)]
    want = np.concatenate([O.typed_chain(x, dst, 1 / 255, 100.0, 0.229, scale=scale) for x in xs])
    if dst == "e4m3":  # the unrounded float32 chain values, for the 1-ulp rule
        v32 = np.concatenate([O.typed_chain(x, "f32", 1 / 255, 100.0, 0.229) for x in xs]).astype(np.float64)
        s32 = float(np.float32(scale))
        assert np.array_equal(O.round_e4m3(v32 / s32), want)

    def check(got, what):
        if dst == "e4m3":
            err = check_lowp(got, v32, "e4m3", s32, what)
            assert err["frac_correctly_rounded"] > 0.99, err
        else:
            assert np.array_equal(got, want), what

    dev = [torch.from_numpy(x).cuda() for x in xs]
    ins = [F.as_fkl(d) for d in dev]
    p = F.Pipeline(ops)
    out = torch.zeros(5 * 2001, dtype=tdt, device="cuda")
    for shape in F.fkl_pipeline_shapes(p.handle):
        F.fkl_pipeline_set_shape(p.handle, shape)
        F.fkl_execute_batch(p.handle, ins, None, F.as_fkl(out))
        torch.cuda.synchronize()
        check(_decode(F, out, dst), shape)
    fused = _decode(F, out, dst)
    for static in (False, True):  # unfused: a float32 workspace, or the static scratch
        out.zero_()
        if static:
            F.fkl_execute_batch_unfused_static(p.handle, ins, None, F.as_fkl(out))
        else:
            nb = F.fkl_unfused_workspace_bytes(p.handle, ins, None, F.as_fkl(out))
            assert nb >= 2001 * 4
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            F.fkl_execute_batch_unfused(p.handle, ins, None, F.as_fkl(out), ws.data_ptr(), nb)
        torch.cuda.synchronize()
        got = _decode(F, out, dst)
        check(got, static)
        assert np.array_equal(got, fused), static  # the unfused forms run the same Op code


@pytest.mark.slow
@pytest.mark.parametrize("dst", ["bf16", "f16", "e4m3"])
def test_device_cast_exhaustive_over_0_to_448(F, W, dst):
    """Every float32 bit pattern in [0, 448] (0x00000000 .. 0x43E00000), cast
    on the GPU by the write of a typed chain, equals the oracle's rounding
    written from the format definitions (round to nearest even; FP8 with
    scale 1 saturates at 448)."""
    tdt, code_name = _NARROW[dst]
    ops = [F.read_f32(), F.write_packed(getattr(F, code_name), 1.0 if dst == "e4m3" else None)]
    p = F.Pipeline(ops)
    last, chunk = 0x43E00000, 1 << 25
    rnd = {"bf16": O.round_bf16, "f16": O.round_f16, "e4m3": O.round_e4m3}[dst]
    out = torch.empty(chunk, dtype=tdt, device="cuda")
    for start in range(0, last + 1, chunk):
        end = min(start + chunk, last + 1)
        x = torch.arange(start, end, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.float32)
        o = out[:end - start]
        F.fkl_execute_batch(p.handle, [F.as_fkl(x)], None, F.as_fkl(o))
        torch.cuda.synchronize()
        host = np.arange(start, end, dtype=np.uint32).view(np.float32)
        want = rnd(host.astype(np.float64))
        got = _decode(F, o, dst)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (dst, hex(start + int(bad[0])), got[bad[0]], want[bad[0]])


# ------------------------------------------------------------------ pinned host buffers read and written by the kernel

def test_mapped_host_buffers_match_device_path(F, W):
    frames = synth.nv12_frames(15, 6, 720, 1280)
    ops = W.nv12_letterbox_chain(F.FKL_BF16)
    p = F.Pipeline(ops)
    dev_in = torch.from_numpy(frames).cuda()
    base = torch.empty((6, 3, 640, 640), dtype=torch.bfloat16, device="cuda")
    F.fkl_execute_batch(p.handle, [F.as_fkl(dev_in[i], F.FKL_LAYOUT_NV12) for i in range(6)], None,
                        F.as_fkl(base, F.FKL_LAYOUT_NCHW))
    host_in = torch.from_numpy(frames).pin_memory()
    host_out = torch.zeros((6, 3, 640, 640), dtype=torch.bfloat16).pin_memory()
    ins_h = [F.as_fkl(host_in[i], F.FKL_LAYOUT_NV12) for i in range(6)]
    F.fkl_execute_batch_mapped(p.handle, ins_h, None, F.as_fkl(host_out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    assert torch.equal(host_out.view(torch.int16), base.cpu().view(torch.int16))
    # mixed: host inputs, device output
    dev_out = torch.zeros_like(base)
    F.fkl_execute_batch_mapped(p.handle, ins_h, None, F.as_fkl(dev_out, F.FKL_LAYOUT_NCHW))
    torch.cuda.synchronize()
    assert torch.equal(dev_out.view(torch.int16), base.view(torch.int16))
    want = O.preprocess_nv12(frames[5], 640, 640, pad=114.0, mul=1 / 255)
    check_output(host_out[5], want, "bf16", 1.0, "mapped frame 5")


def test_mapped_typed_chain_and_pageable_memory_is_refused(F, W):
    xs = [synth.linear_values(31 + i, 5000, "u16") for i in range(4)]
    ops = W.typed_chain(F.FKL_U16, F.FKL_F32, 1 / 255, 0.5, 0.25)
    p = F.Pipeline(ops)
    want = np.concatenate([O.typed_chain(x, "f32", 1 / 255, 0.5, 0.25) for x in xs])
    host = [torch.from_numpy(x).pin_memory() for x in xs]
    out = torch.full((4 * 5000,), float("nan")).pin_memory()
    F.fkl_execute_batch_mapped(p.handle, [F.as_fkl(h) for h in host], None, F.as_fkl(out))
    torch.cuda.synchronize()
    assert _bits_equal(out.numpy(), want)
    pageable = torch.from_numpy(xs[0].copy())          # ordinary host memory: never handed to a kernel
    out2 = torch.full((5000,), -1.0).pin_memory()
    with pytest.raises(F.FklError) as e:
        F.fkl_execute_batch_mapped(p.handle, [F.as_fkl(pageable)], None, F.as_fkl(out2))
    assert e.value.status == F.FKL_ERR_INVALID
    torch.cuda.synchronize()
    assert float(out2[0]) == -1.0


def test_dynamic_fp8_scale_is_the_same_on_every_launch_shape(F, W):
    """fkl_execute_batch_scaled reads the device-side 1/s in every kernel form
    (register kernels, the row-staged kernel): identical codes."""
    frames = synth.nv12_frames(18, 3, 720, 1280)
    dev = torch.from_numpy(frames).cuda()
    ins = [F.as_fkl(dev[i], F.FKL_LAYOUT_NV12) for i in range(3)]
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, scale=1.0))
    stats = torch.zeros(32, device="cuda")
    probe = torch.zeros((3, 3, 640, 640), dtype=torch.float8_e4m3fn, device="cuda")
    F.fkl_reduce_batch(p.handle, ins, None, F.as_fkl(probe, F.FKL_LAYOUT_NCHW), stats.data_ptr())
    outs = []
    for shape in [(8, 16, 8, 1), (16, 8, 16, 1), (8, 16, 8, 2), (16, 128, 4, -2), (8, 128, 2, -2)]:
        F.fkl_pipeline_set_shape(p.handle, shape)
        out = torch.zeros_like(probe)
        F.fkl_execute_batch_scaled(p.handle, ins, None, F.as_fkl(out, F.FKL_LAYOUT_NCHW), stats.data_ptr() + 11 * 4)
        outs.append(out)
    torch.cuda.synchronize()
    F.fkl_device_check()
    for o in outs[1:]:
        assert torch.equal(o.view(torch.uint8), outs[0].view(torch.uint8))
    assert outs[0].view(torch.uint8).max().item() == 0x7E


def test_typed_chain_replays_in_a_cuda_graph(F, W):
    xs = [torch.from_numpy(synth.linear_values(90 + i, 4096, "f64")).cuda() for i in range(8)]
    p = F.Pipeline(W.typed_chain(F.FKL_F64, F.FKL_BF16, 1 / 3, 0.25, 0.5))
    ins = [F.as_fkl(x) for x in xs]
    out = torch.zeros(8 * 4096, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        F.fkl_execute_batch(p.handle, ins, None, F.as_fkl(out), stream=s)  # warm
        torch.cuda.synchronize()
        out.zero_()
        with torch.cuda.graph(g, stream=s):
            F.fkl_execute_batch(p.handle, ins, None, F.as_fkl(out), stream=s)
    g.replay()
    torch.cuda.synchronize()
    want = np.concatenate([O.typed_chain(x.cpu().numpy(), "bf16", 1 / 3, 0.25, 0.5) for x in xs])
    assert np.array_equal(_decode(F, out, "bf16"), want)


@pytest.mark.parametrize("fmt", ["f32", "e4m3"])
@pytest.mark.parametrize("src", ["nv12", "packed"])
def test_pillarbox_fill_columns_every_shape(F, W, src, fmt):
    """A portrait image letterboxed into a square: fill columns left and right.
    Spans wholly in the fill run the chain once, spans across the window edge
    mix fill and image pixels; every launch shape, the unfused form and the
    oracle agree."""
    ow = oh = 128
    scale = W.E4M3_SCALE if fmt == "e4m3" else None
    if src == "nv12":
        frames = synth.nv12_frames(23, 2, 320, 180)        # window 72 x 128 at x = 28
        srcs = [torch.from_numpy(frames[i]).cuda() for i in range(2)]
        layout, read = F.FKL_LAYOUT_NV12, F.read_nv12()
        rgb = [O.nv12_to_rgb(frames[i]) for i in range(2)]
    else:
        imgs = [synth.packed_image(24 + i, 300, 170) for i in range(2)]   # window 73 x 128 at x = 27
        srcs = [torch.from_numpy(im).cuda() for im in imgs]
        layout, read = None, F.read_u8c3()
        rgb = [im.astype(np.float64) for im in imgs]
    ops = [read, F.letterbox(ow, oh, 114.0), F.mul(W.INV255), F.write_split(code(F, fmt), scale)]
    base = run_batch(F, ops, srcs, None, (2, 3, oh, ow), fmt, layout_in=layout)
    unf = run_batch(F, ops, srcs, None, (2, 3, oh, ow), fmt, layout_in=layout, unfused=True)
    assert torch.equal(base.view(torch.uint8), unf.view(torch.uint8))
    p = F.Pipeline(ops)
    for shape in F.fkl_pipeline_shapes(p.handle):
        got = run_batch(F, ops, srcs, None, (2, 3, oh, ow), fmt, layout_in=layout, shape=shape)
        assert torch.equal(got.view(torch.uint8), base.view(torch.uint8)), shape
    F.fkl_device_check()
    for i in range(2):
        want = O.split(O.multiply(O.letterbox(rgb[i], ow, oh, 114.0), 1 / 255))
        check_output(base[i], want, fmt, W.E4M3_SCALE if fmt == "e4m3" else 1.0, f"pillarbox {src} {fmt}")
        cols = O.letterbox_geometry(rgb[i].shape[1], rgb[i].shape[0], ow, oh)
        assert cols[2] > 0, "the window is inset: there are fill columns"


def test_reduce_empty_batch_gives_the_documented_stats(F, W):
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, scale=1.0))
    out = torch.zeros((1, 3, 640, 640), dtype=torch.float8_e4m3fn, device="cuda")   # fixes the size only
    stats = torch.full((32,), 7.0, device="cuda")
    F.fkl_reduce_batch(p.handle, [], None, F.as_fkl(out, F.FKL_LAYOUT_NCHW), stats.data_ptr())
    torch.cuda.synchronize()
    st = stats.cpu().numpy()
    assert np.isnan(st[0:6]).all()                      # no value: no extremes
    assert (st[6:9] == 0).all() and st[9] == 0 and st[10] == 1 and st[11] == 1


def test_largest_dimension(F, W):
    """16384 pixels along a row, the largest size the ABI accepts: the packed
    reader (general resize) and the NV12 exact-2x vector path agree with the
    oracle and with their unfused forms."""
    src = synth.packed_image(25, 64, 16384)
    ops = W.normalize_chain(16384, 32)                    # 1x horizontally, 2x vertically
    d = torch.from_numpy(src).cuda()
    got = run_batch(F, ops, [d], None, (1, 3, 32, 16384), "f32")
    unf = run_batch(F, ops, [d], None, (1, 3, 32, 16384), "f32", unfused=True)
    assert torch.equal(got.view(torch.int32), unf.view(torch.int32))
    want = O.preprocess_packed(src, (0, 0, 16384, 64), 16384, 32, swap=True, mul=1 / 255,
                               sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(got)[0], want, "16384-wide packed")

    frames = synth.nv12_frames(26, 1, 64, 16384)
    ops = [F.read_nv12(), F.resize(8192, 32), F.mul(W.INV255), F.write_split(F.FKL_BF16)]
    dev = torch.from_numpy(frames).cuda()
    got = run_batch(F, ops, [dev[0]], None, (1, 3, 32, 8192), "bf16", layout_in=F.FKL_LAYOUT_NV12)
    unf = run_batch(F, ops, [dev[0]], None, (1, 3, 32, 8192), "bf16", layout_in=F.FKL_LAYOUT_NV12, unfused=True)
    assert torch.equal(got.view(torch.int16), unf.view(torch.int16))
    want = O.split(O.multiply(O.resize_bilinear(O.nv12_to_rgb(frames[0]), 8192, 32), 1 / 255))
    check_output(got[0], want, "bf16", 1.0, "16384-wide NV12")


@pytest.mark.parametrize("src", ["nv12", "packed"])
def test_reduce_pillarbox_fill_columns(F, W, src):
    """ReduceDPP over a portrait image letterboxed into a square: spans wholly
    in the fill columns are reduced from one chain evaluation, spans across
    the window edge pixel by pixel; the statistics match the oracle's."""
    ow = oh = 128
    if src == "nv12":
        frames = synth.nv12_frames(27, 2, 320, 180)
        srcs = [torch.from_numpy(frames[i]).cuda() for i in range(2)]
        layout, read = F.FKL_LAYOUT_NV12, F.read_nv12()
        rgb = [O.nv12_to_rgb(frames[i]) for i in range(2)]
    else:
        imgs = [synth.packed_image(28 + i, 300, 170) for i in range(2)]
        srcs = [torch.from_numpy(im).cuda() for im in imgs]
        layout, read = None, F.read_u8c3()
        rgb = [im.astype(np.float64) for im in imgs]
    p = F.Pipeline([read, F.letterbox(ow, oh, 114.0), F.mul(W.INV255), F.write_split(F.FKL_E4M3, 1.0)])
    out = torch.zeros((2, 3, oh, ow), dtype=torch.float8_e4m3fn, device="cuda")
    stats = torch.zeros(32, device="cuda")
    F.fkl_reduce_batch(p.handle, [F.as_fkl(s, layout) for s in srcs], None, F.as_fkl(out, F.FKL_LAYOUT_NCHW),
                       stats.data_ptr())
    torch.cuda.synchronize()
    st = stats.cpu().numpy().astype(np.float64)
    vals = np.stack([O.split(O.multiply(O.letterbox(rgb[i], ow, oh, 114.0), 1 / 255)) for i in range(2)])
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-6)
    check_f32(st[9], want["amax"], "amax")


# ------------------------------------------------------------------ the per-op form over the batch


def _per_op(F, ops, srcs, rois, out_shape, fmt, layout_in=None, chunk=0, timed=False):
    p = F.Pipeline(ops)
    out = torch.full(out_shape, float("nan") if fmt not in ("u8", "e4m3") else 0, dtype=tdtype(fmt), device="cuda")
    layout = F.FKL_LAYOUT_NCHW if out_shape[1] == 3 else F.FKL_LAYOUT_NHWC
    ins = [F.as_fkl(s, layout_in) for s in srcs]
    o = F.as_fkl(out, layout)
    nb = F.fkl_per_op_workspace_bytes(p.handle, ins, rois, o, chunk)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device="cuda")
    rep = F.fkl_execute_batch_per_op(p.handle, ins, rois, o, ws.data_ptr(), nb, chunk=chunk, timed=timed)
    torch.cuda.synchronize()
    return out, rep, nb


@pytest.mark.parametrize("fmt", ["bf16", "e4m3", "f32", "f16"])
def test_per_op_nv12_equals_fused_bitwise(F, W, fmt):
    """One kernel per op over the batch (decode, letterbox, x1/255, split +
    cast) gives the fused kernel's bytes; chunks of 3 frames (ragged last
    chunk) give the same."""
    frames = synth.nv12_frames(31, 5, 720, 1280)
    dev = [torch.from_numpy(f).cuda() for f in frames]
    ops = W.nv12_letterbox_chain(code(F, fmt))
    fused = run_batch(F, ops, dev, None, (5, 3, 640, 640), fmt, layout_in=F.FKL_LAYOUT_NV12)
    bits = torch.int8 if fmt == "e4m3" else (torch.int32 if fmt == "f32" else torch.int16)
    for chunk in (0, 3):
        got, _, _ = _per_op(F, ops, dev, None, (5, 3, 640, 640), fmt, F.FKL_LAYOUT_NV12, chunk=chunk)
        assert torch.equal(got.view(bits), fused.view(bits)), chunk
    want = O.preprocess_nv12(frames[4], 640, 640, pad=114.0, mul=1 / 255)
    check_output(got[4], want, fmt, W.E4M3_SCALE if fmt == "e4m3" else 1.0, "per-op frame 4")


def test_per_op_packed_crops_equal_fused_and_report_kernels(F, W):
    """The 50-crop normalise chain: one kernel per op over all crops equals
    the fused kernel bit for bit; the timed call names every kernel in chain
    order with its launches, algorithmic bytes and time."""
    cfg = W.HF
    src = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
    rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
    d = torch.from_numpy(src).cuda()
    ops = W.normalize_chain(cfg["out_w"], cfg["out_h"])
    shape = (cfg["n"], 3, cfg["out_h"], cfg["out_w"])
    fused = run_batch(F, ops, [d] * cfg["n"], rois, shape, "f32")
    got, rep, nb = _per_op(F, ops, [d] * cfg["n"], rois, shape, "f32", timed=True)
    assert torch.equal(got.view(torch.int32), fused.view(torch.int32))
    names = [r[0] for r in rep]
    assert names == ["crop + resize u8 -> f32", "BGR <-> RGB", "multiply", "subtract", "divide", "split + cast"]
    px = cfg["n"] * cfg["out_h"] * cfg["out_w"]
    assert all(r[1] == 1 and r[3] > 0 for r in rep), rep
    assert rep[1][2] == 24 * px and rep[5][2] == 24 * px  # read 12 B + write 12 B per pixel
    assert nb == 2 * cfg["n"] * ((cfg["out_h"] * cfg["out_w"] * 12 + 767) // 768 * 768)  # packed: both slots output-size
    # chunks of 16: four rounds of every kernel, the same bytes
    got, rep, _ = _per_op(F, ops, [d] * cfg["n"], rois, shape, "f32", chunk=16, timed=True)
    assert torch.equal(got.view(torch.int32), fused.view(torch.int32))
    assert all(r[1] == 4 for r in rep), rep


def test_per_op_nv12_mixed_windows_and_normalise(F, W):
    """Frames of two sizes (one decode launch per run of equal windows), a
    general (non-2x) letterbox and the full normalise chain."""
    small = synth.nv12_frames(32, 2, 360, 640)
    big = synth.nv12_frames(33, 2, 720, 1280)
    srcs = [torch.from_numpy(f).cuda() for f in (small[0], big[0], big[1], small[1])]
    ops = [F.read_nv12(), F.letterbox(300, 200, 114.0), F.swap_rb(), F.mul(W.INV255), F.sub(W.IMAGENET_MEAN),
           F.div(W.IMAGENET_STD), F.write_split(F.FKL_F16)]
    fused = run_batch(F, ops, srcs, None, (4, 3, 200, 300), "f16", layout_in=F.FKL_LAYOUT_NV12)
    got, rep, _ = _per_op(F, ops, srcs, None, (4, 3, 200, 300), "f16", F.FKL_LAYOUT_NV12, timed=True)
    assert torch.equal(got.view(torch.int16), fused.view(torch.int16))
    assert rep[0][0] == "decode NV12 -> RGB f32" and rep[0][1] == 3  # runs: small, big x2, small


def test_per_op_refuses_other_families(F, W):
    p = F.Pipeline(W.integer_chain())
    src = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FklError) as ei:
        F.fkl_per_op_workspace_bytes(p.handle, [F.as_fkl(src)], None, F.as_fkl(out, F.FKL_LAYOUT_NHWC))
    assert ei.value.status == F.FKL_ERR_UNSUPPORTED


# ------------------------------------------------------------------ tile-staged packed reader (shared memory)


def _tile_shapes(F, p):
    return [s for s in F.fkl_pipeline_shapes(p.handle) if s[3] == -1]


@pytest.mark.parametrize("case", ["hf_crops", "upscale", "odd_pitch", "letterbox"])
def test_tile_staged_reader_equals_register_reader(F, W, case):
    """The packed reader that stages each tile's tap rows in shared memory
    (16-byte loads, ends byte by byte) gives the register reader's bytes on
    every tile shape, and the oracle's values."""
    if case == "hf_crops":
        cfg = W.HF
        src = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
        rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
        ow, oh = cfg["out_w"], cfg["out_h"]
        ops = W.normalize_chain(ow, oh)
        t = torch.from_numpy(src).cuda()
        ins = [t] * len(rois)
    elif case == "upscale":
        src = synth.packed_image(34, 30, 41)
        rois = np.array([[0, 0, 41, 30], [3, 2, 17, 11], [40, 29, 1, 1]], np.int32)
        ow, oh = 97, 61
        ops = W.normalize_chain(ow, oh)
        t = torch.from_numpy(src).cuda()
        ins = [t] * 3
    elif case == "odd_pitch":
        full = synth.packed_image(35, 120, 203)                   # rows of 609 bytes, viewed with a 5-byte gap
        host = np.zeros((120, 614), np.uint8)
        host[:, :609] = full.reshape(120, 609)
        dev = torch.from_numpy(host).cuda()
        view = torch.as_strided(dev, (120, 203, 3), (614, 3, 1), storage_offset=0)
        src = full
        rois = np.array([[0, 0, 203, 120], [1, 1, 200, 117], [77, 13, 101, 99]], np.int32)
        ow, oh = 64, 48
        ops = W.normalize_chain(ow, oh)
        ins = [view] * 3
    else:
        src = synth.packed_image(36, 300, 170)
        rois = None
        ow, oh = 128, 96
        ops = [F.read_u8c3(), F.letterbox(ow, oh, 114.0), F.swap_rb(), F.mul(W.INV255), F.write_split(F.FKL_F32)]
        t = torch.from_numpy(src).cuda()
        ins = [t] * 2
    n = len(ins)
    p = F.Pipeline(ops)
    shapes = _tile_shapes(F, p)
    assert shapes
    base = run_batch(F, ops, ins, rois, (n, 3, oh, ow), "f32", shape=(2, 16, 8, 1))
    for shape in shapes:
        got = run_batch(F, ops, ins, rois, (n, 3, oh, ow), "f32", shape=shape)
        assert torch.equal(got.view(torch.int32), base.view(torch.int32)), (case, shape)
    if case == "letterbox":
        want = np.stack([O.split(O.multiply(O.swap_rb(O.letterbox(src.astype(np.float64), ow, oh, 114.0)), 1 / 255))
                         for _ in range(n)])
    else:
        want = O.preprocess_packed_batch([src] * n, rois, ow, oh, swap=True, mul=1 / 255,
                                         sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(base), want, case)


def test_tile_staged_reader_falls_back_when_a_span_is_too_wide(F, W):
    """A 16384-pixel-wide row shrunk to 128 columns: a tile's tap span does not
    fit shared memory, so the tile shape runs the register reader (same bytes)."""
    src = synth.packed_image(37, 24, 16384)
    ops = W.normalize_chain(128, 12)
    d = torch.from_numpy(src).cuda()
    p = F.Pipeline(ops)
    base = run_batch(F, ops, [d], None, (1, 3, 12, 128), "f32", shape=(2, 16, 8, 1))
    for shape in _tile_shapes(F, p):
        got = run_batch(F, ops, [d], None, (1, 3, 12, 128), "f32", shape=shape)
        assert torch.equal(got.view(torch.int32), base.view(torch.int32)), shape
    want = O.preprocess_packed(src, (0, 0, 16384, 24), 128, 12, swap=True, mul=1 / 255,
                               sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    check_f32(to_numpy(base)[0], want, "16384 -> 128")


@pytest.mark.parametrize("w", [724, 722])
def test_per_op_nv12_decode_widths(F, W, w):
    """The per-op decode kernel with coalesced stores (window width a multiple
    of 4; 724 ends in a partial 128-pixel segment) and the generic decode
    (722): both give the fused kernel's bytes."""
    frames = synth.nv12_frames(38, 3, 362, w)
    dev = [torch.from_numpy(f).cuda() for f in frames]
    ops = [F.read_nv12(), F.letterbox(300, 200, 114.0), F.mul(W.INV255), F.write_split(F.FKL_BF16)]
    fused = run_batch(F, ops, dev, None, (3, 3, 200, 300), "bf16", layout_in=F.FKL_LAYOUT_NV12)
    got, _, _ = _per_op(F, ops, dev, None, (3, 3, 200, 300), "bf16", F.FKL_LAYOUT_NV12)
    assert torch.equal(got.view(torch.int16), fused.view(torch.int16))
    want = O.split(O.multiply(O.letterbox(O.nv12_to_rgb(frames[2]), 300, 200, 114.0), 1 / 255))
    check_output(got[2], want, "bf16", 1.0, f"per-op width {w}")


def test_reduce_over_two_launches_twice_on_one_buffer(F, W):
    """300 images take two reduction launches (256 images each at most); the
    block that completes both writes the statistics. The same stats buffer
    is used twice in a row: the second call starts from a cleared
    accumulator and gives the same bytes. Extremes equal the float32
    write's; mean and amax match the oracle."""
    n = 300
    src = synth.packed_image(31, 48, 64)
    rng = np.random.default_rng(5)
    rois = np.zeros((n, 4), np.int32)
    for i in range(n):
        w, h = int(rng.integers(8, 65)), int(rng.integers(6, 49))
        rois[i] = (int(rng.integers(0, 64 - w + 1)), int(rng.integers(0, 48 - h + 1)), w, h)
    ops = [F.read_u8c3(), F.resize(40, 30), F.swap_rb(), F.mul(1 / 255), F.sub(W.IMAGENET_MEAN),
           F.div(W.IMAGENET_STD), F.write_split(F.FKL_F32)]
    d = torch.from_numpy(src).cuda()
    got = run_batch(F, ops, [d] * n, rois, (n, 3, 30, 40), "f32")
    p = F.Pipeline(ops)
    runs = []
    for _ in range(2):
        stats = torch.full((32,), 7.0, device="cuda") if not runs else runs[0][1]
        F.fkl_reduce_batch(p.handle, [F.as_fkl(d)] * n, rois, F.as_fkl(got, F.FKL_LAYOUT_NCHW), stats.data_ptr())
        torch.cuda.synchronize()
        runs.append((stats[:14].clone(), stats))
    assert torch.equal(runs[0][0].view(torch.int32), runs[1][0].view(torch.int32))
    st, jobs, grid = _reduce_split(runs[1][1])
    assert jobs > grid > 0
    per_c = got.permute(1, 0, 2, 3).reshape(3, -1)
    assert np.array_equal(st[0:3].astype(np.float32), per_c.min(dim=1).values.cpu().numpy())
    assert np.array_equal(st[3:6].astype(np.float32), per_c.max(dim=1).values.cpu().numpy())
    vals = O.preprocess_packed_batch([src] * n, rois, 40, 30, swap=True, mul=1 / 255,
                                     sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
    want = O.reduce_stats(vals)
    check_f32(st[0:3], want["min"], "min")
    check_f32(st[3:6], want["max"], "max")
    np.testing.assert_allclose(st[6:9], want["mean"], rtol=1e-5, atol=1e-6)
    check_f32(st[9], want["amax"], "amax")
