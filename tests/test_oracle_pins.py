"""Pins of the CPU oracle against things other than itself.

Every test here checks an oracle function against a closed form, an invariant,
an independent library routine, a hand-derived worked example under
tests/golden/, or brute force on a tiny input, so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one test.
"""
import json
from fractions import Fraction
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2508_07071_gb300 import synth


def coord_image(h, w, c=3):
    """Pixel value is a known closed form of its coordinates."""
    y, x, ch = np.meshgrid(np.arange(h), np.arange(w), np.arange(c), indexing="ij")
    return ((7 * y + 3 * x + 11 * ch) % 256).astype(np.uint8)


# ---------------------------------------------------------------- crop / swap / split


def test_crop_closed_form():
    img = coord_image(9, 13)
    out = O.crop(img, 5, 2, 4, 3)
    assert out.shape == (3, 4, 3)
    for j in range(3):
        for i in range(4):
            for c in range(3):
                assert out[j, i, c] == (7 * (2 + j) + 3 * (5 + i) + 11 * c) % 256


@pytest.mark.parametrize("roi", [(-1, 0, 2, 2), (0, 0, 14, 1), (12, 8, 2, 2), (0, 0, 0, 3)])
def test_crop_rejects_outside(roi):
    with pytest.raises(ValueError):
        O.crop(coord_image(9, 13), *roi)


def test_swap_is_involution_and_reverses():
    img = synth.packed_image(3, 7, 5)
    assert np.array_equal(O.swap_rb(O.swap_rb(img)), img)
    s = O.swap_rb(img)
    assert np.array_equal(s[..., 0], img[..., 2]) and np.array_equal(s[..., 2], img[..., 0])
    assert np.array_equal(s[..., 1], img[..., 1])


def test_split_closed_form():
    img = coord_image(4, 6)
    planes = O.split(img)
    assert planes.shape == (3, 4, 6)
    for c in range(3):
        for y in range(4):
            for x in range(6):
                assert planes[c, y, x] == (7 * y + 3 * x + 11 * c) % 256


# ---------------------------------------------------------------- bilinear resize


def test_resize_golden_rows(golden_dir):
    spec = json.load(open(os.path.join(golden_dir, "resize_halfpixel_rows.json")))
    for case in spec["cases"]:
        src = np.array(case["src"], dtype=np.float64).reshape(1, -1, 1)
        out = O.resize_bilinear(src, case["dst_w"], 1)
        np.testing.assert_allclose(out[0, :, 0], case["expected"], rtol=0, atol=1e-12)


def test_resize_identity_is_copy():
    img = O.to_float(synth.packed_image(4, 23, 31))
    assert np.array_equal(O.resize_bilinear(img, 31, 23), img)


def test_resize_one_pixel_source_is_constant():
    img = np.full((1, 1, 3), 0.0)
    img[0, 0] = (17.0, 99.0, 250.0)
    out = O.resize_bilinear(img, 9, 5)
    assert np.array_equal(out, np.broadcast_to(img, (5, 9, 3)))


def test_resize_exact_2x_is_block_mean():
    img = O.to_float(synth.packed_image(5, 18, 26))
    out = O.resize_bilinear(img, 13, 9)
    blocks = img.reshape(9, 2, 13, 2, 3).mean(axis=(1, 3))
    np.testing.assert_allclose(out, blocks, rtol=0, atol=1e-12)


def test_resize_exact_4x_uses_middle_pair():
    # scale 4: u = 4d + 1.5, so every output is the mean of source pixels 4d+1, 4d+2
    img = O.to_float(synth.packed_image(6, 16, 24))
    out = O.resize_bilinear(img, 6, 4)
    sub = img[1::4][:, :] + img[2::4][:, :]
    sub = (sub[:, 1::4] + sub[:, 2::4]) / 4.0
    np.testing.assert_allclose(out, sub, rtol=0, atol=1e-12)


def test_resize_reproduces_linear_ramp():
    # S(x, y) = x + 2y; bilinear interpolation is exact on affine functions,
    # so D(d, e) = u(d) + 2 v(e) wherever the sample needs no clamping.
    h, w = 30, 40
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    img = (xs + 2 * ys).astype(np.float64)[..., None]
    out_w, out_h = 17, 23
    out = O.resize_bilinear(img, out_w, out_h)[..., 0]
    u = (np.arange(out_w) + 0.5) * w / out_w - 0.5
    v = (np.arange(out_h) + 0.5) * h / out_h - 0.5
    ok_u = (u >= 0) & (u <= w - 1)
    ok_v = (v >= 0) & (v <= h - 1)
    expect = u[None, :] + 2 * v[:, None]
    mask = ok_v[:, None] & ok_u[None, :]
    assert mask.sum() > 0.8 * mask.size
    np.testing.assert_allclose(out[mask], expect[mask], rtol=0, atol=1e-9)


@pytest.mark.parametrize("src_hw,dst_hw", [((30, 40), (17, 23)), ((7, 5), (19, 13)),
                                           ((480, 640), (224, 224)), ((64, 33), (64, 128)),
                                           ((3, 2), (3, 2)), ((1, 9), (4, 4))])
def test_resize_matches_torch_interpolate(src_hw, dst_hw):
    # torch's bilinear with align_corners=False uses the same half-pixel
    # mapping and border clamp; an independent library routine.
    img = O.to_float(synth.packed_image(7, *src_hw))
    ours = O.resize_bilinear(img, dst_hw[1], dst_hw[0])
    t = torch.from_numpy(np.ascontiguousarray(img.transpose(2, 0, 1)))[None]
    ref = F.interpolate(t, size=dst_hw, mode="bilinear", align_corners=False)[0]
    np.testing.assert_allclose(ours, ref.numpy().transpose(1, 2, 0), rtol=0, atol=1e-9)


def test_resize_is_separable_brute_force():
    # brute force on a tiny image: four explicit taps per output pixel
    img = O.to_float(synth.packed_image(8, 5, 4))
    out = O.resize_bilinear(img, 7, 3)
    for e in range(3):
        v = min(max((e + 0.5) * 5 / 3 - 0.5, 0.0), 4.0)
        y0 = int(np.floor(v)); y1 = min(y0 + 1, 4); b = v - y0
        for d in range(7):
            u = min(max((d + 0.5) * 4 / 7 - 0.5, 0.0), 3.0)
            x0 = int(np.floor(u)); x1 = min(x0 + 1, 3); a = u - x0
            want = ((1 - a) * (1 - b) * img[y0, x0] + a * (1 - b) * img[y0, x1]
                    + (1 - a) * b * img[y1, x0] + a * b * img[y1, x1])
            np.testing.assert_allclose(out[e, d], want, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- NV12 / BT.601


def nv12_from_planes(luma, u, v):
    h, w = luma.shape
    uv = np.empty((h // 2, w), dtype=np.uint8)
    uv[:, 0::2] = u
    uv[:, 1::2] = v
    return np.concatenate([luma, uv], axis=0)


def test_bt601_coefficients_closed_form():
    c_y, c_rv, c_gu, c_gv, c_bu = O.bt601_limited_coefficients()
    np.testing.assert_allclose([c_y, c_rv, c_gu, c_gv, c_bu],
                               [1.164383562, 1.596026786, 0.391762290, 0.812967647, 2.017232143],
                               atol=1e-8)


def test_nv12_black_white_gray():
    for yv, want in [(16, 0.0), (235, 255.0), (126, 110 * 255 / 219)]:
        f = nv12_from_planes(np.full((4, 6), yv, np.uint8), np.full((2, 3), 128, np.uint8),
                             np.full((2, 3), 128, np.uint8))
        np.testing.assert_allclose(O.nv12_to_rgb(f), want, atol=1e-9)


def test_nv12_inverts_bt601_forward_transform():
    # Decode integer NV12 frames with the oracle, then re-encode the RGB with
    # the forward BT.601 definition, E'Y = Kr R + Kg G + Kb B,
    # E'Cb = (B - E'Y) / (2 (1 - Kb)), E'Cr = (R - E'Y) / (2 (1 - Kr)),
    # Y = 16 + 219 E'Y, Cb = 128 + 224 E'Cb, Cr = 128 + 224 E'Cr (E' = RGB/255):
    # every pixel that needed no clamping must give back its Y, U, V.
    frame = synth.nv12_frames(12, 1, 32, 48, lo=60, hi=190)[0]
    rgb = O.nv12_to_rgb(frame)
    kr, kb = 0.299, 0.114
    kg = 1 - kr - kb
    e = rgb / 255.0
    ey = kr * e[..., 0] + kg * e[..., 1] + kb * e[..., 2]
    Y = 16 + 219 * ey
    U = 128 + 224 * (e[..., 2] - ey) / (2 * (1 - kb))
    V = 128 + 224 * (e[..., 0] - ey) / (2 * (1 - kr))
    luma = frame[:32].astype(np.float64)
    u = np.repeat(np.repeat(frame[32:, 0::2], 2, axis=0), 2, axis=1).astype(np.float64)
    v = np.repeat(np.repeat(frame[32:, 1::2], 2, axis=0), 2, axis=1).astype(np.float64)
    inside = np.all((rgb > 0) & (rgb < 255), axis=-1)
    assert inside.sum() > 100
    np.testing.assert_allclose(Y[inside], luma[inside], atol=1e-9)
    np.testing.assert_allclose(U[inside], u[inside], atol=1e-9)
    np.testing.assert_allclose(V[inside], v[inside], atol=1e-9)


def test_nv12_decode_matches_per_pixel_brute_force():
    frame = synth.nv12_frames(9, 1, 6, 8)[0]
    out = O.nv12_to_rgb(frame)
    c_y, c_rv, c_gu, c_gv, c_bu = O.bt601_limited_coefficients()
    for y in range(6):
        for x in range(8):
            Y = float(frame[y, x])
            U = float(frame[6 + y // 2, 2 * (x // 2)])
            V = float(frame[6 + y // 2, 2 * (x // 2) + 1])
            r = c_y * (Y - 16) + c_rv * (V - 128)
            g = c_y * (Y - 16) - c_gu * (U - 128) - c_gv * (V - 128)
            b = c_y * (Y - 16) + c_bu * (U - 128)
            want = np.clip([r, g, b], 0, 255)
            np.testing.assert_allclose(out[y, x], want, atol=1e-12)


def test_nv12_clamps():
    f = nv12_from_planes(np.full((2, 2), 255, np.uint8), np.full((1, 1), 255, np.uint8),
                         np.full((1, 1), 255, np.uint8))
    rgb = O.nv12_to_rgb(f)
    assert rgb.max() == 255.0 and rgb.min() >= 0.0
    assert rgb[0, 0, 0] == 255.0 and rgb[0, 0, 2] == 255.0


# ---------------------------------------------------------------- letterbox


def test_letterbox_1280x720_to_640():
    assert O.letterbox_geometry(1280, 720, 640, 640) == (640, 360, 0, 140)
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 255, size=(720, 1280, 3))
    out = O.letterbox(img, 640, 640, 114.0)
    assert np.all(out[:140] == 114.0) and np.all(out[500:] == 114.0)
    blocks = img.reshape(360, 2, 640, 2, 3).mean(axis=(1, 3))
    np.testing.assert_allclose(out[140:500], blocks, rtol=0, atol=1e-10)


def test_letterbox_odd_padding_floor_on_top():
    # 100x51 into 64x64: r = 0.64, height round(32.64) = 33, 31 pad rows: 15 top, 16 bottom
    assert O.letterbox_geometry(100, 51, 64, 64) == (64, 33, 0, 15)
    out = O.letterbox(np.zeros((51, 100, 3)), 64, 64, 7.0)
    assert np.all(out[:15] == 7.0) and np.all(out[48:] == 7.0) and np.all(out[15:48] == 0.0)
    # portrait source pads left/right
    assert O.letterbox_geometry(30, 60, 64, 64) == (32, 64, 16, 0)


# ---------------------------------------------------------------- compute ops


def test_normalise_constant_image_closed_form():
    mean = (0.485, 0.456, 0.406)
    std = (0.229, 0.224, 0.225)
    src = np.empty((4, 4, 3), np.uint8)
    src[..., 0], src[..., 1], src[..., 2] = 10, 20, 30      # B, G, R
    out = O.preprocess_packed(src, (0, 0, 4, 4), 2, 2, swap=True,
                              mul=1 / 255, sub=mean, div=std)
    # after BGR->RGB the first plane is R=30 and uses mean[0], std[0]
    for c, val in enumerate((30, 20, 10)):
        np.testing.assert_allclose(out[c], (val / 255 - mean[c]) / std[c], atol=1e-12)
    np.testing.assert_allclose(out[0, 0, 0], (30 / 255 - 0.485) / 0.229, atol=1e-12)
    np.testing.assert_allclose(out[0, 0, 0], -1.60416130, atol=1e-8)


def test_imagenet_extremes():
    mean = np.array((0.485, 0.456, 0.406)); std = np.array((0.229, 0.224, 0.225))
    lo = O.divide(O.subtract(O.multiply(np.zeros((1, 1, 3)), 1 / 255), mean), std)[0, 0]
    hi = O.divide(O.subtract(O.multiply(np.full((1, 1, 3), 255.0), 1 / 255), mean), std)[0, 0]
    np.testing.assert_allclose(lo, [-2.117904, -2.035714, -1.804444], atol=1e-6)
    np.testing.assert_allclose(hi, [2.248908, 2.428571, 2.640000], atol=1e-6)


def test_add_saturate_u8():
    x = np.array([[[0, 5, 250]]], np.uint8)
    assert O.add_saturate_u8(x, 10).tolist() == [[[10, 15, 255]]]
    assert O.add_saturate_u8(x, -10).tolist() == [[[0, 0, 240]]]
    assert O.add_saturate_u8(x, (1, -6, 5)).tolist() == [[[1, 0, 255]]]


def test_saturate_cast_u8():
    x = np.array([2.5, 3.5, -0.6, 255.5, 254.5, 300.0, 0.49, 127.5])
    assert O.saturate_cast_u8(x).tolist() == [2, 4, 0, 255, 254, 255, 0, 128]


# ---------------------------------------------------------------- output casts


def _random_f32(n, seed, lo_exp=-20, hi_exp=8):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1, 2, n)
    exp = rng.integers(lo_exp, hi_exp, n)
    sign = rng.choice([-1.0, 1.0], n)
    return (sign * np.ldexp(mant, exp)).astype(np.float32)


def test_bf16_matches_torch():
    x = _random_f32(200000, 1, -100, 100)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x.astype(np.float64)), ref)


def test_f16_matches_numpy_half():
    x = np.concatenate([_random_f32(200000, 2, -24, 15).astype(np.float64),
                        np.random.default_rng(3).uniform(-60000, 60000, 10000)])
    ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(O.round_f16(x), ref)


def test_e4m3_matches_torch_float8():
    x = np.concatenate([_random_f32(200000, 4, -12, 9),
                        np.random.default_rng(5).uniform(-448, 448, 20000).astype(np.float32)])
    x = x[np.abs(x) <= 448]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.round_e4m3(x.astype(np.float64)), ref)


def test_e4m3_golden_ties_and_saturation(golden_dir):
    spec = json.load(open(os.path.join(golden_dir, "e4m3_ties.json")))
    for case in spec["cases"]:
        assert O.round_e4m3(np.array([case["q"]]))[0] == case["expected"], case


def test_e4m3_decode_all_codes_round_trip():
    codes = np.arange(256, dtype=np.uint8)
    vals = O.decode_e4m3(codes)
    finite = ~np.isnan(vals)
    assert finite.sum() == 254                      # 0x7F and 0xFF are NaN
    assert np.nanmax(vals) == 448.0 and np.nanmin(vals) == -448.0
    # every finite code is a fixed point of the rounding
    assert np.array_equal(O.round_e4m3(vals[finite]), vals[finite])
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(vals[finite], ref[finite])


def test_decode_bf16():
    x = _random_f32(1000, 6)
    bits = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.decode_bf16(bits), ref)


def test_format_ulp():
    assert O.format_ulp(np.array([1.0]), "bf16")[0] == 2.0 ** -7
    assert O.format_ulp(np.array([1.5]), "f16")[0] == 2.0 ** -10
    assert O.format_ulp(np.array([300.0]), "e4m3")[0] == 32.0
    assert O.format_ulp(np.array([1e-9]), "e4m3")[0] == 2.0 ** -9


def test_quantize_e4m3_scale():
    v = np.array([0.0, 0.5, 1.0, 1.1])
    q = O.quantize_e4m3(v, 1.0 / 448.0)
    assert q.tolist() == [0.0, 224.0, 448.0, 448.0]


# ---------------------------------------------------------------- vertical chain


def test_vertical_chain_no_contraction():
    # x*c0 = 1 + 2^-11 + 2^-24 is a tie at binary32 and rounds to 1 + 2^-11;
    # adding -1 then gives exactly 2^-11. A fused multiply-add would keep the
    # 2^-24 and return 2^-11 + 2^-24.
    x = np.array([1 + 2.0 ** -12], np.float32)
    out = O.vertical_chain_f32(x, [O.KIND_MUL, O.KIND_ADD], [1 + 2.0 ** -12, -1.0])
    assert out[0] == np.float32(2.0 ** -11)


def test_vertical_chain_order():
    x = np.array([2.0], np.float32)
    assert O.vertical_chain_f32(x, [O.KIND_MUL, O.KIND_ADD], [3.0, 1.0])[0] == 7.0
    assert O.vertical_chain_f32(x, [O.KIND_ADD, O.KIND_MUL], [1.0, 3.0])[0] == 9.0


def test_vertical_chain_identity_and_error_bound():
    x = synth.f32_uniform(2, 4096)
    kinds = [O.KIND_MUL, O.KIND_ADD] * 50
    assert np.array_equal(O.vertical_chain_f32(x, kinds, [1.0, 0.0] * 50), x)
    k, c = synth.chain_constants(2, 1000)
    assert k[0] == O.KIND_MUL and k[1] == O.KIND_ADD
    got = O.vertical_chain_f32(x, k, c).astype(np.float64)
    exact = x.astype(np.float64)
    for kind, cc in zip(k, c.astype(np.float64)):
        exact = exact * cc if kind == O.KIND_MUL else exact + cc
    # each of the 1000 ops adds at most half an ulp of a value of magnitude < 2
    assert np.max(np.abs(got - exact)) < 1000 * 2.0 ** -23


# ---------------------------------------------------------------- whole chains


def test_preprocess_chain_is_op_by_op():
    src = synth.packed_image(11, 40, 50)
    roi = (3, 4, 30, 20)
    out = O.preprocess_packed(src, roi, 16, 12, swap=True, mul=2.0, sub=(1, 2, 3), div=(4, 5, 6))
    t = src[4:24, 3:33].astype(np.float64)
    t = F.interpolate(torch.from_numpy(np.ascontiguousarray(t.transpose(2, 0, 1)))[None],
                      size=(12, 16), mode="bilinear", align_corners=False)[0].numpy()
    t = t[::-1]                                            # BGR -> RGB on planes
    want = (t * 2.0 - np.array([1, 2, 3.0])[:, None, None]) / np.array([4, 5, 6.0])[:, None, None]
    np.testing.assert_allclose(out, want, atol=1e-10)


def test_integer_chain_bit_exact_brute_force():
    src = coord_image(9, 13)
    out = O.integer_chain_packed(src, (2, 1, 5, 4), swap=True, add_k=(100, -50, 0))
    for j in range(4):
        for i in range(5):
            for c in range(3):
                val = (7 * (1 + j) + 3 * (2 + i) + 11 * (2 - c)) % 256
                val = min(255, max(0, val + (100, -50, 0)[c]))
                assert out[j, i, c] == val


# ---------------------------------------------------------------- parity rule itself


def test_lowp_rule_accepts_roundings_inside_the_f32_bound_only():
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from parity import check_lowp
    o = np.array([8.2607667e-05, 1.0, 0.3])
    # correct roundings pass
    check_lowp(O.round_f16(o), o, "f16")
    # near zero: a rounding of a value 1e-7 away (inside 1e-6) passes
    check_lowp(O.round_f16(o - np.array([1e-7, 0, 0])), o, "f16")
    # two ulps away at 1.0 fails
    with pytest.raises(AssertionError):
        check_lowp(np.array([O.round_f16(o)[0], 1.0 + 2 * 2.0 ** -10, 0.3]), o, "f16")
    # a value 1e-5 away near zero fails
    with pytest.raises(AssertionError):
        check_lowp(O.round_f16(o - np.array([1e-5, 0, 0])), o, "f16")


def test_reduce_stats_closed_forms():
    v = np.zeros((2, 3, 4, 5))
    v[:, 0] = 7.0
    v[:, 1, 0, 0] = -3.0          # one negative pixel per image in channel 1
    v[:, 2] = np.arange(20).reshape(4, 5)
    st = O.reduce_stats(v)
    assert st["min"].tolist() == [7.0, -3.0, 0.0]
    assert st["max"].tolist() == [7.0, 0.0, 19.0]
    np.testing.assert_allclose(st["mean"], [7.0, -3.0 / 20, 9.5])
    assert st["amax"] == 19.0 and st["scale"] == 19.0 / 448
    assert O.reduce_stats(np.zeros((3, 2, 2)))["scale"] == 1.0


# ------------------------------------------------------------------ typed chains (§VI-I data types)

def _f32_bits(v):
    return int(np.array(v, dtype=np.float32).view(np.uint32))


def test_typed_cast_f64_to_f32_rounds_ties_to_even():
    # 1 + 2^-24 lies halfway between 1 and 1 + 2^-23: the even neighbour is 1.
    # 1 + 3*2^-24 lies halfway between 1 + 2^-23 and 1 + 2^-22: the even one is 1 + 2^-22.
    # 1 + 2^-24 + 2^-50 is just above the first midpoint: rounds up.
    x = np.array([1 + 2.0**-24, 1 + 3 * 2.0**-24, 1 + 2.0**-24 + 2.0**-50, -(1 + 2.0**-24)])
    y = O.typed_chain(x, "f32")
    assert [_f32_bits(v) for v in y] == [0x3F800000, 0x3F800002, 0x3F800001, 0xBF800000]


def test_typed_cast_integers_are_exact():
    assert O.typed_chain(np.array([0, 65535], np.uint16), "f32").tolist() == [0.0, 65535.0]
    assert O.typed_chain(np.array([255], np.uint8), "f64").tolist() == [255.0]
    x = np.float32(0.1)
    assert Fraction(float(O.typed_chain(np.array([x]), "f64")[0])) == Fraction(float(x))


def test_typed_chain_exact_rationals_and_op_order():
    # with mul 2, sub 1, div 4 every step is exact in binary: y = (2x - 1) / 4
    x = np.array([0, 1, 3, 255], np.uint8)
    for ct in ("f32", "f64"):
        y = O.typed_chain(x, ct, mul=2, sub=1, div=4)
        assert [Fraction(float(v)) for v in y] == [Fraction(2 * int(v) - 1, 4) for v in x]
    # Mul before Sub: 3*2 - 1 = 5 (not 2*(3 - 1) = 4)
    assert O.typed_chain(np.array([3], np.uint8), "f32", mul=2, sub=1)[0] == 5.0


def test_typed_chain_constants_are_float32_values():
    # the descriptor carries float32: a f64 chain multiplies by fl32(0.1), not 0.1
    y = O.typed_chain(np.array([1.0]), "f64", mul=0.1)[0]
    assert Fraction(float(y)) == Fraction(float(np.float32(0.1))) != Fraction(0.1)


def _correctly_rounded(y, exact: Fraction, ct) -> bool:
    """y is the ct value nearest to `exact`, ties to the even significand."""
    y = ct(y)
    lo, hi = np.nextafter(y, ct(-np.inf)), np.nextafter(y, ct(np.inf))
    d = abs(Fraction(float(y)) - exact)
    for nb in (lo, hi):
        dn = abs(Fraction(float(nb)) - exact)
        if dn < d:
            return False
        if dn == d:  # a tie: y must have the even significand
            bits = int(np.array(y).view(np.uint32 if ct is np.float32 else np.uint64))
            if bits & 1:
                return False
    return True


@pytest.mark.parametrize("ct,name", [(np.float32, "f32"), (np.float64, "f64")])
def test_typed_ops_are_correctly_rounded(ct, name):
    """Each op alone equals the exact rational result rounded to nearest even
    (checked against both neighbours with exact fractions)."""
    rng = np.random.default_rng(7)
    xs = rng.uniform(-4, 4, 40).astype(ct)
    cs = [np.float32(0.3), np.float32(-1.7), np.float32(1 / 3), np.float32(2.5e-3)]
    for c in cs:
        C = Fraction(float(c))
        for x in xs:
            X = Fraction(float(x))
            assert _correctly_rounded(O.typed_chain(np.array([x]), name, mul=c)[0], X * C, ct)
            assert _correctly_rounded(O.typed_chain(np.array([x]), name, sub=c)[0], X - C, ct)
            assert _correctly_rounded(O.typed_chain(np.array([x]), name, div=c)[0], X / C, ct)


def _round_exact(q: Fraction, ct):
    """The ct value nearest to the rational q, ties to even (brute force
    around a first guess; independent of numpy's arithmetic)."""
    y = ct(float(q))  # within a couple of ulps of q
    for _ in range(4):
        best = y
        for nb in (np.nextafter(y, ct(-np.inf)), np.nextafter(y, ct(np.inf))):
            dn, db = abs(Fraction(float(nb)) - q), abs(Fraction(float(best)) - q)
            odd = int(np.array(best).view(np.uint32 if ct is np.float32 else np.uint64)) & 1
            if dn < db or (dn == db and odd):
                best = nb
        if best == y:
            return y
        y = best
    return y


@pytest.mark.parametrize("src,name", [("f64", "f32"), ("u16", "f32"), ("f32", "f64"), ("u8", "f32")])
def test_typed_chain_rounds_after_every_op(src, name):
    """Cast, Mul, Sub, Div each rounded to the compute type in turn (an f32
    chain evaluated in f64 and rounded once would fail here)."""
    ct = np.float32 if name == "f32" else np.float64
    x = synth.linear_values(5, 300, src)
    m, s, d = np.float32(1 / 255), np.float32(0.485), np.float32(0.229)
    y = O.typed_chain(x, name, mul=m, sub=s, div=d)
    M, S, D = (Fraction(float(c)) for c in (m, s, d))
    for xi, yi in zip(x, y):
        t = _round_exact(Fraction(float(xi)), ct)
        t = _round_exact(Fraction(float(t)) * M, ct)
        t = _round_exact(Fraction(float(t)) - S, ct)
        t = _round_exact(Fraction(float(t)) / D, ct)
        assert np.array(t).tobytes() == np.array(yi, dtype=ct).tobytes(), (xi, yi, t)


def test_f16_overflow_matches_numpy_half():
    x = np.array([65504.0, 65519.99, 65520.0, 70000.0, -65520.0, 1e9, -65519.0])
    want = np.array(x, dtype=np.float64).astype(np.float16).astype(np.float64)
    got = O.round_f16(x)
    assert np.array_equal(got, want), (got, want)
    assert np.isinf(got[2]) and got[1] == 65504.0


def test_typed_chain_narrow_outputs_against_torch():
    """16-bit writes equal an independent library's conversion of the float32
    chain (torch's bf16 / f16 casts round to nearest even)."""
    x = synth.linear_values(9, 5000, "u16")
    y32 = O.typed_chain(x, "f32", mul=1 / 255, sub=100.0, div=0.229)
    t = torch.from_numpy(y32)
    assert np.array_equal(O.typed_chain(x, "bf16", 1 / 255, 100.0, 0.229),
                          t.to(torch.bfloat16).double().numpy())
    assert np.array_equal(O.typed_chain(x, "f16", 1 / 255, 100.0, 0.229),
                          t.to(torch.float16).double().numpy())


# Every finite non-negative E4M3 value with its code (codes 0x00 .. 0x7E), as
# exact rationals: (-1)^0 * 2^(e - 7) * (1 + m/8), subnormals 2^-6 * m/8.
_E4M3_GRID = [(Fraction(m, 8) * Fraction(2) ** -6 if e == 0 else (1 + Fraction(m, 8)) * Fraction(2) ** (e - 7),
               (e << 3) | m) for e in range(16) for m in range(8) if (e, m) != (15, 7)]


def _e4m3_rne_exact(q: Fraction) -> Fraction:
    """Round an exact rational to E4M3: nearest value, ties to the even code,
    magnitudes beyond 448 saturate (OCP satfinite)."""
    sign = -1 if q < 0 else 1
    a = abs(q)
    if a >= 448:
        return sign * Fraction(448)
    best, code = min(_E4M3_GRID, key=lambda vc: (abs(vc[0] - a), vc[1] & 1))
    return sign * best


@pytest.mark.parametrize("scale", [0.75, 1 / 448, 3.0, 0.1])
def test_typed_chain_e4m3_is_the_rounded_exact_quotient(scale):
    """The FP8 write stores sat_RNE(v / s), v the float32 chain value and s the
    float32 scale, checked against the exact rational quotient rounded by
    enumeration of the E4M3 grid. The inputs include values whose quotient
    sits one float32 step below or above an E4M3 tie: there v * fl32(1/s) (a
    reciprocal's product, rounded to float32 before the cast) lands on the
    tie itself and rounds the other way, so an oracle built on that product
    fails here."""
    s32 = np.float32(scale)
    S = Fraction(float(s32))
    # ties of E4M3 between 1 and 2 (1 + (2k+1)/16) and in the subnormal range,
    # moved back by the scale and nudged one float32 step either way
    ties = [(1 + Fraction(2 * k + 1, 16)) for k in range(8)] + [Fraction(2 * k + 1, 1024) for k in range(4)]
    near = []
    for tq in ties:
        v = np.float32(float(tq * S))
        near += [np.nextafter(v, np.float32(-np.inf)), v, np.nextafter(v, np.float32(np.inf))]
    x = np.concatenate([np.array(near, np.float32), synth.linear_values(9, 3000, "f32"),
                        np.array([0.0, -0.0, 500.0 * float(s32), -1e6, 1e-30], np.float32)])
    got = O.typed_chain(x, "e4m3", scale=scale)
    for xi, gi in zip(x, got):
        assert Fraction(float(gi)) == _e4m3_rne_exact(Fraction(float(xi)) / S), (xi, gi, scale)
    # the same inputs through a reciprocal's float32 product round differently
    # for some of them at s = 0.75 (fl32(4/3) is inexact), so the pin has power
    if scale == 0.75:
        prod = O.round_e4m3(np.multiply(x, np.float32(1.0 / float(s32)), dtype=np.float32).astype(np.float64))
        assert np.any(prod != got)
