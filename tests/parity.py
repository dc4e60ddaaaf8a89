"""Comparison rules of the parity tests (CUDA path vs the CPU oracle).

* float32 outputs: |g - o| <= 1e-5 |o| + 1e-6 elementwise. The kernels
  compute in float32; the analysis of the worst case (exact integer bilinear
  weights, then ~6 roundings before the normalise step, each at most half an
  ulp of a value below 2^8, divided by std >= 0.224 and by 255) bounds the
  absolute error near zero by about 7e-7, so the 1e-6 floor covers outputs
  that cross zero, where a purely relative bound is meaningless.
* bf16 / f16 / FP8-E4M3 outputs: |g - round_fmt(o)| <= 1 ulp_fmt(o), i.e. the
  stored value is the correctly rounded oracle value or its neighbour (the
  float32 value fed to the rounding can sit on the other side of a tie).
  Near zero, where a normalised value comes out of a cancellation
  (v/255 - mean), the float32 intermediate carries the absolute error the
  float32 rule allows (1e-6), which can exceed one ulp of the format (f16
  spacing below 6.1e-5 is 6e-8). There the stored value must be a correct
  rounding of some value inside the float32 bound:
  round_fmt(o - d) <= g <= round_fmt(o + d), d = 1e-5 |o| + 1e-6.
* integer / byte outputs: bit-exact.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as O

F32_RTOL = 1e-5
F32_ATOL = 1e-6


def to_numpy(t: torch.Tensor) -> np.ndarray:
    if t.dtype == torch.float8_e4m3fn:
        return O.decode_e4m3(t.view(torch.uint8).cpu().numpy())
    if t.dtype in (torch.bfloat16, torch.float16):
        return t.float().cpu().numpy().astype(np.float64)
    return t.cpu().numpy()


def check_f32(got, want, what=""):
    g = np.asarray(got, dtype=np.float64)
    o = np.asarray(want, dtype=np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    err = np.abs(g - o)
    bound = F32_RTOL * np.abs(o) + F32_ATOL
    bad = err > bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} outside |g-o| <= 1e-5|o| + 1e-6; "
                           f"max err {err.max():.3g} at {np.unravel_index(err.argmax(), err.shape)}")
    return float(err.max())


def check_lowp(got_values, want, fmt: str, scale: float = 1.0, what=""):
    """got_values are the decoded stored values (for e4m3: the codes' values,
    i.e. v / scale); want is the float64 oracle value v."""
    g = np.asarray(got_values, dtype=np.float64)
    o = np.asarray(want, dtype=np.float64) / scale
    assert g.shape == o.shape, (g.shape, o.shape)
    rnd = {"bf16": O.round_bf16, "f16": O.round_f16, "e4m3": O.round_e4m3}[fmt]
    ref = rnd(o)
    ulp = O.format_ulp(o, fmt)
    err = np.abs(g - ref)
    d = (F32_RTOL * np.abs(o * scale) + F32_ATOL) / scale
    inside_f32_bound = (g >= rnd(o - d)) & (g <= rnd(o + d))
    bad = (err > ulp) & ~inside_f32_bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} values more than 1 {fmt} ulp from the "
                           f"rounded oracle; worst {err.max():.3g}")
    exact = float(np.mean(err == 0))
    return {"max_abs_err_vs_fp64": float(np.max(np.abs(g - o)) * scale),
            "mean_abs_err_vs_fp64": float(np.mean(np.abs(g - o)) * scale),
            "frac_correctly_rounded": exact}


def check_output(out: torch.Tensor, want: np.ndarray, fmt: str, scale: float = 1.0, what=""):
    if fmt == "f32":
        return check_f32(to_numpy(out), want, what)
    return check_lowp(to_numpy(out), want, fmt, scale, what)


_cudart = None


def copy_device(ptr: int, nbytes: int) -> torch.Tensor:
    """Copy `nbytes` of device memory at a raw pointer into a new uint8
    tensor on the GPU (for outputs the library hands back as pointers)."""
    import ctypes
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("libcudart.so.13")
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _cudart.cudaMemcpy.restype = ctypes.c_int
    out = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rc = _cudart.cudaMemcpy(out.data_ptr(), ptr, nbytes, 3)  # device to device
    assert rc == 0, f"cudaMemcpy failed with {rc}"
    return out
