"""ctypes binding of the C ABI in include/fkl.h.

The functions here carry the C names and only marshal arguments: torch
tensors become ``fkl_tensor`` structs (pointer, dims, row pitch, dtype,
layout), op descriptors become ``fkl_op_desc`` arrays, and the CUDA stream is
passed as a raw handle. Every computation runs in libfkl.so. Importing this
module loads the library and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfkl.so")

# status codes
FKL_OK, FKL_ERR_INVALID, FKL_ERR_UNSUPPORTED, FKL_ERR_OOM, FKL_ERR_CUDA, FKL_ERR_TIMEOUT = range(6)
# element types
FKL_U8, FKL_F32, FKL_F16, FKL_BF16, FKL_E4M3, FKL_U16, FKL_F64 = range(7)
# layouts
FKL_LAYOUT_LINEAR, FKL_LAYOUT_HWC, FKL_LAYOUT_NV12, FKL_LAYOUT_NCHW, FKL_LAYOUT_NHWC = range(5)
# op codes
FKL_OP_READ_U8C3 = 1
FKL_OP_READ_NV12 = 2
FKL_OP_READ_F32 = 3
FKL_OP_READ_U8 = 4
FKL_OP_READ_U16 = 5
FKL_OP_READ_F64 = 6
FKL_OP_CROP = 10
FKL_OP_RESIZE = 11
FKL_OP_LETTERBOX = 12
FKL_OP_SWAP_RB = 20
FKL_OP_MUL = 21
FKL_OP_ADD = 22
FKL_OP_SUB = 23
FKL_OP_DIV = 24
FKL_OP_ADD_SAT_U8 = 25
FKL_OP_WRITE_PACKED = 40
FKL_OP_WRITE_SPLIT = 41


class fkl_tensor(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dims", ctypes.c_int64 * 4),
                ("pitch_bytes", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("layout", ctypes.c_int32)]


class fkl_op_desc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("f", ctypes.c_float * 8), ("i", ctypes.c_int32 * 8)]


class fkl_launch_shape(ctypes.Structure):
    _fields_ = [("vec", ctypes.c_int32), ("tx", ctypes.c_int32), ("ty", ctypes.c_int32),
                ("ry", ctypes.c_int32)]

    def as_tuple(self):
        return (self.vec, self.tx, self.ty, self.ry)


FKL_SERVE_PERSISTENT, FKL_SERVE_BATCH, FKL_SERVE_UNFUSED = range(3)


class fkl_server_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("arena_bytes", ctypes.c_size_t),
                ("ctas_per_sm", ctypes.c_int32), ("idle_us", ctypes.c_int32)]


class fkl_request_info(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_ready", ctypes.c_double),
                ("t_done", ctypes.c_double), ("n_images", ctypes.c_int32), ("state", ctypes.c_int32)]


class fkl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("images_completed", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("arena_peak_bytes", ctypes.c_uint64), ("queued", ctypes.c_int32), ("inflight", ctypes.c_int32)]


class FklError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"fkl status {status}: {message}")
        self.status = status


EXPORTS = {
    # name: (restype, argtypes)
    "fkl_pipeline_create": (ctypes.c_int, [ctypes.POINTER(fkl_op_desc), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "fkl_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fkl_tensor),
                                   ctypes.POINTER(fkl_tensor), ctypes.c_void_p]),
    "fkl_execute_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                         ctypes.c_void_p]),
    "fkl_pipeline_destroy": (None, [ctypes.c_void_p]),
    "fkl_last_error": (ctypes.c_char_p, []),
    "fkl_unfused_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                   ctypes.POINTER(fkl_tensor),
                                                   ctypes.POINTER(ctypes.c_int32),
                                                   ctypes.POINTER(fkl_tensor),
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "fkl_execute_batch_unfused": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.POINTER(fkl_tensor),
                                                 ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(fkl_tensor), ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p]),
    "fkl_execute_batch_unfused_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                        ctypes.POINTER(fkl_tensor),
                                                        ctypes.POINTER(ctypes.c_int32),
                                                        ctypes.POINTER(fkl_tensor), ctypes.c_void_p]),
    "fkl_per_op_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "fkl_execute_batch_per_op": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "fkl_pipeline_kernel_name": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fkl_pipeline_get_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fkl_launch_shape)]),
    "fkl_pipeline_set_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fkl_launch_shape)]),
    "fkl_pipeline_shape_count": (ctypes.c_int32, [ctypes.c_void_p]),
    "fkl_pipeline_shape_at": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(fkl_launch_shape)]),
    "fkl_pipeline_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                             ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(fkl_launch_shape),
                                             ctypes.POINTER(ctypes.c_float)]),
    "fkl_pipeline_autotune_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.POINTER(fkl_tensor),
                                                ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(fkl_tensor), ctypes.c_void_p,
                                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.POINTER(fkl_launch_shape),
                                                ctypes.POINTER(ctypes.c_float)]),
    "fkl_host_executor_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_size_t, ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_void_p)]),
    "fkl_execute_batch_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                              ctypes.c_void_p]),
    "fkl_host_executor_destroy": (None, [ctypes.c_void_p]),
    "fkl_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fkl_server_config),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "fkl_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "fkl_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(fkl_tensor)]),
    "fkl_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                       ctypes.POINTER(fkl_tensor)]),
    "fkl_server_request_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                               ctypes.POINTER(fkl_request_info)]),
    "fkl_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "fkl_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fkl_server_stats)]),
    "fkl_server_destroy": (None, [ctypes.c_void_p]),
    "fkl_reduce_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "fkl_execute_batch_scaled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "fkl_device_check": (ctypes.c_int, []),
    "fkl_execute_batch_mapped": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fkl_tensor),
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fkl_tensor),
                                                ctypes.c_void_p]),
    "fkl_set_device_wait_limit": (ctypes.c_int, [ctypes.c_uint64]),
    "fkl_version": (ctypes.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2508_07071_gb300.build.build() "
                           "(needs nvcc). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status: int):
    if status != FKL_OK:
        raise FklError(status, _lib.fkl_last_error().decode())


# ---------------------------------------------------------------- op descriptors


def _desc(op: int, f: Sequence[float] = (), i: Sequence[int] = ()) -> fkl_op_desc:
    d = fkl_op_desc()
    d.op = op
    for k, v in enumerate(f):
        d.f[k] = float(v)
    for k, v in enumerate(i):
        d.i[k] = int(v)
    return d


def _c3(c) -> list:
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (3,))
    return [float(x) for x in c]


def read_u8c3():
    return _desc(FKL_OP_READ_U8C3)


def read_nv12():
    return _desc(FKL_OP_READ_NV12)


def read_f32():
    return _desc(FKL_OP_READ_F32)


def read_u8():
    return _desc(FKL_OP_READ_U8)


def read_u16():
    return _desc(FKL_OP_READ_U16)


def read_f64():
    return _desc(FKL_OP_READ_F64)


def read_linear(dtype: int):
    """The linear read op of an element type (typed and vertical chains)."""
    return {FKL_U8: read_u8, FKL_U16: read_u16, FKL_F32: read_f32, FKL_F64: read_f64}[dtype]()


def crop(x, y, w, h):
    return _desc(FKL_OP_CROP, i=(x, y, w, h))


def resize(w, h):
    return _desc(FKL_OP_RESIZE, i=(w, h))


def letterbox(w, h, pad):
    return _desc(FKL_OP_LETTERBOX, f=(pad,), i=(w, h))


def swap_rb():
    return _desc(FKL_OP_SWAP_RB)


def mul(c):
    return _desc(FKL_OP_MUL, f=_c3(c))


def add(c):
    return _desc(FKL_OP_ADD, f=_c3(c))


def sub(c):
    return _desc(FKL_OP_SUB, f=_c3(c))


def div(c):
    return _desc(FKL_OP_DIV, f=_c3(c))


def add_sat_u8(k):
    k = np.broadcast_to(np.asarray(k, dtype=np.int64), (3,))
    return _desc(FKL_OP_ADD_SAT_U8, i=[int(x) for x in k])


def write_split(dtype: int, scale: float | None = None):
    return _desc(FKL_OP_WRITE_SPLIT, f=(scale,) if scale is not None else (), i=(dtype,))


def write_packed(dtype: int, scale: float | None = None):
    return _desc(FKL_OP_WRITE_PACKED, f=(scale,) if scale is not None else (), i=(dtype,))


def scalar_op(op: int, c: float) -> fkl_op_desc:
    """MUL/ADD descriptor of a float32 tensor chain (one constant)."""
    return _desc(op, f=(c,))


# ---------------------------------------------------------------- tensors


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    m = {torch.uint8: FKL_U8, torch.float32: FKL_F32, torch.float16: FKL_F16,
         torch.bfloat16: FKL_BF16, torch.float64: FKL_F64}
    if hasattr(torch, "uint16"):
        m[torch.uint16] = FKL_U16
    if hasattr(torch, "float8_e4m3fn"):
        m[torch.float8_e4m3fn] = FKL_E4M3
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _tensor(data_ptr, dims, pitch, dtype, layout) -> fkl_tensor:
    t = fkl_tensor()
    t.data = data_ptr
    for k, v in enumerate(dims):
        t.dims[k] = int(v)
    t.pitch_bytes = int(pitch)
    t.dtype = dtype
    t.layout = layout
    return t


def tensor_hwc(t) -> fkl_tensor:
    """uint8 [H, W, 3] with unit channel and pixel strides (rows may be padded)."""
    if t.dim() != 3 or t.shape[2] != 3 or t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("expected a uint8 [H, W, 3] tensor with packed pixels")
    return _tensor(t.data_ptr(), (t.shape[0], t.shape[1], 3), t.stride(0) * t.element_size(),
                   dtype_code(t), FKL_LAYOUT_HWC)


def tensor_nv12(t) -> fkl_tensor:
    """uint8 [H*3/2, W]: luma rows then interleaved chroma rows, same pitch."""
    if t.dim() != 2 or t.stride(1) != 1 or t.shape[0] % 3:
        raise ValueError("expected a uint8 [H*3/2, W] NV12 tensor")
    return _tensor(t.data_ptr(), (t.shape[0] * 2 // 3, t.shape[1]), t.stride(0), dtype_code(t),
                   FKL_LAYOUT_NV12)


def tensor_nchw(t, dtype: int | None = None) -> fkl_tensor:
    """[N, 3, H, W] with planes H*pitch apart and images 3*H*pitch apart."""
    if t.dim() != 4 or t.stride(3) != 1:
        raise ValueError("expected an [N, C, H, W] tensor with unit column stride")
    n, c, h, w = t.shape
    es = t.element_size()
    pitch = t.stride(2) * es
    if t.stride(1) * es != h * pitch or (n > 1 and t.stride(0) * es != c * h * pitch):
        raise ValueError("NCHW tensor must have planes H*pitch and images C*H*pitch apart")
    return _tensor(t.data_ptr(), (n, c, h, w), pitch, dtype if dtype is not None else dtype_code(t),
                   FKL_LAYOUT_NCHW)


def tensor_nhwc(t, dtype: int | None = None) -> fkl_tensor:
    if t.dim() != 4 or t.stride(3) != 1 or t.stride(2) != t.shape[3]:
        raise ValueError("expected an [N, H, W, C] tensor with packed pixels")
    n, h, w, c = t.shape
    es = t.element_size()
    pitch = t.stride(1) * es
    if n > 1 and t.stride(0) * es != h * pitch:
        raise ValueError("NHWC tensor must have images H*pitch apart")
    return _tensor(t.data_ptr(), (n, h, w, c), pitch, dtype if dtype is not None else dtype_code(t),
                   FKL_LAYOUT_NHWC)


def tensor_linear(t) -> fkl_tensor:
    if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
        raise ValueError("expected a contiguous 1-D tensor")
    return _tensor(t.data_ptr(), (t.numel(),), 0, dtype_code(t), FKL_LAYOUT_LINEAR)


def as_fkl(t, layout: int | None = None, dtype: int | None = None) -> fkl_tensor:
    """Marshal a tensor (or pass an fkl_tensor through)."""
    if isinstance(t, fkl_tensor):
        return t
    if layout is None:
        layout = FKL_LAYOUT_LINEAR if t.dim() == 1 else FKL_LAYOUT_HWC
    if layout == FKL_LAYOUT_HWC:
        return tensor_hwc(t)
    if layout == FKL_LAYOUT_NV12:
        return tensor_nv12(t)
    if layout == FKL_LAYOUT_NCHW:
        return tensor_nchw(t, dtype)
    if layout == FKL_LAYOUT_NHWC:
        return tensor_nhwc(t, dtype)
    return tensor_linear(t)


def _stream(stream) -> int:
    if stream is None:
        torch = _torch()
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C ABI, same names


def fkl_pipeline_create(ops: Sequence[fkl_op_desc]) -> int:
    arr = (fkl_op_desc * len(ops))(*ops)
    h = ctypes.c_void_p()
    _check(_lib.fkl_pipeline_create(arr, len(ops), ctypes.byref(h)))
    return h.value


def fkl_pipeline_destroy(p: int) -> None:
    _lib.fkl_pipeline_destroy(p)


def fkl_last_error() -> str:
    return _lib.fkl_last_error().decode()


def fkl_version() -> str:
    return _lib.fkl_version().decode()


def fkl_device_check() -> None:
    """Raises FklError(FKL_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(_lib.fkl_device_check())


def fkl_set_device_wait_limit(ns: int) -> None:
    """Limit of one bounded device wait (0: the default, 1 s)."""
    _check(_lib.fkl_set_device_wait_limit(int(ns)))


def fkl_pipeline_kernel_name(p: int) -> str:
    return _lib.fkl_pipeline_kernel_name(p).decode()


def fkl_execute(p: int, inp: fkl_tensor, out: fkl_tensor, stream=None) -> None:
    _check(_lib.fkl_execute(p, ctypes.byref(inp), ctypes.byref(out), _stream(stream)))


def _rois(rois):
    if rois is None:
        return None
    r = np.ascontiguousarray(np.asarray(rois, dtype=np.int32).reshape(-1, 4))
    return r, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def fkl_execute_batch(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, stream=None) -> None:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                  _stream(stream)))


def fkl_execute_batch_mapped(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, stream=None) -> None:
    """fkl_execute_batch on pinned host (or device) buffers, read and written
    by the fused kernel over the host link."""
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch_mapped(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                         _stream(stream)))


FKL_REDUCE_STATS_BYTES = 128


def fkl_reduce_batch(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, stats_ptr: int,
                     stream=None) -> None:
    """ReduceDPP: stats (device, 128 bytes) = min[3], max[3], mean[3], amax,
    s = amax/448, 1/s."""
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_reduce_batch(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out), stats_ptr,
                                 _stream(stream)))


def fkl_execute_batch_scaled(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, scale_inv_ptr: int,
                             stream=None) -> None:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch_scaled(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                         scale_inv_ptr, _stream(stream)))


def fkl_unfused_workspace_bytes(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor) -> int:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    n = ctypes.c_size_t()
    _check(_lib.fkl_unfused_workspace_bytes(p, len(ins), arr, keep[1] if keep else None,
                                            ctypes.byref(out), ctypes.byref(n)))
    return n.value


def fkl_execute_batch_unfused(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor,
                              workspace_ptr: int, workspace_bytes: int, stream=None) -> None:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch_unfused(p, len(ins), arr, keep[1] if keep else None,
                                          ctypes.byref(out), workspace_ptr, workspace_bytes,
                                          _stream(stream)))


class fkl_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32), ("bytes", ctypes.c_double),
                ("ms", ctypes.c_double)]


def fkl_per_op_workspace_bytes(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, chunk: int = 0) -> int:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    n = ctypes.c_size_t()
    _check(_lib.fkl_per_op_workspace_bytes(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                           int(chunk), ctypes.byref(n)))
    return n.value


def fkl_execute_batch_per_op(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, workspace_ptr: int,
                             workspace_bytes: int, chunk: int = 0, stream=None, timed: bool = False):
    """The unfused chain with one kernel per op over the batch; with
    `timed`, returns [(name, launches, bytes, ms)] per operation (the call
    then synchronizes the stream)."""
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    times = (fkl_kernel_time * 16)() if timed else None
    nt = ctypes.c_int32()
    _check(_lib.fkl_execute_batch_per_op(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                         int(chunk), workspace_ptr, workspace_bytes, _stream(stream),
                                         ctypes.cast(times, ctypes.c_void_p) if timed else None, 16,
                                         ctypes.byref(nt)))
    if not timed:
        return None
    return [(t.name.decode(), t.launches, t.bytes, t.ms) for t in times[:nt.value]]


def fkl_execute_batch_unfused_static(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor,
                                     stream=None) -> None:
    """Unfused form on the library's static device scratch (no allocation)."""
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch_unfused_static(p, len(ins), arr, keep[1] if keep else None,
                                                 ctypes.byref(out), _stream(stream)))


def fkl_pipeline_get_shape(p: int) -> tuple:
    s = fkl_launch_shape()
    _check(_lib.fkl_pipeline_get_shape(p, ctypes.byref(s)))
    return s.as_tuple()


def fkl_pipeline_set_shape(p: int, shape: Sequence[int]) -> None:
    s = fkl_launch_shape(*[int(v) for v in shape])
    _check(_lib.fkl_pipeline_set_shape(p, ctypes.byref(s)))


def fkl_pipeline_shapes(p: int) -> list:
    out = []
    for k in range(_lib.fkl_pipeline_shape_count(p)):
        s = fkl_launch_shape()
        _check(_lib.fkl_pipeline_shape_at(p, k, ctypes.byref(s)))
        out.append(s.as_tuple())
    return out


_BEFORE = ctypes.CFUNCTYPE(None, ctypes.c_void_p)


def fkl_pipeline_autotune(p: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, stream=None,
                          reps: int = 5, before=None):
    """Returns (best shape, median microseconds per launch). `before()` (a
    Python callable) runs before every timed launch, e.g. an L2 flush."""
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    best = fkl_launch_shape()
    us = ctypes.c_float()
    if before is not None:
        cb = _BEFORE(lambda _user: before())
        _check(_lib.fkl_pipeline_autotune_ex(p, len(ins), arr, keep[1] if keep else None,
                                             ctypes.byref(out), _stream(stream), reps,
                                             ctypes.cast(cb, ctypes.c_void_p), None,
                                             ctypes.byref(best), ctypes.byref(us)))
    else:
        _check(_lib.fkl_pipeline_autotune(p, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                          _stream(stream), reps, ctypes.byref(best), ctypes.byref(us)))
    return best.as_tuple(), us.value


def fkl_host_executor_create(p: int, chunk: int, depth: int, in_bytes: int, out_bytes: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.fkl_host_executor_create(p, chunk, depth, in_bytes, out_bytes, ctypes.byref(h)))
    return h.value


def fkl_host_executor_destroy(e: int) -> None:
    _lib.fkl_host_executor_destroy(e)


def fkl_execute_batch_host(e: int, ins: Sequence[fkl_tensor], rois, out: fkl_tensor, stream=None) -> None:
    arr = (fkl_tensor * max(1, len(ins)))(*ins)
    keep = _rois(rois)
    _check(_lib.fkl_execute_batch_host(e, len(ins), arr, keep[1] if keep else None, ctypes.byref(out),
                                       _stream(stream)))


def fkl_server_create(p: int, mode: int = FKL_SERVE_PERSISTENT, max_inflight: int = 64,
                      arena_bytes: int = 4 << 30, ctas_per_sm: int = 1, idle_us: int = 200000) -> int:
    cfg = fkl_server_config(mode, max_inflight, arena_bytes, ctas_per_sm, idle_us)
    h = ctypes.c_void_p()
    _check(_lib.fkl_server_create(p, ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def fkl_server_submit(s: int, images: Sequence[fkl_tensor]) -> int:
    arr = (fkl_tensor * len(images))(*images)
    rid = ctypes.c_uint64()
    _check(_lib.fkl_server_submit(s, len(images), arr, ctypes.byref(rid)))
    return rid.value


def fkl_server_poll(s: int, rid: int):
    done = ctypes.c_int32()
    out = fkl_tensor()
    _check(_lib.fkl_server_poll(s, rid, ctypes.byref(done), ctypes.byref(out)))
    return bool(done.value), out


def fkl_server_wait(s: int, rid: int, timeout_ms: int = 10000) -> fkl_tensor:
    out = fkl_tensor()
    _check(_lib.fkl_server_wait(s, rid, timeout_ms, ctypes.byref(out)))
    return out


def fkl_server_request_info(s: int, rid: int) -> fkl_request_info:
    info = fkl_request_info()
    _check(_lib.fkl_server_request_info(s, rid, ctypes.byref(info)))
    return info


def fkl_server_release(s: int, rid: int) -> None:
    _check(_lib.fkl_server_release(s, rid))


def fkl_server_get_stats(s: int) -> fkl_server_stats:
    st = fkl_server_stats()
    _check(_lib.fkl_server_get_stats(s, ctypes.byref(st)))
    return st


def fkl_server_destroy(s: int) -> None:
    _lib.fkl_server_destroy(s)


class Pipeline:
    """Owns a pipeline handle (destroyed with the object)."""

    def __init__(self, ops: Sequence[fkl_op_desc]):
        self.handle = fkl_pipeline_create(ops)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            fkl_pipeline_destroy(h)
            self.handle = None

    @property
    def kernel_name(self) -> str:
        return fkl_pipeline_kernel_name(self.handle)
