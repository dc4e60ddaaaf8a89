"""Measurement helpers: algorithmic bytes of a chain and clock sampling.

Algorithmic bytes of a fused launch = the distinct source bytes its bilinear
taps reference + the output bytes it writes. The tap footprint of one image
is a product set (distinct tap rows x distinct tap columns) of the half-pixel
mapping, so it is counted exactly on the host.
"""
from __future__ import annotations

import ctypes
import threading
import time

import numpy as np


def _axis_taps(n_src: int, n_dst: int) -> np.ndarray:
    """Distinct source indices referenced along one axis (half-pixel rule)."""
    if n_dst <= 0:
        return np.zeros(0, dtype=np.int64)
    d = np.arange(n_dst, dtype=np.int64)
    num = (2 * d + 1) * n_src - n_dst          # u = num / (2 n_dst)
    q = np.floor_divide(num, 2 * n_dst)
    r = num - q * 2 * n_dst
    i0 = np.clip(q, 0, n_src - 1)
    i1 = np.where((q >= 0) & (q < n_src - 1) & (r > 0), i0 + 1, i0)
    return np.unique(np.concatenate([i0, i1]))


def letterbox_size(src_w, src_h, out_w, out_h):
    sc = min(out_w / src_w, out_h / src_h)
    dw = max(1, min(out_w, int(np.floor(src_w * sc + 0.5))))
    dh = max(1, min(out_h, int(np.floor(src_h * sc + 0.5))))
    return dw, dh


def packed_tap_bytes(rw, rh, dw, dh) -> int:
    return int(len(_axis_taps(rw, dw)) * len(_axis_taps(rh, dh)) * 3)


def nv12_tap_bytes(rx, ry, rw, rh, dw, dh) -> int:
    xs = _axis_taps(rw, dw) + rx
    ys = _axis_taps(rh, dh) + ry
    luma = len(xs) * len(ys)
    chroma = len(np.unique(xs // 2)) * len(np.unique(ys // 2)) * 2
    return int(luma + chroma)


def out_bytes(n, h, w, bytes_per_el, channels=3) -> int:
    return int(n * h * w * channels * bytes_per_el)


SECTOR = 32  # bytes per DRAM sector


def _row_sectors(starts: np.ndarray, offsets: np.ndarray) -> int:
    """32-byte sectors touched by bytes `offsets` of rows starting at `starts`
    (row starts are absolute byte addresses from a 32-byte aligned base)."""
    total = 0
    for st in np.asarray(starts, dtype=np.int64):
        total += len(np.unique((st + offsets) // SECTOR))
    return total


def packed_tap_sector_bytes(rx, ry, rw, rh, dw, dh, pitch) -> int:
    """Sector-level source footprint of one crop's bilinear taps in a packed
    3-channel u8 image (base 32-byte aligned, `pitch` bytes per row)."""
    xs = _axis_taps(rw, dw) + rx
    cols = (3 * xs[:, None] + np.arange(3)[None, :]).ravel()
    rows = (_axis_taps(rh, dh) + ry) * int(pitch)
    return SECTOR * _row_sectors(rows, cols)


def nv12_tap_sector_bytes(rx, ry, rw, rh, dw, dh, pitch, height) -> int:
    """Sector-level footprint of the NV12 taps: luma rows, then the chroma
    plane (U, V pairs) starting `height` rows after the luma base."""
    xs = _axis_taps(rw, dw) + rx
    ys = _axis_taps(rh, dh) + ry
    luma = _row_sectors(ys * int(pitch), xs)
    cx = np.unique(xs // 2)
    ccols = (2 * cx[:, None] + np.arange(2)[None, :]).ravel()
    chroma = _row_sectors((height + np.unique(ys // 2)) * int(pitch), ccols)
    return SECTOR * (luma + chroma)


def planar_out_sector_bytes(n, h, w, bytes_per_el, channels=3) -> int:
    """Sectors written by dense [n, C, h, w] planes (32-byte aligned base)."""
    row = w * bytes_per_el
    starts = np.arange(n * channels * h, dtype=np.int64) * row
    first, last = starts // SECTOR, (starts + row - 1) // SECTOR
    # rows may share a sector at their boundary: count distinct sectors
    return SECTOR * int(len(np.unique(np.concatenate([np.arange(a, b + 1) for a, b in zip(first, last)])))
                        if row % SECTOR else np.sum(last - first + 1))


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """Samples SM clock, max clock and clock-event reasons through NVML
    (libnvidia-ml, read-only queries) on a background thread."""

    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, index: int = 0, period_s: float = 0.002):
        self.period = period_s
        self.samples = []
        self.ok = False
        self._stop = threading.Event()
        self._thread = None
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))
            self.max_mhz = mx.value
            self._reasons = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.ok = True
        except OSError:
            self.ok = False

    def _sample(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        pw = ctypes.c_uint()
        self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk))
        self._reasons(self.h, ctypes.byref(rs))
        self.nvml.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(pw))
        return (time.perf_counter(), clk.value, rs.value, pw.value / 1000.0)

    def _run(self):
        while not self._stop.is_set():
            self.samples.append(self._sample())
            time.sleep(self.period)

    def start(self):
        if self.ok:
            self.samples.append(self._sample())
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()

    def stop(self):
        if self._thread:
            self._stop.set()
            self._thread.join()
            self.samples.append(self._sample())

    def summary(self) -> dict:
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable: NVML not loaded"]}
        mhz = [s[1] for s in self.samples]
        mask = 0
        for s in self.samples:
            mask |= s[2]
        reasons = [name for bit, name in self.REASONS.items() if mask & bit]
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": float(self.max_mhz),
                "sm_mhz_min": float(min(mhz)), "power_w_max": float(max(s[3] for s in self.samples)),
                "samples": len(self.samples), "reasons": reasons}
