"""Benchmark of the fused preprocessing path on GB300.

Default workload (N=1): 256 NV12 1280x720 frames -> BT.601 RGB -> letterbox
640x640 (pad 114) -> x1/255 -> planar BF16, one fused launch per step.
value = algorithmic bytes / device time (GB/s), beside the unfused
one-kernel-per-op chain on the same GPU, the HBM roofline of the fused kernel
and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload nv12|single|hf|vchain]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun every rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Fused GB/s vs 8 TB/s HBM & speedup over unfused per-op kernels, same GB300"


def measured_traffic(key: str):
    """DRAM bytes per launch (read + write) from the committed ncu summary,
    or None when the kernel's sources or build flags changed since."""
    from paper_2508_07071_gb300.ncu_traffic import TRAFFIC, entry_hash
    if not os.path.exists(TRAFFIC):
        return None
    d = json.load(open(TRAFFIC)).get(key)
    if not d or d.get("source_hash") != entry_hash(d):
        return None
    return int(d["dram_bytes_per_launch"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ workloads


class Workload:
    """Inputs resident in HBM plus the fused and unfused calls of one step."""

    name = ""
    unit = "GB/s"

    def step(self, stream):  # fused: one pass of the hot path
        raise NotImplementedError

    def step_unfused(self, stream):
        raise NotImplementedError


class NV12Letterbox(Workload):
    def __init__(self, F, W, synth, metrics, torch, n, fmt="bf16", seed=3):
        cfg = W.NV12
        self.F, self.torch = F, torch
        self.n, self.h, self.w, self.out = n, cfg["h"], cfg["w"], cfg["out"]
        self.fmt = fmt
        code = {"bf16": F.FKL_BF16, "f16": F.FKL_F16, "e4m3": F.FKL_E4M3, "f32": F.FKL_F32}[fmt]
        tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "e4m3": torch.float8_e4m3fn,
               "f32": torch.float32}[fmt]
        self.el = {"bf16": 2, "f16": 2, "e4m3": 1, "f32": 4}[fmt]
        self.frames_host = synth.nv12_frames(seed, n, self.h, self.w)
        self.frames = torch.from_numpy(self.frames_host).cuda()
        self.dst = torch.empty((n, 3, self.out, self.out), dtype=tdt, device="cuda")
        self.pipe = F.Pipeline(W.nv12_letterbox_chain(code, out=self.out, pad=cfg["pad"]))
        self.ins = [F.as_fkl(self.frames[i], F.FKL_LAYOUT_NV12) for i in range(n)]
        self.o = F.as_fkl(self.dst, F.FKL_LAYOUT_NCHW)
        dw, dh = metrics.letterbox_size(self.w, self.h, self.out, self.out)
        self.bytes = n * (metrics.nv12_tap_bytes(0, 0, self.w, self.h, dw, dh)
                          + metrics.out_bytes(1, self.out, self.out, self.el))
        self.sector_bytes = n * (metrics.nv12_tap_sector_bytes(0, 0, self.w, self.h, dw, dh, self.w, self.h)
                                 + metrics.planar_out_sector_bytes(1, self.out, self.out, self.el))
        self.oracle_spec = ("nv12", {"fmt": fmt, "seed": seed, "h": self.h, "w": self.w, "out": self.out},
                            self.bytes / n)
        self.name = (f"NV12 {n}x{self.w}x{self.h} -> BT.601 -> letterbox {self.out}x{self.out} pad 114 "
                     f"-> x1/255 -> planar {fmt}")
        self.traffic_key = f"nv12_letterbox_{fmt}_{n}"
        self.launches_per_step = (n + 255) // 256
        self.ws = None
        self.h2d_bytes = self.frames_host.nbytes
        self.d2h_bytes = self.dst.numel() * self.el

    def step(self, stream):
        self.F.fkl_execute_batch(self.pipe.handle, self.ins, None, self.o, stream=stream)

    def step_unfused(self, stream):
        if self.ws is None:
            nb = self.F.fkl_unfused_workspace_bytes(self.pipe.handle, self.ins, None, self.o)
            self.ws = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
            self.ws_bytes = nb
        self.F.fkl_execute_batch_unfused(self.pipe.handle, self.ins, None, self.o,
                                         self.ws.data_ptr(), self.ws_bytes, stream=stream)

    def step_per_op(self, stream, timed=False):
        if getattr(self, "ws_op", None) is None:
            nb = self.F.fkl_per_op_workspace_bytes(self.pipe.handle, self.ins, None, self.o)
            self.ws_op = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
            self.ws_op_bytes = nb
        return self.F.fkl_execute_batch_per_op(self.pipe.handle, self.ins, None, self.o, self.ws_op.data_ptr(),
                                               self.ws_op_bytes, stream=stream, timed=timed)

    def unfused_bytes(self):
        # decode (read NV12, write f32 RGB), letterbox (read taps, write f32),
        # x1/255 (read + write f32), split+cast (read f32, write out)
        rgb = self.h * self.w * 12
        img = self.out * self.out * 12
        nv12 = self.h * self.w * 3 // 2
        per = (nv12 + rgb) + (rgb + img) + (2 * img) + (img + self.out * self.out * 3 * self.el)
        return self.n * per

    def e2e_setup(self, chunk=32, depth=3):
        """Pinned host frames in, pinned host planes out, through the
        library's overlapped host executor (fkl_execute_batch_host)."""
        torch, F = self.torch, self.F
        self.host_in = torch.from_numpy(self.frames_host).pin_memory()
        self.host_out = torch.empty(self.dst.shape, dtype=self.dst.dtype).pin_memory()
        self.host_ins = [F.as_fkl(self.host_in[i], F.FKL_LAYOUT_NV12) for i in range(self.n)]
        self.host_o = F.as_fkl(self.host_out, F.FKL_LAYOUT_NCHW)
        self.executor = F.fkl_host_executor_create(self.pipe.handle, chunk, depth, self.h * 3 // 2 * self.w,
                                                   3 * self.out * self.out * self.el)
        self.e2e_launches = self.launches_per_step
        self.e2e_note = ("fkl_execute_batch_mapped: the fused kernel reads the pinned host frames and writes "
                         "the pinned host planes over the host link (no staging copies)")
        self.e2e_staged_note = f"fkl_execute_batch_host, chunks of {chunk} frames, {depth} device slots"

    def e2e_step(self, stream):
        self.F.fkl_execute_batch_mapped(self.pipe.handle, self.host_ins, None, self.host_o, stream=stream)

    def e2e_staged_step(self, stream):
        self.F.fkl_execute_batch_host(self.executor, self.host_ins, None, self.host_o, stream=stream)

    def link_copy(self, stream):
        """The step's host<->device bytes alone: H2D of the frames and D2H of
        the planes on two streams at once (the e2e ceiling of this link)."""
        torch = self.torch
        if not hasattr(self, "_s2"):
            self._s2 = torch.cuda.Stream()
        e = torch.cuda.Event()
        e.record(stream)
        self._s2.wait_event(e)
        with torch.cuda.stream(stream):
            self.frames.copy_(self.host_in, non_blocking=True)
        with torch.cuda.stream(self._s2):
            self.host_out.copy_(self.dst, non_blocking=True)
        stream.wait_event(self._s2.record_event())

    def oracle_sample(self, O, k):
        O.preprocess_nv12(self.frames_host[k % self.n], self.out, self.out, pad=114.0, mul=1 / 255)
        return self.bytes / self.n


class PackedBatch(Workload):
    """Crops of packed u8 frames -> resize -> BGR->RGB -> normalise -> planar."""

    def __init__(self, F, W, synth, metrics, torch, single: bool):
        self.F, self.torch = F, torch
        if single:
            cfg = W.SINGLE
            src = synth.packed_image(0, cfg["src_h"], cfg["src_w"])
            rois = np.array([cfg["roi"]], np.int32)
            n, ow, oh = 1, cfg["out_w"], cfg["out_h"]
            self.name = "1920x1080 u8 BGR, crop 640x480@(320,200) -> 224x224 -> RGB -> /255 -> norm -> planar f32"
        else:
            cfg = W.HF
            src = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
            rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
            n, ow, oh = cfg["n"], cfg["out_w"], cfg["out_h"]
            self.name = "50 crops of 3840x2160 u8 -> 128x64 -> RGB -> /255 -> norm -> planar f32 [50,3,64,128]"
        self.n, self.rois, self.src_host = n, rois, src
        self.src = torch.from_numpy(src).cuda()
        self.dst = torch.empty((n, 3, oh, ow), dtype=torch.float32, device="cuda")
        self.pipe = F.Pipeline(W.normalize_chain(ow, oh))
        self.ins = [F.as_fkl(self.src)] * n
        self.o = F.as_fkl(self.dst, F.FKL_LAYOUT_NCHW)
        self.bytes = sum(metrics.packed_tap_bytes(r[2], r[3], ow, oh) for r in rois) + \
            metrics.out_bytes(n, oh, ow, 4)
        pitch = src.shape[1] * 3
        self.sector_bytes = sum(metrics.packed_tap_sector_bytes(r[0], r[1], r[2], r[3], ow, oh, pitch)
                                for r in rois) + metrics.planar_out_sector_bytes(n, oh, ow, 4)
        self.oracle_spec = ("single" if single else "hf", {}, self.bytes / n)
        self.ow, self.oh = ow, oh
        self.launches_per_step = 1
        self.ws = None
        self.h2d_bytes = src.nbytes
        self.d2h_bytes = self.dst.numel() * 4
        # L2 is larger than this working set: flush between timed steps
        self.flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step(self, stream):
        self.F.fkl_execute_batch(self.pipe.handle, self.ins, self.rois, self.o, stream=stream)

    def step_unfused(self, stream):
        if self.ws is None:
            nb = self.F.fkl_unfused_workspace_bytes(self.pipe.handle, self.ins, self.rois, self.o)
            self.ws = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
            self.ws_bytes = nb
        self.F.fkl_execute_batch_unfused(self.pipe.handle, self.ins, self.rois, self.o,
                                         self.ws.data_ptr(), self.ws_bytes, stream=stream)

    def step_per_op(self, stream, timed=False):
        if getattr(self, "ws_op", None) is None:
            nb = self.F.fkl_per_op_workspace_bytes(self.pipe.handle, self.ins, self.rois, self.o)
            self.ws_op = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
            self.ws_op_bytes = nb
        return self.F.fkl_execute_batch_per_op(self.pipe.handle, self.ins, self.rois, self.o, self.ws_op.data_ptr(),
                                               self.ws_op_bytes, stream=stream, timed=timed)

    def between_steps(self):
        self.flush.fill_(1)

    def unfused_bytes(self):
        # resize writes a float32 image; swap, x1/255, -mean, /std each read
        # and write one; split reads one and writes the float32 planes
        img = self.oh * self.ow * 12
        taps = self.bytes - self.n * img
        return taps + self.n * 11 * img

    def e2e_setup(self):
        self.host_in = self.torch.from_numpy(self.src_host).pin_memory()
        self.host_out = self.torch.empty(self.dst.shape, dtype=self.dst.dtype).pin_memory()

    def e2e_step(self, stream):
        self.src.copy_(self.host_in, non_blocking=True)
        self.step(stream)
        self.host_out.copy_(self.dst, non_blocking=True)

    def oracle_sample(self, O, k):
        import paper_2508_07071_gb300.configs as W
        r = self.rois[k % self.n]
        O.preprocess_packed(self.src_host, r, self.ow, self.oh, swap=True, mul=1 / 255,
                            sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
        return self.bytes / self.n


class VChain(Workload):
    def __init__(self, F, W, synth, metrics, torch, L):
        self.F, self.torch = F, torch
        n = W.VCHAIN["n"]
        self.n, self.L = n, L
        self.x_host = synth.f32_uniform(2, n)
        self.x = torch.from_numpy(self.x_host).cuda()
        self.y = torch.empty_like(self.x)
        kinds, consts = synth.chain_constants(2, L)
        self.kinds, self.consts = kinds, consts
        self.pipe = F.Pipeline(W.vertical_chain(kinds, consts))
        self.i, self.o = F.as_fkl(self.x), F.as_fkl(self.y)
        self.bytes = 8 * n
        self.alu_ops = n * L  # one FP32 multiply or add per element and op (no contraction)
        self.sector_bytes = 8 * n
        self.oracle_spec = ("vchain", {"L": L}, 8 * (1 << 20))
        self.name = f"64M f32 uniform[-1,1], {L} alternating mul/add (FMA off), f32 out"
        self.traffic_key = f"vchain_f32_64M_L{L}"
        self.launches_per_step = max(1, (L + 4095) // 4096)
        self.h2d_bytes = 4 * n
        self.d2h_bytes = 4 * n

    def step(self, stream):
        self.F.fkl_execute(self.pipe.handle, self.i, self.o, stream=stream)

    def step_unfused(self, stream):
        self.F.fkl_execute_batch_unfused(self.pipe.handle, [self.i], None, self.o, 0, 0, stream=stream)

    def unfused_bytes(self):
        return 8 * self.n * max(1, self.L)

    def e2e_setup(self):
        self.host_in = self.torch.from_numpy(self.x_host).pin_memory()
        self.host_out = self.torch.empty_like(self.host_in).pin_memory()

    def e2e_step(self, stream):
        self.x.copy_(self.host_in, non_blocking=True)
        self.step(stream)
        self.host_out.copy_(self.y, non_blocking=True)

    def oracle_sample(self, O, k):
        m = 1 << 20
        O.vertical_chain_f32(self.x_host[(k * m) % self.n:][:m], self.kinds, self.consts)
        return 8 * m


def make_workload(args, F, W, synth, metrics, torch):
    if args.workload == "nv12":
        return NV12Letterbox(F, W, synth, metrics, torch, args.frames, args.out_dtype)
    if args.workload in ("single", "hf"):
        return PackedBatch(F, W, synth, metrics, torch, single=args.workload == "single")
    if args.workload == "vchain":
        return VChain(F, W, synth, metrics, torch, args.chain_len)
    raise SystemExit(f"unknown workload {args.workload}")


# ------------------------------------------------------------------ timing


def aggregate_ranks(dev_ms: float, bytes_per_rank: int, world: int):
    """Whole-job timing across ranks: the slowest rank's device time and the
    bytes all ranks processed (weak scaling: each rank runs its own batch)."""
    if world <= 1:
        return dev_ms, bytes_per_rank
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([bytes_per_rank], dtype=torch.float64, device=dev)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), int(b.item())


def time_steps(torch, fn, K, stream, between=None):
    """Device time of K calls, each bracketed by events on `stream`; an
    optional `between` (L2 flush) runs outside the bracketed regions."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in ev:
        if between:
            between()
        a.record(stream)
        fn(stream)
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def time_steps_queued(torch, fn, K, stream):
    """Device time of K back-to-back calls with warm caches: a bounded GPU
    spin (~25 ms) runs first so that the host queues all K calls before the
    GPU reaches them, and no call waits for the host to submit it."""
    with torch.cuda.stream(stream):
        torch.cuda._sleep(50_000_000)
    return time_steps(torch, fn, K, stream)


def measure_unfused(torch, wl, steps, stream, between, fused_ms, peak):
    """The unfused chain on the same GPU in both forms: one kernel per op over
    the whole batch (the paper's unfused chain, per-kernel GB/s from a timed
    call) and one kernel per op and image (the horizontal-fusion comparison),
    each also replayed as a captured CUDA graph."""
    out = {"traffic_ratio": round(wl.unfused_bytes() / wl.bytes, 2), "steps": steps}

    def timed(fn):
        fn(stream)
        torch.cuda.synchronize()
        ms = float(np.mean(time_steps(torch, fn, steps, stream, between)))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fn(stream)
        graph.replay()
        torch.cuda.synchronize()
        gms = float(np.mean(time_steps(torch, lambda st: graph.replay(), steps, stream, between)))
        return {"ms_per_step": round(ms, 4), "speedup": round(ms / fused_ms, 2),
                "cuda_graph_ms_per_step": round(gms, 4), "speedup_vs_cuda_graph": round(gms / fused_ms, 2)}

    if hasattr(wl, "step_per_op"):
        d = timed(wl.step_per_op)
        if between:
            between()
        rep = wl.step_per_op(stream, timed=True)  # one call with events around every kernel
        d["kernels"] = [{"name": name, "launches": int(k), "ms": round(ms, 4),
                         "GBps": round(b / (ms * 1e-3) / 1e9, 1) if ms > 0 else None,
                         "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4) if ms > 0 else None}
                        for name, k, b, ms in rep]
        d["launches_per_step"] = int(sum(k for _, k, _, _ in rep))
        d["form"] = "one kernel per op over the batch (fkl_execute_batch_per_op)"
        out["per_op"] = d
        d = timed(wl.step_unfused)
        d["form"] = "one kernel per op and image (fkl_execute_batch_unfused)"
        out["per_image"] = d
    else:  # tensor chains: the unfused form is already one kernel per op over the tensor
        d = timed(wl.step_unfused)
        d["form"] = "one kernel per op over the tensor (fkl_execute_batch_unfused)"
        d["launches_per_step"] = int(max(1, wl.L))
        d["kernel_GBps"] = round(wl.bytes / (d["ms_per_step"] / max(1, wl.L) * 1e-3) / 1e9, 1)
        d["kernel_frac"] = round(d["kernel_GBps"] / peak, 4)
        out["per_op"] = d
    return out


def roofline_of(torch, wl, kernel_ms, peak, peak_kind, clocks, local):
    achieved = wl.bytes / wl.launches_per_step / (kernel_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(getattr(wl, "traffic_key", "")),
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "frac_of_8tbs": round(achieved / 8000.0, 4)}
    if getattr(wl, "alu_ops", 0):
        # FP32 ALU roofline: SMs x 128 FP32 lanes x the maximum SM clock, one
        # op per lane and clock; the bound is whichever of the two takes longer
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_max_mhz") or 2070.0
        alu_peak = sms * 128 * mhz * 1e6 / 1e12
        alu_achieved = wl.alu_ops / wl.launches_per_step / (kernel_ms * 1e-3) / 1e12
        if wl.alu_ops / (alu_peak * 1e12) > wl.bytes / (peak * 1e9):
            roofline = {"bound": "alu", "achieved": round(alu_achieved, 2), "peak": round(alu_peak, 2),
                        "unit": "Top/s", "frac": round(alu_achieved / alu_peak, 4), "traffic": None,
                        "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (max SM clock)",
                        "hbm_frac": round(achieved / peak, 4)}
    return roofline


def autotune(F, wl, args, stream, between):
    ins = wl.ins if hasattr(wl, "ins") else [wl.i]
    rois = getattr(wl, "rois", None)
    best, us = F.fkl_pipeline_autotune(wl.pipe.handle, ins, rois, wl.o, stream=stream,
                                       reps=args.autotune_reps, before=between)
    return {"shape": list(best), "us_per_launch": round(us, 2),
            "candidates": len(F.fkl_pipeline_shapes(wl.pipe.handle))}


def secondary_configs(args, F, W, synth, metrics, torch, stream, peak, peak_kind, clocks, local):
    """The other workloads, measured in the same run: fused and unfused time
    and the roofline of the fused kernel (timed after the main workload)."""
    specs = [("single_image_224_f32", lambda: PackedBatch(F, W, synth, metrics, torch, single=True)),
             ("hf_50_crops_128x64_f32", lambda: PackedBatch(F, W, synth, metrics, torch, single=False)),
             ("vchain_64M_L10", lambda: VChain(F, W, synth, metrics, torch, 10)),
             ("vchain_64M_L1000", lambda: VChain(F, W, synth, metrics, torch, 1000)),
             ("nv12_256_letterbox_fp8", lambda: NV12Letterbox(F, W, synth, metrics, torch, args.frames, "e4m3")),
             ("nv12_256_letterbox_f16", lambda: NV12Letterbox(F, W, synth, metrics, torch, args.frames, "f16"))]
    out = {}
    for key, make in specs:
        wl = make()
        between = getattr(wl, "between_steps", None)
        with torch.cuda.stream(stream):
            tuned = autotune(F, wl, args, stream, between)
            for _ in range(3):
                wl.step(stream)
            torch.cuda.synchronize()
            k = args.secondary_steps
            times = time_steps(torch, wl.step, k, stream, between)
            ms = float(np.mean(times))
            kernel_ms = ms / wl.launches_per_step
            warm_ms = None
            if between is not None:
                warm_ms = float(np.mean(time_steps_queued(torch, wl.step, k, stream)))
            unf = measure_unfused(torch, wl, min(k, 3 if getattr(wl, "L", 0) >= 1000 else 5), stream, between,
                                  ms, peak)
        out[key] = {"workload": wl.name, "ms_per_step": round(ms, 5),
                    "best_ms": round(float(np.min(times)), 5), "median_ms": round(float(np.median(times)), 5),
                    "value": round(wl.bytes / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                    "algorithmic_bytes_per_step": int(wl.bytes), "steps": k,
                    "warm_ms_per_step": None if warm_ms is None else round(warm_ms, 5),
                    "roofline": roofline_of(torch, wl, kernel_ms, peak, peak_kind, clocks, local),
                    "unfused": unf, "autotune": tuned, "kernel": F.fkl_pipeline_kernel_name(wl.pipe.handle)}
        print(json.dumps({"secondary": key, "ms": out[key]["ms_per_step"],
                          "frac": out[key]["roofline"]["frac"]}), file=sys.stderr, flush=True)
        del wl
        torch.cuda.empty_cache()
    out["nv12_256_letterbox_fp8_dynamic_scale"] = dynamic_fp8(args, F, W, synth, torch, stream, peak)
    print(json.dumps({"secondary": "nv12_256_letterbox_fp8_dynamic_scale",
                      "ms": out["nv12_256_letterbox_fp8_dynamic_scale"]["ms_per_step"]}), file=sys.stderr, flush=True)
    if args.serve_requests > 0:
        _, _, pipe, fk = serve_setup(F, W, synth, torch, args.pool, args.serve_requests)
        sv = {"workload": f"Poisson requests at 1000 req/s, {args.serve_requests} requests of 1-64 pinned u8 BGR "
                          f"images 320-3840 x 240-2160 -> 224x224 RGB normalised planar f16"}
        for mode, mname in ((F.FKL_SERVE_PERSISTENT, "persistent"), (F.FKL_SERVE_UNFUSED, "unfused_per_request")):
            sv[mname] = serve_rate(F, synth, pipe, fk, 1000.0, mode, args.slots, args.arena_gb, args.ctas_per_sm)
        out["serving_1000rps"] = sv
        print(json.dumps({"secondary": "serving_1000rps", "images_per_s": sv["persistent"]["images_per_s"]}),
              file=sys.stderr, flush=True)
    return out


def dynamic_fp8(args, F, W, synth, torch, stream, peak):
    """ReduceDPP over the 256-frame NV12 batch (the statistics and the FP8
    scale in device memory), then the FP8 write with that scale: the dynamic
    per-tensor scaling step, CUDA events per step, no L2 flush (354 MB of
    frames are larger than L2)."""
    cfg = W.NV12
    n, h, w, side = args.frames, cfg["h"], cfg["w"], cfg["out"]
    frames = torch.from_numpy(synth.nv12_frames(3, n, h, w)).cuda()
    ins = [F.as_fkl(frames[i], F.FKL_LAYOUT_NV12) for i in range(n)]
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, out=side, pad=cfg["pad"]))
    dst = torch.empty((n, 3, side, side), dtype=torch.float8_e4m3fn, device="cuda")
    o = F.as_fkl(dst, F.FKL_LAYOUT_NCHW)
    stats = torch.zeros(32, dtype=torch.float32, device="cuda")
    sp = stats.data_ptr()
    with torch.cuda.stream(stream):
        F.fkl_pipeline_autotune(p.handle, ins, None, o, stream=stream, reps=args.autotune_reps)

        def red(st):
            F.fkl_reduce_batch(p.handle, ins, None, o, sp, stream=st)

        def step(st):
            red(st)
            F.fkl_execute_batch_scaled(p.handle, ins, None, o, sp + 11 * 4, stream=st)
        for _ in range(3):
            step(stream)
        torch.cuda.synchronize()
        k = args.secondary_steps
        step_times = time_steps(torch, step, k, stream)
        red_times = time_steps(torch, red, k, stream)
        ms, red_ms = float(np.mean(step_times)), float(np.mean(red_times))
    read_b, write_b = n * h * w * 3 // 2, n * 3 * side * side
    return {"workload": f"NV12 {n}x{w}x{h} -> letterbox {side}x{side} -> x1/255 -> FP8-E4M3 with the scale "
                        f"amax/448 from ReduceDPP (reduce pass, then the scaled write)",
            "ms_per_step": round(ms, 5), "value": round((read_b + write_b) / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
            "best_ms": round(float(np.min(step_times)), 5), "median_ms": round(float(np.median(step_times)), 5),
            "steps": k, "reduce_ms": round(red_ms, 5), "reduce_best_ms": round(float(np.min(red_times)), 5),
            "reduce_GBps": round(read_b / (red_ms * 1e-3) / 1e9, 1),
            "reduce_frac": round(read_b / (red_ms * 1e-3) / 1e9 / peak, 4),
            "scale": round(float(stats[10].item()), 9)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_07071_gb300 import fkl as F, metrics, synth, workloads as W

    wl = make_workload(args, F, W, synth, metrics, torch)
    stream = torch.cuda.Stream()
    between = getattr(wl, "between_steps", None)
    tuned = None
    peak, peak_kind = measured_peaks()
    with torch.cuda.stream(stream):
        if args.shape:
            F.fkl_pipeline_set_shape(wl.pipe.handle, [int(v) for v in args.shape.split(",")])
        elif not args.no_autotune:
            tuned = autotune(F, wl, args, stream, between)
        for _ in range(args.warmup):
            wl.step(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        sampler = metrics.ClockSampler(local)
        sampler.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        times = time_steps(torch, wl.step, args.steps, stream, between)
        wall = time.perf_counter() - t0
        sampler.stop()
        if world > 1:
            dist.barrier()
        dev_ms, total_bytes = aggregate_ranks(float(np.sum(times)), wl.bytes, world)
        ms_per_step = dev_ms / args.steps
        kernel_ms = float(np.mean(times)) / wl.launches_per_step
        warm_ms = None
        if between is not None:  # L2-sized workloads: also without the flush (inputs stay in L2)
            warm_ms = float(np.mean(time_steps_queued(torch, wl.step, min(args.steps, 100), stream)))

        # the same step captured once in a CUDA graph and replayed
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            wl.step(stream)
        graph.replay()
        torch.cuda.synchronize()
        graph_ms = float(np.mean(time_steps(torch, lambda st: graph.replay(), min(args.steps, 100), stream, between)))

        # unfused chain on the same GPU (a few steps)
        ku = min(args.steps, args.unfused_steps)
        unfused = measure_unfused(torch, wl, ku, stream, between, ms_per_step, peak) if ku > 0 else None

        # end to end through the public call with host buffers
        ke = min(args.steps, args.e2e_steps)
        e2e_ms = link_ms = None
        e2e_paths = {}
        if ke > 0:
            wl.e2e_setup()
            # each public host-buffer call the workload offers, staged copies first
            calls = [(getattr(wl, "e2e_staged_note", None), getattr(wl, "e2e_staged_step", None)),
                     (getattr(wl, "e2e_note", "torch pinned copies + fkl_execute_batch on one stream"), wl.e2e_step)]
            for note, fn in calls:
                if fn is None:
                    continue
                for _ in range(2):
                    fn(stream)
                torch.cuda.synchronize()
                e2e_paths[note] = float(np.mean(time_steps(torch, fn, ke, stream)))
            e2e_note, e2e_ms = min(e2e_paths.items(), key=lambda kv: kv[1])
            if hasattr(wl, "link_copy"):
                wl.link_copy(stream)
                link_ms = float(np.mean(time_steps(torch, wl.link_copy, ke, stream)))

    value = total_bytes / (ms_per_step * 1e-3) / 1e9
    clocks = sampler.summary()
    roofline = roofline_of(torch, wl, kernel_ms, peak, peak_kind, clocks, local)
    secondary = None
    if rank == 0 and args.secondary and args.workload == "nv12":
        main_name = wl.name
        launches_main = int(args.steps * wl.launches_per_step)
        wl_keep = wl
        secondary = secondary_configs(args, F, W, synth, metrics, torch, stream, peak, peak_kind, clocks, local)
        wl = wl_keep
        assert wl.name == main_name and launches_main == int(args.steps * wl.launches_per_step)
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded), resident in HBM",
        "config": {"workload": wl.name, "algorithmic_bytes_per_step": int(wl.bytes),
                   "best_ms": round(float(np.min(times)), 5), "median_ms": round(float(np.median(times)), 5),
                   "cuda_graph_ms_per_step": round(graph_ms, 5),
                   "sector_bytes_per_step": int(getattr(wl, "sector_bytes", wl.bytes)),
                   "warm_ms_per_step": None if warm_ms is None else round(warm_ms, 5),
                   "warm_value": None if warm_ms is None else round(wl.bytes / (warm_ms * 1e-3) / 1e9, 1),
                   "l2": getattr(wl, "l2_note", "inputs+outputs larger than L2 (no flush)" if between is None
                                 else "L2 flushed (256 MiB write) between timed steps, outside the events"),
                   "parallelism": f"replicas x{world}", "launch_shape": list(F.fkl_pipeline_get_shape(wl.pipe.handle))
                   if hasattr(wl, "pipe") else None,
                   "kernel": F.fkl_pipeline_kernel_name(wl.pipe.handle), "autotune": tuned},
        "unfused": unfused,
        "roofline": roofline,
        "e2e": None if e2e_ms is None else {
            "value": round(wl.bytes * world / (e2e_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
            "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(wl.h2d_bytes),
            "d2h_bytes_per_step": int(wl.d2h_bytes), "steps": ke,
            "path": e2e_note,
            "link_copy_ms": None if link_ms is None else round(link_ms, 4),
            "frac_of_link": None if link_ms is None else round(link_ms / e2e_ms, 3),
            "ms_per_step_by_path": {k: round(v, 4) for k, v in e2e_paths.items()}},
        "gpu_launches": int(args.steps * wl.launches_per_step),
        "clocks": clocks,
        "wall_s_timed": round(wall, 4),
        "configs": secondary,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args)
        if not args.no_cpu_parallel:
            line["cpu_baseline_parallel"] = cpu_baseline_parallel(wl, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(wl, args, budget_s=None):
    import oracle as O
    budget = budget_s if budget_s is not None else args.cpu_seconds
    t0 = time.perf_counter()
    b = wl.oracle_sample(O, 0)
    one = time.perf_counter() - t0
    k = int(max(1, min(1024, budget / max(one, 1e-6))))
    t0 = time.perf_counter()
    nbytes = 0
    for i in range(k):
        nbytes += wl.oracle_sample(O, i)
    dt = time.perf_counter() - t0
    return {"value": round(nbytes / dt / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} unit(s) of the workload (images/frames, or 1M-element slices), "
                      f"{dt:.1f} s, float64 numpy, single thread"}


_WORKER = {}


def _oracle_worker_init(kind, params):
    """Builds one worker's inputs (the workload's seeded generators) and the
    oracle call of one unit; runs in a spawned process."""
    import oracle as O
    from paper_2508_07071_gb300 import configs as W, synth  # no CUDA library in the workers
    if kind == "nv12":
        frames = synth.nv12_frames(params["seed"], 4, params["h"], params["w"])
        _WORKER["f"] = lambda k: O.preprocess_nv12(frames[k % 4], params["out"], params["out"], pad=114.0,
                                                   mul=1 / 255)
    elif kind in ("single", "hf"):
        if kind == "single":
            cfg = W.SINGLE
            src = synth.packed_image(0, cfg["src_h"], cfg["src_w"])
            rois = np.array([cfg["roi"]], np.int32)
        else:
            cfg = W.HF
            src = synth.packed_image(1, cfg["src_h"], cfg["src_w"])
            rois = synth.crop_rois(1, cfg["n"], cfg["src_w"], cfg["src_h"], cfg["w_range"], cfg["h_range"])
        _WORKER["f"] = lambda k: O.preprocess_packed(src, rois[k % len(rois)], cfg["out_w"], cfg["out_h"],
                                                     swap=True, mul=1 / 255, sub=W.IMAGENET_MEAN,
                                                     div=W.IMAGENET_STD)
    else:
        x = synth.f32_uniform(2, 4 << 20)
        kinds, consts = synth.chain_constants(2, params["L"])
        m = 1 << 20
        _WORKER["f"] = lambda k: O.vertical_chain_f32(x[(k % 4) * m:][:m], kinds, consts)


def _oracle_unit(k):
    _WORKER["f"](k)
    return k


def cpu_baseline_parallel(wl, args):
    """The oracle over all allowed host cores: one spawned worker process per
    core, units (frames, crops or 1M-element slices) handed out one at a time;
    the pool is started and warmed before the timed map."""
    import multiprocessing as mp
    kind, params, unit_bytes = wl.oracle_spec
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(kind, params)) as pool:
        pool.map(_oracle_unit, range(cores), chunksize=1)  # every worker initialised and warm
        t0 = time.perf_counter()
        pool.map(_oracle_unit, range(cores), chunksize=1)
        one_round = time.perf_counter() - t0  # wall time of `cores` units in parallel
        k = int(max(cores, min(4096, cores * args.cpu_seconds / max(one_round, 1e-6))))
        t0 = time.perf_counter()
        pool.map(_oracle_unit, range(k), chunksize=1)
        dt = time.perf_counter() - t0
    return {"value": round(k * unit_bytes / dt / 1e9, 6), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{k} unit(s) of the workload over {cores} spawned worker processes, {dt:.1f} s, "
                      f"float64 numpy (one thread per process)"}


def serve_setup(F, W, synth, torch, n_pool, n_requests):
    """The serving workload: a pool of pinned host images of 320-3840 x
    240-2160 and requests of 1-64 of them (seeded)."""
    rng = np.random.default_rng(4)
    pool = []
    for k in range(n_pool):
        w, h = int(rng.integers(320, 3841)), int(rng.integers(240, 2161))
        pool.append(torch.from_numpy(synth.packed_image(1000 + k, h, w)).pin_memory())
    reqs = [list(rng.integers(0, len(pool), int(rng.integers(1, 65)))) for _ in range(n_requests)]
    pipe = F.Pipeline(W.normalize_chain(224, 224, out_dtype=F.FKL_F16))
    fk = [[F.as_fkl(pool[i]) for i in r] for r in reqs]
    return pool, reqs, pipe, fk


def serve_rate(F, synth, pipe, fk, rate, mode, slots, arena_gb, ctas_per_sm):
    """Requests submitted at seeded Poisson arrival times against one server;
    latency = completion minus scheduled arrival."""
    arrivals = synth.poisson_arrivals(4, rate, len(fk))
    srv = F.fkl_server_create(pipe.handle, mode, max_inflight=slots, arena_bytes=arena_gb << 30,
                              ctas_per_sm=ctas_per_sm)
    try:
        # warm-up: one request through the server
        rid = F.fkl_server_submit(srv, fk[0])
        F.fkl_server_wait(srv, rid, 60000)
        F.fkl_server_release(srv, rid)
        t0 = time.monotonic() + 0.01
        live, lat, q, h2d, nimg = {}, [], [], [], 0
        i = 0
        t_last = t0
        while i < len(fk) or live:
            now = time.monotonic()
            while i < len(fk) and t0 + arrivals[i] <= now:
                live[F.fkl_server_submit(srv, fk[i])] = t0 + arrivals[i]
                i += 1
            for rid in list(live):
                done, _ = F.fkl_server_poll(srv, rid)
                if done:
                    info = F.fkl_server_request_info(srv, rid)
                    lat.append(info.t_done - live.pop(rid))
                    q.append(info.t_admit - info.t_submit)
                    h2d.append(info.t_ready - info.t_admit)
                    nimg += info.n_images
                    t_last = max(t_last, info.t_done)
                    F.fkl_server_release(srv, rid)
            time.sleep(0.0001)
        st = F.fkl_server_get_stats(srv)
    finally:
        F.fkl_server_destroy(srv)
    lat_ms = np.array(lat) * 1e3
    return {"rate_req_s": rate, "requests": len(fk), "images": nimg,
            "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
            "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
            "queue_p50_ms": round(float(np.median(q)) * 1e3, 3),
            "h2d_p50_ms": round(float(np.median(h2d)) * 1e3, 3),
            "images_per_s": round(nimg / (t_last - t0), 1),
            "kernel_launches": int(st.kernel_launches),
            "arena_peak_gb": round(st.arena_peak_bytes / 2**30, 3)}


def run_serve(args):
    """Serving loop: Poisson arrivals of requests of 1-64 images of mixed
    sizes (320-3840 x 240-2160) through fkl_server_*, full-frame resize to
    224x224 -> RGB -> normalise -> planar FP16. Latency = completion minus
    scheduled arrival (copies to the device included)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_07071_gb300 import fkl as F, synth, workloads as W

    _, _, pipe, fk = serve_setup(F, W, synth, torch, args.pool, args.requests)
    results = []
    for rate in [float(x) for x in args.rates.split(",")]:
        for mode, mname in ((F.FKL_SERVE_PERSISTENT, "persistent"), (F.FKL_SERVE_UNFUSED, "unfused_per_request")):
            r = serve_rate(F, synth, pipe, fk, rate, mode, args.slots, args.arena_gb, args.ctas_per_sm)
            results.append({"rate_req_s": rate, "mode": mname, **{k: v for k, v in r.items() if k != "rate_req_s"}})
            print(json.dumps(results[-1]), flush=True)
    print(json.dumps({"metric": "serving latency and throughput", "workload": "Poisson requests, 1-64 u8 BGR "
                      "images 320-3840 x 240-2160 -> 224x224 RGB normalised planar f16", "results": results}),
          flush=True)


def run_sweeps(args):
    """The paper's parameter sweeps on GB300, fused vs unfused per point:
    Exp 4 (§VI-D) VF+HF: 50 images of 60x120 u8, 1..10,000 Mul+Add pairs;
    Exp 7 (§VI-G) data size: 100 .. 16,654,030 floats, 100 Mul+Add pairs;
    Exp 5 (§VI-E) instructions per op: 500 Mul/Add instructions on
    3840*2160*8 floats split into N kernels of M = 500/N ops each;
    Exp 6 (§VI-F) host time of one call; Exp 9 (§VI-I) data types: 50
    matrices of 60x120, Read -> Cast -> Mul -> Sub -> Div -> Write for every
    (input, output) type pair; ReduceDPP (§IV-C) with dynamic FP8 scaling
    on the 256-frame NV12 letterbox batch. `--only exp4,exp9` runs a
    subset."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_07071_gb300 import fkl as F, synth, workloads as W

    stream = torch.cuda.Stream()
    res = {"exp4_vf_hf": [], "exp7_data_size": [], "exp5_ops_per_kernel": []}
    only = set(filter(None, args.only.split(",")))

    def want(name):
        return not only or name in only

    def t(fn, k):
        # device time of k queued calls: the small sizes are launch-bound,
        # and a call that waits for the host would time the host
        fn(stream)
        torch.cuda.synchronize()
        return float(np.median(time_steps_queued(torch, fn, k, stream)))

    with torch.cuda.stream(stream):
        # Exp 4: VF + HF, u8 input, batch 50 x 60 x 120 (one launch for the batch)
        n = 50 * 60 * 120
        pairs_list = [1, 10, 100, 1000, 5000, 10000] if want("exp4") else []
        x = torch.from_numpy(synth.packed_image(40, 1, n, 1).reshape(-1)).cuda()
        y = torch.empty(n, device="cuda")
        for pairs in pairs_list:
            kinds, consts = synth.chain_constants(40, 2 * pairs)
            p = F.Pipeline(W.vertical_chain(kinds, consts, u8_input=True))
            F.fkl_pipeline_autotune(p.handle, [F.as_fkl(x)], None, F.as_fkl(y), stream=stream, reps=5)
            fused = t(lambda st: F.fkl_execute(p.handle, F.as_fkl(x), F.as_fkl(y), stream=st), 10)
            k_unf = 3 if pairs <= 1000 else 1
            unf = t(lambda st: F.fkl_execute_batch_unfused(p.handle, [F.as_fkl(x)], None, F.as_fkl(y), 0, 0,
                                                           stream=st), k_unf)
            ops = n * 2 * pairs
            res["exp4_vf_hf"].append({"pairs": pairs, "fused_ms": round(fused, 4), "unfused_ms": round(unf, 3),
                                      "speedup": round(unf / fused, 1),
                                      "fused_Gops_per_s": round(ops / fused / 1e6, 1)})
            print(json.dumps({"exp4": res["exp4_vf_hf"][-1]}), flush=True)
        # Exp 7: data size, 100 Mul+Add pairs, float32
        kinds, consts = synth.chain_constants(41, 200)
        p = F.Pipeline(W.vertical_chain(kinds, consts))
        for n in [100, 10_000, 282_370, 1_000_000, 9_032_740, 16_654_030] if want("exp7") else []:
            x = torch.from_numpy(synth.f32_uniform(41, n)).cuda()
            y = torch.empty_like(x)
            F.fkl_pipeline_autotune(p.handle, [F.as_fkl(x)], None, F.as_fkl(y), stream=stream, reps=5)
            fused = t(lambda st: F.fkl_execute(p.handle, F.as_fkl(x), F.as_fkl(y), stream=st), 20)
            unf = t(lambda st: F.fkl_execute_batch_unfused(p.handle, [F.as_fkl(x)], None, F.as_fkl(y), 0, 0,
                                                           stream=st), 5)
            res["exp7_data_size"].append({"elements": n, "fused_ms": round(fused, 4), "unfused_ms": round(unf, 3),
                                          "speedup": round(unf / fused, 1),
                                          "fused_GBps": round(8 * n / fused / 1e6, 1)})
            print(json.dumps({"exp7": res["exp7_data_size"][-1]}), flush=True)
        # Exp 5: 500 instructions split into N kernels of M ops (M * N = 500)
        if want("exp5"):
            n = 3840 * 2160 * 8
            x = torch.from_numpy(synth.f32_uniform(42, n)).cuda()
            y = torch.empty_like(x)
            kinds, consts = synth.chain_constants(42, 500)
            full = F.Pipeline(W.vertical_chain(kinds, consts))
            F.fkl_pipeline_autotune(full.handle, [F.as_fkl(x)], None, F.as_fkl(y), stream=stream, reps=3)
            fused = t(lambda st: F.fkl_execute(full.handle, F.as_fkl(x), F.as_fkl(y), stream=st), 5)
            for m in [1, 5, 25, 100, 250, 500]:
                parts = [F.Pipeline(W.vertical_chain(kinds[i:i + m], consts[i:i + m])) for i in range(0, 500, m)]
                for q in parts:
                    F.fkl_pipeline_set_shape(q.handle, F.fkl_pipeline_get_shape(full.handle))

                def chain(st):
                    F.fkl_execute(parts[0].handle, F.as_fkl(x), F.as_fkl(y), stream=st)
                    for q in parts[1:]:
                        F.fkl_execute(q.handle, F.as_fkl(y), F.as_fkl(y), stream=st)
                split = t(chain, 3)
                res["exp5_ops_per_kernel"].append({"ops_per_kernel": m, "kernels": len(parts),
                                                   "split_ms": round(split, 3), "fused_500_ms": round(fused, 3),
                                                   "speedup": round(split / fused, 2)})
                print(json.dumps({"exp5": res["exp5_ops_per_kernel"][-1]}), flush=True)
        # Exp 6: host time of one call, fused vs one launch per op and image:
        if want("exp6"):
            # Batch(Crop -> Resize 64x128 -> BGR->RGB -> Mul -> Sub -> Div -> Split)
            import ctypes
            frame = torch.from_numpy(synth.packed_image(43, 2160, 3840)).cuda()
            p = F.Pipeline(W.normalize_chain(64, 128))
            res["exp6_cpu_time"] = []
            for n in [2, 10, 50, 100, 152]:
                rois = np.ascontiguousarray(synth.crop_rois(43, n, 3840, 2160, (32, 640), (32, 480)))
                out = torch.empty((n, 3, 128, 64), device="cuda")
                arr = (F.fkl_tensor * n)(*([F.as_fkl(frame)] * n))
                rp = rois.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
                o = F.as_fkl(out, F.FKL_LAYOUT_NCHW)
                nb = F.fkl_unfused_workspace_bytes(p.handle, list(arr), rois, o)
                ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
                sh = stream.cuda_stream

                def host_us(call, reps):
                    call()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(reps):
                        call()
                    dt = (time.perf_counter() - t0) / reps
                    torch.cuda.synchronize()
                    return dt * 1e6
                fused = host_us(lambda: F._lib.fkl_execute_batch(p.handle, n, arr, rp, ctypes.byref(o), sh), 200)
                unf = host_us(lambda: F._lib.fkl_execute_batch_unfused(p.handle, n, arr, rp, ctypes.byref(o),
                                                                       ws.data_ptr(), nb, sh), 20)
                res["exp6_cpu_time"].append({"batch": n, "fused_host_us": round(fused, 2),
                                             "unfused_host_us": round(unf, 1), "launches_unfused": 6 * n,
                                             "speedup": round(unf / fused, 1)})
                print(json.dumps({"exp6": res["exp6_cpu_time"][-1]}), flush=True)
        # Exp 9: data types, 50 x 60x120, Read -> Cast -> Mul -> Sub -> Div -> Write.
        # "eager": one call per step from pre-marshalled arguments, queued
        # like every sweep call (device time of separately submitted
        # launches); "graph": the same calls captured once in a CUDA graph
        # and replayed.
        import ctypes
        cfg = W.DTYPES
        res["exp9_data_types"] = []
        L = cfg["rows"] * cfg["cols"]
        code = {"u8": F.FKL_U8, "u16": F.FKL_U16, "f32": F.FKL_F32, "f64": F.FKL_F64}
        size = {"u8": 1, "u16": 2, "f32": 4, "f64": 8}
        nt = cfg["n"]
        for src in cfg["ins"] if want("exp9") else []:
            xs = [torch.from_numpy(synth.linear_values(100 + i, L, src)).cuda() for i in range(nt)]
            arr = (F.fkl_tensor * nt)(*[F.as_fkl(x) for x in xs])
            for dst in cfg["outs"]:
                y = torch.empty(nt * L, dtype=torch.float32 if dst == "f32" else torch.float64, device="cuda")
                o = F.as_fkl(y)
                p = F.Pipeline(W.typed_chain(code[src], code[dst], cfg["mul"], cfg["sub"], cfg["div"]))
                F.fkl_pipeline_autotune(p.handle, list(arr), None, o, stream=stream, reps=7)
                h = p.handle

                def fused_call(st):
                    F._check(F._lib.fkl_execute_batch(h, nt, arr, None, ctypes.byref(o), st.cuda_stream))

                def unfused_call(st):
                    F._check(F._lib.fkl_execute_batch_unfused(h, nt, arr, None, ctypes.byref(o), None, 0,
                                                              st.cuda_stream))
                row = {"in": src, "out": dst}
                for name, call, k in (("fused", fused_call, 50), ("unfused", unfused_call, 10)):
                    row[name + "_eager_us"] = round(1000 * t(call, k), 2)
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=stream):
                        call(stream)
                    g.replay()
                    row[name + "_graph_us"] = round(1000 * t(lambda st: g.replay(), k), 2)
                row["speedup_eager"] = round(row["unfused_eager_us"] / row["fused_eager_us"], 1)
                row["speedup_graph"] = round(row["unfused_graph_us"] / row["fused_graph_us"], 1)
                row["launches_unfused"] = 4 * nt
                row["fused_graph_GBps"] = round(nt * L * (size[src] + size[dst]) / row["fused_graph_us"] / 1e3, 1)
                row["shape"] = list(F.fkl_pipeline_get_shape(h))
                res["exp9_data_types"].append(row)
                print(json.dumps({"exp9": row}), flush=True)
        # ReduceDPP (§IV-C) and dynamic FP8 scaling on the 256-frame NV12
        # letterbox batch: the reduction pass alone (it reads the frames and
        # writes no image), the FP8 write with the scale that pass leaves in
        # device memory, the two as one step, and the static-scale write.
        if want("reduce"):
            cfgn = W.NV12
            n, h, w, side = cfgn["n"], cfgn["h"], cfgn["w"], cfgn["out"]
            frames = torch.from_numpy(synth.nv12_frames(3, n, h, w)).cuda()
            ins = [F.as_fkl(frames[i], F.FKL_LAYOUT_NV12) for i in range(n)]
            p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_E4M3, out=side, pad=cfgn["pad"]))
            dst = torch.empty((n, 3, side, side), dtype=torch.float8_e4m3fn, device="cuda")
            o = F.as_fkl(dst, F.FKL_LAYOUT_NCHW)
            F.fkl_pipeline_autotune(p.handle, ins, None, o, stream=stream, reps=3)
            stats = torch.zeros(32, dtype=torch.float32, device="cuda")
            sp = stats.data_ptr()

            def red(st):
                F.fkl_reduce_batch(p.handle, ins, None, o, sp, stream=st)

            def scaled(st):
                F.fkl_execute_batch_scaled(p.handle, ins, None, o, sp + 11 * 4, stream=st)

            def step(st):
                red(st)
                scaled(st)

            def static(st):
                F.fkl_execute_batch(p.handle, ins, None, o, stream=st)
            read_b = n * h * w * 3 // 2
            write_b = n * 3 * side * side
            peak, peak_kind = measured_peaks()
            ms = {name: t(fn, 20) for name, fn in (("reduce", red), ("scaled_write", scaled),
                                                    ("dynamic_step", step), ("static_write", static))}
            row = {k + "_us": round(1000 * v, 1) for k, v in ms.items()}
            row["reduce_GBps"] = round(read_b / ms["reduce"] / 1e6, 1)
            row["reduce_frac"] = round(read_b / ms["reduce"] / 1e6 / peak, 3)
            row["dynamic_step_GBps"] = round((read_b + write_b) / ms["dynamic_step"] / 1e6, 1)
            row["static_write_GBps"] = round((read_b + write_b) / ms["static_write"] / 1e6, 1)
            row["peak_GBps"] = peak
            row["peak"] = f"{peak_kind} copy bandwidth"
            row["stats"] = [round(float(v), 6) for v in stats[:12].tolist()]
            res["reduce_dynamic_fp8"] = row
            print(json.dumps({"reduce": row}), flush=True)
    print(json.dumps({"metric": "paper sweeps (Exp 4, 5, 6, 7, 9) and ReduceDPP on GB300", "results": res}),
          flush=True)


def run_reference(args):
    """The reference arm: the CPU oracle, unchanged, on all allowed host cores
    (one spawned worker process per core, one frame per core per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_2508_07071_gb300 import configs as W, metrics  # the oracle arm needs no CUDA library

    cfg = W.NV12
    if args.workload != "nv12":
        raise SystemExit("--impl reference supports --workload nv12")
    dw, dh = metrics.letterbox_size(cfg["w"], cfg["h"], cfg["out"], cfg["out"])
    el = {"bf16": 2, "f16": 2, "e4m3": 1, "f32": 4}[args.out_dtype]
    per = metrics.nv12_tap_bytes(0, 0, cfg["w"], cfg["h"], dw, dh) + metrics.out_bytes(1, 640, 640, el)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    params = {"fmt": args.out_dtype, "seed": 3, "h": cfg["h"], "w": cfg["w"], "out": cfg["out"]}
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=("nv12", params)) as pool:
        for k in range(args.warmup):
            pool.map(_oracle_unit, range(k * cores, (k + 1) * cores), chunksize=1)
        t0 = time.perf_counter()
        for k in range(args.steps):
            pool.map(_oracle_unit, range(k * cores, (k + 1) * cores), chunksize=1)
        dt = time.perf_counter() - t0
    val = args.steps * cores * per / dt / 1e9
    name = (f"NV12 1280x720 -> letterbox 640 -> planar {args.out_dtype} ({cores} frames per step, one per "
            f"host core)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "config": {"workload": name},
        "cpu_baseline": {"value": round(val, 6), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} 1280x720 frames per step over {cores} spawned worker processes, "
                                   f"float64 numpy (one thread per process)"},
        "e2e": {"value": round(val, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nv12", choices=["nv12", "single", "hf", "vchain", "serve", "sweeps"])
    ap.add_argument("--rates", default="200,500,1000,2000", help="serve: request rates (req/s)")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per rate")
    ap.add_argument("--pool", type=int, default=48, help="serve: distinct host images")
    ap.add_argument("--slots", type=int, default=64, help="serve: request slots")
    ap.add_argument("--arena-gb", type=int, default=16, help="serve: device arena (GiB)")
    ap.add_argument("--ctas-per-sm", type=int, default=1, help="serve: persistent kernel CTAs per SM")
    ap.add_argument("--out-dtype", default="bf16", choices=["bf16", "f16", "e4m3", "f32"])
    ap.add_argument("--frames", type=int, default=256)
    ap.add_argument("--chain-len", type=int, default=10)
    ap.add_argument("--unfused-steps", type=int, default=5)
    ap.add_argument("--secondary", action=argparse.BooleanOptionalAction, default=True,
                    help="nv12: also measure the other workloads (single image, crop batch, vertical chain "
                         "L=10/1000, FP8 and f16 outputs) into the line's `configs`")
    ap.add_argument("--secondary-steps", type=int, default=100)
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="nv12 default run: requests of the serving measurement in `configs` (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-parallel", action="store_true",
                    help="skip timing the oracle over all host cores (spawned worker processes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune-reps", type=int, default=7)
    ap.add_argument("--shape", default="", help="vec,tx,ty,ry launch shape (skips the autotuner)")
    ap.add_argument("--only", default="",
                    help="sweeps: comma-separated subset of exp4,exp5,exp6,exp7,exp9,reduce")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "sweeps":
        run_sweeps(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
