"""Host-side pieces of bench.py that run without a GPU."""
import os
import sys
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("kind,params", [("single", {}), ("vchain", {"L": 10})])
def test_parallel_oracle_baseline_runs_in_spawned_workers(kind, params):
    wl = types.SimpleNamespace(oracle_spec=(kind, params, 1000.0))
    args = types.SimpleNamespace(cpu_seconds=0.2)
    r = bench.cpu_baseline_parallel(wl, args)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    assert r["cores"] == cores and r["kind"] == "oracle" and r["value"] > 0
    assert "spawned worker processes" in r["sample"]


def test_sector_footprints():
    from paper_2508_07071_gb300 import metrics as M
    # a 2x downscale of 64 columns touches every byte of 192 contiguous bytes: 6 sectors per row
    assert M.packed_tap_sector_bytes(0, 0, 64, 2, 32, 1, 4096) == 2 * 6 * 32
    # a 4x downscale reads the middle pair of every 4 columns: 2 of 4 pixels, yet every sector
    assert M.packed_tap_bytes(64, 1, 16, 1) == 32 * 3 and M.packed_tap_sector_bytes(0, 0, 64, 1, 16, 1, 4096) == 6 * 32
    # NV12 exact 2x of aligned rows: sectors equal bytes
    assert M.nv12_tap_sector_bytes(0, 0, 1280, 720, 640, 360, 1280, 720) == M.nv12_tap_bytes(0, 0, 1280, 720, 640, 360)
    # planes of 12-byte rows share sectors across rows: counted once
    assert M.planar_out_sector_bytes(1, 8, 3, 4) == 3 * 8 * 12


def test_reference_arm_prints_the_contract_line():
    """The oracle arm runs without the CUDA library: the binding module is
    made unimportable in the parent before bench.py starts."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    run = ("import runpy, sys; sys.modules['paper_2508_07071_gb300.fkl'] = None; "
           "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '2', '--warmup', '3']; "
           "runpy.run_path('bench.py', run_name='__main__')")
    r = subprocess.run([sys.executable, "-c", run], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "GB/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_workload_constants_live_in_the_library_free_module():
    """configs.py holds the shapes without touching the CUDA binding, and
    workloads.py re-exports the very same objects."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; import paper_2508_07071_gb300.configs as C; "
            "assert 'paper_2508_07071_gb300.fkl' not in sys.modules; print(C.NV12['n'])")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "256", r.stderr[-1000:]
    from paper_2508_07071_gb300 import configs as C, workloads as W
    for name in ("IMAGENET_MEAN", "IMAGENET_STD", "INV255", "E4M3_SCALE", "SINGLE", "HF", "VCHAIN", "NV12",
                 "SERVE", "DTYPES"):
        assert getattr(W, name) is getattr(C, name), name
