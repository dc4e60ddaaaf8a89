"""Per-launch DRAM traffic of a kernel from an ncu launch list.

Reads the CSV that `ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,
dram__bytes_write.sum --csv --log-file <f> <cmd>` writes, averages the
launches whose kernel name matches a pattern, and records the result under a
key in profiles/traffic.json together with the list and hash of the sources
the kernel is compiled from and of the build flags (bench.py reports the
figure only while that hash still matches).

    python -m paper_2508_07071_gb300.ncu_traffic --csv launches.csv \\
        --key nv12_letterbox_bf16_256 --kernel transform2d --unit k_nv12_bf16.cu \\
        [--header fkl/reduce.cuh] --command "<ncu command>"
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def source_hash(files: list[str] | None = None) -> str:
    """Hash of the CUDA sources a kernel is compiled from (paths relative to
    csrc/; all of them when `files` is None) and of the build flags (they
    change the kernels as much as sources do)."""
    h = hashlib.sha256()
    base = os.path.join(PKG, "csrc")
    if files is None:
        files = sorted(os.path.relpath(os.path.join(d, f), base)
                       for d, _, fs in os.walk(base) for f in fs if f.endswith((".cu", ".cuh", ".h")))
    for rel in sorted(files):
        h.update(rel.encode())
        with open(os.path.join(base, rel), "rb") as fh:
            h.update(fh.read())
    from . import build
    h.update(" ".join(build.ARCH + build.NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


# Every header the device code of the fused image-chain kernels comes from
# (core.cuh also fixes the parameter-table capacity, a template argument of
# the kernels). A traffic entry hashes these plus its translation unit;
# host-only sources (registry.h, api.cu, the other families) are not part of it.
DEVICE_HEADERS = ["fkl/core.cuh", "fkl/ops.cuh", "fkl/dpp.cuh", "fkl/staged.cuh", "fkl/tiles.cuh", "float_family.cuh"]


def entry_hash(entry: dict) -> str:
    """Hash over the sources an entry names (all sources for old entries)."""
    return source_hash(entry.get("sources"))


def parse_launches(path: str, kernel: str) -> list[dict]:
    """{metric name: value} per launch ID of the kernels matching `kernel`."""
    with open(path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    launches: dict[str, dict] = {}
    pat = re.compile(kernel)
    for row in csv.DictReader(lines):
        if not pat.search(row["Kernel Name"]):
            continue
        value = float(row["Metric Value"].replace(",", ""))
        launches.setdefault(row["ID"], {})[row["Metric Name"]] = value
    return [launches[k] for k in sorted(launches, key=int)]


def summarise(launches: list[dict]) -> dict:
    if not launches:
        raise ValueError("no launch of the kernel in the CSV")
    n = len(launches)
    rd = sum(l["dram__bytes_read.sum"] for l in launches) / n
    wr = sum(l["dram__bytes_write.sum"] for l in launches) / n
    t = sum(l["gpu__time_duration.sum"] for l in launches) / n
    return {"dram_bytes_per_launch": int(round(rd + wr)), "dram_read_bytes": int(round(rd)),
            "dram_write_bytes": int(round(wr)), "launches": n,
            "mean_time_us_cold_serialised": round(t / 1000.0, 2)}


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--csv", required=True)
    ap.add_argument("--key", required=True)
    ap.add_argument("--kernel", default="transform2d", help="regular expression on the kernel name")
    ap.add_argument("--command", required=True, help="the ncu command line that wrote the CSV")
    ap.add_argument("--unit", required=True, help="translation unit of the kernel, relative to csrc/")
    ap.add_argument("--header", action="append", default=[],
                    help="a further header the kernel is defined in, relative to csrc/ (repeatable)")
    a = ap.parse_args()
    entry = summarise(parse_launches(a.csv, a.kernel))
    entry["sources"] = sorted(set(DEVICE_HEADERS + a.header + [a.unit]))
    entry["source_hash"] = source_hash(entry["sources"])
    entry["command"] = a.command
    data = json.load(open(TRAFFIC)) if os.path.exists(TRAFFIC) else {}
    data[a.key] = entry
    with open(TRAFFIC, "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")
    print(a.key, entry)


if __name__ == "__main__":
    main()
