"""The ncu launch-list reader that records per-launch DRAM traffic."""
import json
import os

from paper_2508_07071_gb300 import ncu_traffic as T

HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
        '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","7","(8, 16, 1)","(5, 40, 256)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"\n')


def test_parse_and_summarise(tmp_path):
    lines = ["==PROF== Connected to process 1\n", HEAD]
    for i, (rd, wr, t) in enumerate([(100, 50, 2000), (300, 150, 4000)]):
        k = "void transform2d_kernel<16, 1, X>(Args2D<T3, T4, T5>)"
        lines += [row(i, k, "dram__bytes_read.sum", "byte", rd), row(i, k, "dram__bytes_write.sum", "byte", wr),
                  row(i, k, "gpu__time_duration.sum", "ns", f"{t:,}")]
    lines += [row(2, "void other_kernel()", "dram__bytes_read.sum", "byte", 9),
              row(2, "void other_kernel()", "dram__bytes_write.sum", "byte", 9),
              row(2, "void other_kernel()", "gpu__time_duration.sum", "ns", 9)]
    p = tmp_path / "l.csv"
    p.write_text("".join(lines))
    s = T.summarise(T.parse_launches(str(p), "transform2d"))
    assert s == {"dram_bytes_per_launch": 300, "dram_read_bytes": 200, "dram_write_bytes": 100,
                 "launches": 2, "mean_time_us_cold_serialised": 3.0}


def test_source_hash_is_stable_and_short():
    a, b = T.source_hash(), T.source_hash()
    assert a == b and len(a) == 16 and int(a, 16) >= 0
    part = T.source_hash(T.DEVICE_HEADERS + ["k_nv12_bf16.cu"])
    assert part != a and part == T.entry_hash({"sources": T.DEVICE_HEADERS + ["k_nv12_bf16.cu"]})
    assert T.entry_hash({}) == a  # an entry without a source list hashes everything


def test_committed_traffic_file_is_well_formed():
    d = json.load(open(T.TRAFFIC))
    for key, e in d.items():
        # the total and the parts are rounded separately
        assert abs(e["dram_bytes_per_launch"] - e["dram_read_bytes"] - e["dram_write_bytes"]) <= 2, key
        assert len(e["source_hash"]) == 16 and e["command"].startswith("ncu ")
        for rel in e.get("sources", []):
            assert os.path.exists(os.path.join(T.PKG, "csrc", rel)), rel


def test_cli_records_the_kernel_headers(tmp_path, monkeypatch):
    """--header adds the files a kernel is defined in to the hashed sources."""
    import sys
    k = "void fkl::reduce2d_kernel<16, 0, X>(ReduceArgs<T3, T4>)"
    lines = [HEAD, row(0, k, "dram__bytes_read.sum", "byte", 400), row(0, k, "dram__bytes_write.sum", "byte", 4),
             row(0, k, "gpu__time_duration.sum", "ns", "1,000")]
    csv_path = tmp_path / "l.csv"
    csv_path.write_text("".join(lines))
    out = tmp_path / "traffic.json"
    out.write_text('{"other": {"kept": true}}')
    monkeypatch.setattr(T, "TRAFFIC", str(out))
    monkeypatch.setattr(sys, "argv", ["ncu_traffic", "--csv", str(csv_path), "--key", "r", "--kernel", "reduce2d",
                                      "--unit", "k_reduce.cu", "--header", "fkl/reduce.cuh",
                                      "--command", "ncu --metrics x"])
    T.main()
    d = json.load(open(out))
    assert d["other"] == {"kept": True}                      # other entries survive
    e = d["r"]
    assert e["dram_bytes_per_launch"] == 404 and e["launches"] == 1
    assert "fkl/reduce.cuh" in e["sources"] and "k_reduce.cu" in e["sources"]
    assert set(T.DEVICE_HEADERS) <= set(e["sources"])
    assert e["source_hash"] == T.entry_hash(e)
    assert e["source_hash"] != T.source_hash([s for s in e["sources"] if s != "fkl/reduce.cuh"])
