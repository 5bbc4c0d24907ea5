"""The bench's reading of an ncu raw-page CSV into per-image DRAM traffic (host logic, no GPU)."""

import json

import bench


def _raw_csv(path):
    # header row, unit row, one row per captured launch (the layout ncu's raw page prints)
    rows = [
        ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"],
        ["", "", "Mbyte", "Kbyte", "usecond"],
        ["0", "void k_grid_cells<0, 1, 0>(SegmentGeom, ...)", "185.5", "15,400", "53.3"],
        ["1", "void k_colfft<1024>(SegmentGeom, ...)", "30.9", "662,600", "166.5"],
        ["2", "void k_rowfft_stats<1024, 0>(SegmentGeom, ...)", "723.6", "7,000", "225.4"],
        ["3", "void k_rowfft_stats<1024, 0>(SegmentGeom, ...)", "0.7236", "7", "225.4"],
    ]
    with open(path, "w") as f:
        for r in rows:
            f.write(",".join('"%s"' % c for c in r) + "\n")


def test_write_traffic_units_averages_and_hash(tmp_path):
    raw = tmp_path / "raw.csv"
    out = tmp_path / "traffic.json"
    _raw_csv(raw)
    doc = bench.write_traffic(str(raw), 256, "ncu ...", "realtime", path=str(out))
    k = json.load(open(out))["kernels"]
    assert doc["source_hash"] == bench.source_hash()
    # Mbyte and Kbyte are decimal units; thousands separators are dropped
    assert k["grid_cells"]["dram_bytes_per_launch"] == 185.5e6 + 15.4e6
    assert k["grid_colfft"]["dram_bytes_per_image"] == (30.9e6 + 662.6e6) / 256
    # two captured launches of one kernel are averaged
    rs = k["rowfft_stats"]
    assert rs["launches_captured"] == 2
    assert abs(rs["dram_bytes_per_launch"] - (723.6e6 + 7e6 + 0.7236e6 + 7e3) / 2) < 1e-3


def test_traffic_is_taken_only_for_matching_sources(tmp_path, monkeypatch):
    import os
    raw = tmp_path / "raw.csv"
    _raw_csv(raw)
    prof = tmp_path / "profiles"
    prof.mkdir()
    bench.write_traffic(str(raw), 256, "ncu ...", "realtime", path=str(prof / "traffic.json"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the committed kernel sources are read from ROOT too: point them at a copy
    csrc = tmp_path / "paper_1802_03084_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "paper_1802_03084_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_bytes(open(os.path.join(src, name), "rb").read())
    assert bench.load_traffic("rowfft_stats", 1000) is not None
    (csrc / bench.KERNEL_SOURCES[0]).write_bytes(b"changed")
    assert bench.load_traffic("rowfft_stats", 1000) is None


def test_write_traffic_reads_concatenated_logs_with_ncu_notes(tmp_path):
    # one ncu log file per kernel, concatenated: each starts with ncu's one-field
    # notes and repeats the header and unit rows; only launch rows count
    parts = []
    for i in range(2):
        one = tmp_path / f"k{i}.csv"
        _raw_csv(one)
        parts.append("==WARNING== Note: a profiler note\n==PROF== Connected to process 1\n" + one.read_text())
    raw = tmp_path / "all.csv"
    raw.write_text("".join(parts))
    doc = bench.write_traffic(str(raw), 256, "ncu ...", "realtime", path=str(tmp_path / "traffic.json"))
    k = doc["kernels"]
    assert k["grid_cells"]["launches_captured"] == 2
    assert k["grid_cells"]["dram_bytes_per_launch"] == 185.5e6 + 15.4e6
    assert k["rowfft_stats"]["launches_captured"] == 4
