"""Host logic of bench.py's roofline fields (no GPU): the DRAM traffic figure is
taken from the committed record (written by `bench.py --record-traffic` from an
ncu CSV) only while the kernel sources match the hash recorded in it, and the
CSR-equivalent roofline arithmetic."""
import hashlib
import os
import re

import pytest

import bench


def test_series_traffic_matches_committed_record():
    import json
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    rec = json.load(open(bench.TRAFFIC_RECORD))
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    # the markdown summary quotes the same capture
    text = open(os.path.join(bench.ROOT, "profiles", "series_kernel_er1000.md")).read()
    assert re.search(r"kernel sources sha256: ([0-9a-f]{64})", text).group(1) == \
        rec["kernel_sources_sha256"]
    rows = {m.group(1): int(m.group(2).replace(",", ""))
            for m in re.finditer(r"\| (dram__bytes_(?:read|write)\.sum) \| ([0-9,]+) \|", text)}
    assert rows["dram__bytes_read.sum"] == rec["dram_bytes_read"]
    assert rows["dram__bytes_write.sum"] == rec["dram_bytes_write"]
    if rec["kernel_sources_sha256"] == h.hexdigest():
        assert bench.series_traffic() == rec["dram_bytes_per_launch"]
    else:
        assert bench.series_traffic() is None


def test_record_traffic_parses_ncu_csv(tmp_path, monkeypatch):
    # an ncu --csv log in the format ncu writes (units ns and byte), with a
    # launch of another kernel first
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"\n')
    def row(i, k, m, u, v):
        return (f'"{i}","1","python3","h","{k}","1","7","(256, 1, 1)","(608, 1, 1)","0","10.3",'
                f'"Command line profiler metrics","{m}","{u}","{v}"\n')
    text = ("==PROF== noise line\n" + head +
            row(0, "qsw::other_kernel(int)", "gpu__time_duration.sum", "ns", "5,000") +
            row(1, "void qsw::series_kernel<double2, 2, 1>(SeriesArgs)", "dram__bytes_read.sum", "byte", "1,000") +
            row(1, "void qsw::series_kernel<double2, 2, 1>(SeriesArgs)", "dram__bytes_write.sum", "byte", "2,500") +
            row(1, "void qsw::series_kernel<double2, 2, 1>(SeriesArgs)", "gpu__time_duration.sum", "ns", "88,000,000"))
    csv_path = tmp_path / "t.csv"
    csv_path.write_text(text)
    out = tmp_path / "rec.json"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(out))
    bench.record_traffic(str(csv_path), "cmd")
    import json
    rec = json.load(open(out))
    assert rec["dram_bytes_per_launch"] == 3500
    assert rec["gpu_time_duration_ms"] == pytest.approx(88.0)
    assert bench.series_traffic() == 3500


def test_series_traffic_is_none_when_sources_change(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// a different kernel source\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [str(src)])
    assert bench.series_traffic() is None


def test_csr_equivalent_arithmetic():
    # 10 rows, 30 entries: 30 * 20 + 11 * 4 + 4 * 10 * 16 bytes per application
    r = bench.csr_equivalent(30, 10, 1.0, 2.0, 4)
    assert r["csr_bytes_per_application"] == 30 * 20 + 11 * 4 + 640
    assert r["csr_at_hbm_peak_ms"] == pytest.approx(1284 / 1e9 * 1e3)
    assert r["ms_per_application"] == pytest.approx(0.5)
    assert r["ratio"] == pytest.approx(r["csr_at_hbm_peak_ms"] / 0.5)
