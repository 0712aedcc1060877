"""Host logic of bench.py's roofline fields (no GPU): the DRAM traffic figure is
taken from the committed ncu summary only while the kernel sources match the
hash recorded beside it, and the CSR-equivalent roofline arithmetic."""
import hashlib
import os
import re

import pytest

import bench


def test_series_traffic_matches_committed_summary():
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    text = open(os.path.join(bench.ROOT, "profiles", "series_kernel_er1000.md")).read()
    recorded = re.search(r"kernel sources sha256: ([0-9a-f]{64})", text).group(1)
    bytes_ = int(re.search(r"dram bytes per full launch: ([0-9]+)", text).group(1))
    if recorded == h.hexdigest():
        assert bench.series_traffic() == bytes_
        # the figure is the read + write rows of the same summary
        rows = {m.group(1): int(m.group(2).replace(",", ""))
                for m in re.finditer(r"\| (dram__bytes_(?:read|write)\.sum) \| ([0-9,]+) \|", text)}
        assert rows["dram__bytes_read.sum"] + rows["dram__bytes_write.sum"] == bytes_
    else:
        assert bench.series_traffic() is None


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
