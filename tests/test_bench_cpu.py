"""Host logic of bench.py's roofline reporting (no GPU): the algorithmic
bytes of a batch, the traffic figure and the issue roofline, and that both
measured figures are withheld once the kernel sources differ from the
captured ones."""
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.syspath_prepend(ROOT)
    import bench as b

    return b


def test_algorithmic_bytes(bench):
    # input bytes + interior code bytes + 4-byte histogram words per image
    assert bench.algorithmic_bytes([490], [640], 2352) == 490 * 640 + 488 * 638 + 2352 * 4
    assert bench.algorithmic_bytes([3, 10], [5, 4], 0) == 15 + 40 + 1 * 3 + 8 * 2


def test_measured_figures_follow_the_sources(bench, monkeypatch):
    px = 4096 * 640 * 490
    monkeypatch.setattr(bench, "sources_match", lambda: True)
    t = bench.measured_traffic(px, 3, 490, 640)
    assert t == int(round(bench.TRAFFIC_PER_PX * px))
    r = bench.issue_roofline(px, 3, 490, 640, 2.0, 152, 2070.0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 4 * 32 * 2070e6 / 1e12, rel=1e-3)
    assert r["achieved"] == pytest.approx(bench.ISSUE_SLOTS_PER_PX * px / 2.0e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    # another workload or tile variant, or no clock sample: no figure
    assert bench.measured_traffic(px, 2, 490, 640) is None
    assert bench.measured_traffic(px, 3, 490, 640, "r8w4b6t0") is None
    assert bench.issue_roofline(px, 3, 490, 640, 2.0, 152, 2070.0, "r8w4b6t0") is None
    assert bench.issue_roofline(px, 3, 480, 640, 2.0, 152, 2070.0) is None
    assert bench.issue_roofline(px, 3, 490, 640, 2.0, 152, None) is None
    # kernel sources changed since the capture: both withheld
    monkeypatch.setattr(bench, "sources_match", lambda: False)
    assert bench.measured_traffic(px, 3, 490, 640) is None
    assert bench.issue_roofline(px, 3, 490, 640, 2.0, 152, 2070.0) is None


def test_source_hash_covers_the_kernel_files(bench, tmp_path, monkeypatch):
    files = [os.path.join(ROOT, f) for f in bench.TRAFFIC_SOURCES]
    assert all(os.path.exists(f) for f in files)
    # a copy of the tree with one byte changed in a kernel file no longer matches
    for f in bench.TRAFFIC_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    with open(tmp_path / bench.TRAFFIC_SOURCES[0], "ab") as fh:
        fh.write(b"\n")
    assert bench.sources_match() is False
