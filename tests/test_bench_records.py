"""Host logic of the bench line's rooflines: the committed ncu record of the
collide-stream is used only when it was taken on the current kernel sources
and storage, scaled by sites, and the issue-slot roofline follows from its
instruction count, the live launch time and the SM count and clock."""
import json

import pytest

import bench


def _record(tmp_path, monkeypatch, source_sha256):
    """A record taken on sources hashing to source_sha256; the current sources
    hash to "current"."""
    rec = {"kernel": "lb3_kernel<float, 0, 1>", "storage": 0, "sites": 1000, "dram_bytes_per_launch": 158000,
           "warp_inst_per_launch": 36000, "source_sha256": source_sha256}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "lb_kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "lb_source_sha", lambda: "current")


def test_record_scales_traffic_by_sites(tmp_path, monkeypatch):
    _record(tmp_path, monkeypatch, source_sha256="current")
    assert bench.lb_traffic(0, 4000) == pytest.approx(4 * 158000)


def test_stale_or_other_storage_record_is_not_used(tmp_path, monkeypatch):
    _record(tmp_path, monkeypatch, source_sha256="older sources")
    assert bench.lb_traffic(0, 1000) is None
    assert bench.lb_issue_roofline(0, 1000, 1.0, 152, 2070.0) is None
    monkeypatch.setattr(bench, "lb_source_sha", lambda: "older sources")
    assert bench.lb_traffic(0, 1000) == pytest.approx(158000)
    assert bench.lb_traffic(1, 1000) is None  # the record is of FP32 storage


def test_issue_roofline_arithmetic(tmp_path, monkeypatch):
    _record(tmp_path, monkeypatch, source_sha256="current")
    # 36000 warp instructions per 1000 sites: 1152 thread instructions per site
    r = bench.lb_issue_roofline(0, 2000, 0.5, 152, 2070.0)
    achieved = 32 * 72000 / 0.5e-3 / 1e12
    peak = 152 * 4 * 32 * 2070e6 / 1e12
    assert r["bound"] == "alu" and r["inst_per_site"] == pytest.approx(1152)
    assert r["achieved"] == pytest.approx(achieved) and r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(achieved / peak)
    assert bench.lb_issue_roofline(0, 2000, 0.0, 152, 2070.0) is None  # no launch time
