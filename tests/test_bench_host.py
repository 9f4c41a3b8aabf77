"""Host-side logic of bench.py: the roofline figure from the library's per-class profile, and the
DRAM traffic read from the committed ncu summaries (bytes per spinor-gridpoint unit scaled to the
launch, plus a per-launch constant for tables that every launch reads once)."""
import os

import pytest

import bench


def _write(tmp_path, name, text):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / name).write_text(text)


def test_measured_traffic_scales_per_unit_and_adds_the_constant(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda cls: "abc")
    _write(tmp_path, "traffic_epilogue_w.txt",
           "# title\n\nkernel_class: epilogue\nsource_sha256: abc\ndram_bytes_per_unit: 2.5\n"
           "dram_bytes_per_launch_const: 1000\n")
    value, src = bench.measured_traffic("epilogue", "w", 400)
    assert value == pytest.approx(2.5 * 400 + 1000) and src == "traffic_epilogue_w.txt"
    # without the constant the per-unit part alone
    _write(tmp_path, "traffic_fft_xy_w.txt", "source_sha256: abc\ndram_bytes_per_unit: 32\n")
    assert bench.measured_traffic("fft_xy", "w", 10)[0] == pytest.approx(320.0)


def test_measured_traffic_is_dropped_when_stale_or_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda cls: "new")
    _write(tmp_path, "traffic_epilogue_w.txt", "source_sha256: old\ndram_bytes_per_unit: 2.5\n")
    value, why = bench.measured_traffic("epilogue", "w", 400)
    assert value is None and "changed" in why
    value, why = bench.measured_traffic("proj_gather", "w", 400)
    assert value is None and "no ncu summary" in why


def test_roofline_picks_the_dominant_class(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = {"fft_xy": {"ms": 10.0, "launches": 4, "bytes": 4e9},
            "epilogue": {"ms": 30.0, "launches": 3, "bytes": 6e10}}
    r = bench.roofline_of(prof, 1000, "w")
    assert r["kernel"] == "epilogue"
    assert r["avg_launch_ms"] == pytest.approx(10.0)
    assert r["achieved"] == pytest.approx(2e10 / 1e-2 / 1e9)  # GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["share"] == pytest.approx(0.75)


def test_committed_traffic_summaries_match_the_kernel_sources():
    """The committed summaries belong to the kernels in the tree (bench.py would drop them
    otherwise), and carry the keys bench.py reads."""
    pdir = os.path.join(bench.ROOT, "profiles")
    files = [f for f in os.listdir(pdir) if f.startswith("traffic_") and f.endswith(".txt")]
    assert files
    for f in files:
        kv = {}
        for line in open(os.path.join(pdir, f)):
            if ":" in line and not line.startswith((" ", "#")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        assert float(kv["dram_bytes_per_unit"]) > 0
        assert kv["source_sha256"] == bench.kernel_source_hash(kv["kernel_class"]), f
