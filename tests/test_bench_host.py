"""Host-side logic of bench.py that needs no GPU: the committed ncu figures
are used only while they describe the current kernel source, and the gather
byte counts follow from the stencil widths."""
import os
import shutil

import pytest

import bench


def test_recorded_profiles_match_the_current_kernel():
    for scheme in ("bilinear", "catmull_rom"):
        prof = bench.recorded_profile(scheme)
        assert prof, scheme
        per = (float(prof["dram_bytes_read"]) + float(prof["dram_bytes_write"])) / float(prof["particles"])
        assert abs(per - bench.recorded_traffic(scheme)) < 0.01
        assert 0.0 < float(prof["lts_throughput_pct"]) < 100.0


def test_a_stale_profile_is_ignored(tmp_path, monkeypatch):
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    src = os.path.join(bench.ROOT, "profiles", "k_rk4_bilinear_traffic.txt")
    text = open(src).read().replace("source_hash=", "source_hash=0")
    (prof_dir / "k_rk4_bilinear_traffic.txt").write_text(text)
    for rel in ("paper_2607_17836_b300/csrc",):
        shutil.copytree(os.path.join(bench.ROOT, rel), tmp_path / rel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_profile("bilinear") == {}
    assert bench.recorded_traffic("bilinear") is None
    assert bench.recorded_profile("bspline") == {}


def test_gather_bytes():
    # 6 snapshot evaluations of W x W nodes of (u, v) FP32, or one 16-byte
    # level pair per node
    assert bench.GATHER_PLAIN == {0: 192, 1: 768, 2: 768}
    assert bench.GATHER_CACHED == {0: 64, 1: 256, 2: 256}


def test_oracle_timing_of_the_taylor_green_case_in_full():
    t = bench.cpu_oracle_config1()
    assert t["seconds"] > 0 and t["cores"] >= 1
    assert t["particle_steps_per_s"] == pytest.approx(4096 * 200 / t["seconds"])
    assert t["fluid_steps_per_s"] > t["particle_steps_per_s"] / 4096
