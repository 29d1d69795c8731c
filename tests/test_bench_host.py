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


def test_profile_commands_name_existing_bench_modes():
    """Every `bench.py --profile-launch X` (and `--scheme`, `--gather`) that
    a committed ncu summary cites is one the benchmark still accepts, so the
    summaries' commands stay runnable."""
    import re
    src = open(os.path.join(os.path.dirname(bench.__file__), "bench.py")).read()
    modes = set(re.search(r'"--profile-launch", choices=\[([^\]]*)\]', src).group(1).replace('"', "").replace(" ", "").split(","))
    gathers = set(re.search(r'"--gather", choices=\[([^\]]*)\]', src).group(1).replace('"', "").replace(" ", "").split(","))
    prof = os.path.join(os.path.dirname(bench.__file__), "profiles")
    cited = 0
    for name in sorted(os.listdir(prof)):
        text = open(os.path.join(prof, name)).read().replace("\\\n", " ")
        for m in re.finditer(r"bench\.py([^\n]*)", text):
            args = m.group(1)
            for mode in re.findall(r"--profile-launch (\S+)", args):
                assert mode in modes, (name, mode)
                cited += 1
            for scheme in re.findall(r"--scheme (\S+)", args):
                assert scheme in bench.SCHEMES, (name, scheme)
            for gather in re.findall(r"--gather (\S+)", args):
                assert gather in gathers, (name, gather)
    assert cited >= 5
