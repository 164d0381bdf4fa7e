"""Host-side pieces of bench.py that feed the bench line: the build's
bandwidth figure and the gating of the DRAM-traffic figure on the source
of the sweep kernels it was measured on (no GPU needed)."""
import hashlib
import os

import bench


def test_build_rate_counts_bytes_per_build():
    st = {"builds": 2, "build_ms": [1.0] * 8}
    r = bench.build_rate(st, 1000, {"hbm_gbs": 1000.0}, "measured")
    alg = 1000 * 44 + 2 * 13 * 8 * 1000
    assert r["algorithmic_bytes"] == alg
    assert abs(r["ms_per_build"] - 4.0) < 1e-12       # 8 ms over two builds
    assert abs(r["achieved_gbs"] - alg / 4e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved_gbs"] / 1000.0) < 1e-12


def test_traffic_is_withheld_when_the_sweep_source_changed(tmp_path, monkeypatch):
    root = tmp_path
    (root / "paper_1404_2303_gb300" / "csrc").mkdir(parents=True)
    (root / "profiles").mkdir()
    src = root / "paper_1404_2303_gb300" / "csrc" / "sweep.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (root / "profiles" / "traffic_sweeps_lognormal128.md").write_text(
        f"kernel_source_sha256: {sha}\ntraffic_bytes_per_unit[density]: 10.0\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("density", 3.0) == 30.0
    assert bench.profiled_traffic("force", 3.0) is None          # no figure for that phase
    src.write_text("// kernel source, edited\n")
    assert bench.profiled_traffic("density", 3.0) is None         # stale counters

