"""Host logic of bench.py that decides what the JSON line reports (no GPU): the per-launch DRAM
traffic is taken from the committed ncu summary only while it was captured on the current kernel
sources, and the algorithmic flop counts add up as stated."""
import os

import bench


def _traffic_file(tmp_path, lines):
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "traffic_per_launch.txt").write_text("# header\n" + "\n".join(lines) + "\n")


def test_recorded_traffic_needs_the_current_sources(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha()
    _traffic_file(tmp_path, [
        f"kernel=element_update form=fp64 variant=3 workload=w elements=1000 bytes=300000 src_sha={sha}",
        "kernel=element_update form=fp64 variant=1 workload=w elements=1000 bytes=999 src_sha=0000000000000000",
        f"kernel=limiter_wetdry form=mixed variant=* workload=w elements=2000 bytes=100000 src_sha={sha}",
    ])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    assert bench.recorded_traffic("element_update", "fp64", 1000, 3) == 300000   # the captured mesh
    assert bench.recorded_traffic("element_update", "fp64", 2000, 3) is None     # another mesh size
    assert bench.recorded_traffic("element_update", "fp64", 2000, 3, scale=True) == 600000  # per element
    assert bench.recorded_traffic("element_update", "fp64", 1000, 3, p=2) is None  # another degree
    assert bench.recorded_traffic("element_update", "fp64", 1000, 1) is None     # stale sources
    assert bench.recorded_traffic("element_update", "mixed", 1000, 3) is None    # other form
    assert bench.recorded_traffic("limiter_wetdry", "mixed", 2000, 4) == 100000  # any variant
    assert bench.recorded_traffic("edge_flux", "fp64", 1000, 1) is None


def test_ensemble_traffic_follows_the_launch_mode(tmp_path, monkeypatch):
    """The ensemble's line is a whole step of a smaller batch, scaled per element-stage, and is
    taken only for the launch mode it was captured in."""
    sha = bench.kernel_source_sha()
    _traffic_file(tmp_path, [
        f"kernel=ensemble_step form=mixed variant=persistent p=1 workload=w elements=1000 bytes=800000 src_sha={sha}",
        f"kernel=ensemble_step form=mixed variant=phased p=1 workload=w elements=1000 bytes=700000 src_sha={sha}",
    ])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    assert bench.recorded_traffic("ensemble_step", "mixed", 3000, "persistent", scale=True) == 2400000
    assert bench.recorded_traffic("ensemble_step", "mixed", 3000, "phased", scale=True) == 2100000
    assert bench.recorded_traffic("ensemble_step", "mixed", 3000, "phased") is None  # unscaled: other size


def test_recorded_traffic_without_a_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("element_update", "fp64", 1000, 3) is None


def test_kernel_source_sha_covers_the_device_sources():
    csrc = os.path.join(bench.ROOT, "paper_2508_21208_gb300", "csrc")
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and int(sha, 16) >= 0
    for f in ("kernels.cuh", "kernels_f64.cu", "kernels_f32.cu", "common_kernels.cu", "internal.h", "mesh.cu"):
        assert os.path.exists(os.path.join(csrc, f))


def test_algorithmic_counts():
    # split element kernel 514 flop, edge kernel 172 per edge at 1.5 edges per element: 772 fused
    assert bench.ALG_FLOPS_ELEMENT_P1 == 514 and bench.ALG_FLOPS_EDGE_P1 == 172
    assert bench.ALG_FLOPS_ELEMENT_P1 + 1.5 * bench.ALG_FLOPS_EDGE_P1 == 772
    assert bench.ALG_BYTES[("fp64", 1)] == 72 + 36 + 72 + 64 + 14 + 51
    assert bench.kernel_timed_steps(100) == 10 and bench.kernel_timed_steps(1) == 1
    name, mean_ms, tot = bench.dominant({"a": [1.0, 3.0], "b": [1.5]})
    assert name == "a" and mean_ms == 2.0e-3 and tot == {"a": 4.0, "b": 1.5}
