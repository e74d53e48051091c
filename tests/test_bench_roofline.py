"""bench.py's roofline bookkeeping on CPU: the DRAM traffic figures of the
committed ncu summary apply only to the workload they were taken on and
only while the smoother sources hash to the recorded value."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_only_for_its_workload():
    for form in ("fp64", "mixed"):
        t = bench.traffic_per_launch("vel_smooth_colour_l0", form, bench.TRAFFIC_WORKLOAD)
        assert t is None or t > 0
        assert bench.traffic_per_launch("vel_smooth_colour_l0", form, "bubble_2d_r100_steady_512^2") is None
    assert bench.traffic_per_launch("no_such_family", "fp64", bench.TRAFFIC_WORKLOAD) is None


def test_roofline_alu_and_hbm_fractions():
    fams = [{"name": "vel_smooth_colour_l0", "launches": 10, "ms": 0.4, "bytes": 10 * 134217728.0,
             "flops": 10 * 25165824.0},
            {"name": "vel_residual", "launches": 2, "ms": 0.1, "bytes": 2e8, "flops": 0.0}]
    peaks = {"hbm_gbs": 6790.3}
    r = bench.roofline_of(fams, "fp64", peaks, workload="other")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] is None
    assert abs(r["achieved"] - 10 * 25165824.0 / 0.4e-3 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    m = bench.roofline_of(fams, "mixed", peaks, "vel_smooth_colour_l0", "other")
    assert m["bound"] == "hbm" and m["peak"] == 6790.3
    assert abs(m["achieved"] - 10 * 134217728.0 / 0.4e-3 / 1e9) < 1e-9


def test_dominant_kernel_is_one_kernel_configuration():
    """A family that pools launches on every grid size (the smoothers below
    the finest level) is not the dominant kernel even with the most time."""
    fams = [{"name": "vel_smooth_colour", "launches": 900, "ms": 9.0, "bytes": 1e9, "flops": 1e9},
            {"name": "vel_smooth_colour_l0", "launches": 200, "ms": 8.0, "bytes": 2e10, "flops": 4e9},
            {"name": "arnoldi_update", "launches": 100, "ms": 5.0, "bytes": 2e10, "flops": 0.0}]
    r = bench.roofline_of(fams, "fp64", {"hbm_gbs": 6790.3}, workload="other")
    assert r["kernel"] == "vel_smooth_colour_l0"


def test_traffic_dropped_once_the_sources_change(tmp_path, monkeypatch):
    """A traffic line counts only while stencil.cuh + kernels.cu + pair.cu
    hash to its recorded `sources` value: editing any of them makes the
    figure null until the counters are taken again."""
    import hashlib
    csrc = tmp_path / "paper_1308_4605_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    files = {"stencil.cuh": b"// stencils\n", "kernels.cu": b"// kernels\n", "pair.cu": b"// pairs\n"}
    for name, text in files.items():
        (csrc / name).write_bytes(text)
    h = hashlib.sha256()
    for name in ("stencil.cuh", "kernels.cu", "pair.cu"):
        h.update(files[name])
    src = h.hexdigest()[:16]
    (tmp_path / "profiles" / "kernels_3d_unsteady_periodic_128.md").write_text(
        f"traffic: vel_smooth_colour_l0 fp64 143510016 sources {src}\n"
        f"traffic: vel_smooth_colour_l0 mixed 67484416 sources 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    w = bench.TRAFFIC_WORKLOAD
    assert bench.traffic_per_launch("vel_smooth_colour_l0", "fp64", w) == 143510016.0
    assert bench.traffic_per_launch("vel_smooth_colour_l0", "mixed", w) is None   # other sources
    (csrc / "kernels.cu").write_bytes(b"// kernels, edited\n")
    assert bench.traffic_per_launch("vel_smooth_colour_l0", "fp64", w) is None
