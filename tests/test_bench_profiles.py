"""bench.py's roofline fields that come from the committed ncu summary: the
DRAM traffic per launch and the L1 data-pipe utilisation are reported only
while the fitness kernel's sources are the ones that capture was taken on."""
import bench


def test_committed_capture_matches_the_current_kernel_sources():
    traffic = bench.committed_traffic()
    l1 = bench.committed_l1_pipe()
    assert isinstance(traffic, int) and traffic > 0
    assert l1 is not None
    assert 0.0 < l1["points_on_lanes"] <= 1.0 and 0.0 < l1["particles_on_lanes"] <= 1.0


def test_capture_figures_are_dropped_when_the_kernel_changes(monkeypatch):
    monkeypatch.setattr(bench, "fitness_source_sha", lambda: "0000000000000000")
    assert bench.committed_traffic() is None
    assert bench.committed_l1_pipe() is None


def test_derived_fp32_peak():
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
    assert abs(bench.fp32_peak_tflops() - 80.54784) < 1e-9
