"""CPU tests of bench.py's helpers: the roofline's DRAM traffic is taken from an
ncu summary only while that summary's digest matches the stochastic step's
sources, and the measured peaks load from their file."""
import bench


def _summary(tmp_path, digest, nbytes=123456):
    p = tmp_path / "k.md"
    p.write_text(f"# summary\n\n- `dram_bytes_per_launch: {nbytes}`\n- `sources_sha256: {digest}`\n")
    return str(p)


def test_traffic_read_while_sources_match(tmp_path):
    assert bench.profiled_traffic(_summary(tmp_path, bench.kernel_sources_digest())) == 123456.0


def test_traffic_dropped_when_sources_changed(tmp_path):
    assert bench.profiled_traffic(_summary(tmp_path, "0" * 64)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md")) is None


def test_digest_covers_the_stochastic_step_sources_only():
    assert "ssa.cu" in bench.SSA_SOURCES and "ssa_device.cuh" in bench.SSA_SOURCES
    assert not any(s.startswith("general") or s.startswith("events") for s in bench.SSA_SOURCES)
    assert len(bench.kernel_sources_digest()) == 64


def test_measured_peaks_is_a_mapping():
    assert isinstance(bench.measured_peaks(), dict)
